"""The allocation-free SVD entry point (pt_svd_f64_noalloc) against pt_svd_f64.

pt_svd_f64_noalloc serves callers that cannot allocate device memory (their memory is owned by
another pool, or a device allocation is not acceptable where they run): it runs the same batched
FP64 Jacobi SVD with its workspace in the library's static device array. These checks call both
entry points through the C ABI on the same inputs, twice in a row with different shapes (the
shared workspace keeps the previous call's contents), and require the same results within the
tolerance of the other SVD tests. This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05529_gb300 as pkg
    pkg.build()
    return pkg.load()


def _run(capi, A, noalloc):
    import torch
    b, m, n = A.shape
    k = min(m, n)
    dA = torch.from_numpy(A).cuda()
    s = torch.zeros((b, k), dtype=torch.float64, device="cuda")
    U = torch.zeros((b, m, k), dtype=torch.complex128, device="cuda")
    V = torch.zeros((b, n, k), dtype=torch.complex128, device="cuda")
    if noalloc:
        capi.svd_f64_noalloc(dA, s, U, V)
    else:
        scr = torch.zeros(capi.svd_scratch_bytes(m, n, b), dtype=torch.uint8, device="cuda")
        capi.svd_f64(dA, s, U, V, scr)
    torch.cuda.synchronize()
    return s.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()


def test_noalloc_svd_matches_the_allocating_entry_point_twice(capi):
    rng = np.random.default_rng(11)
    for (m, n, b) in [(48, 30, 3), (20, 72, 2)]:        # second call: a different, wide shape
        A = rng.standard_normal((b, m, n)) + 1j * rng.standard_normal((b, m, n))
        s0, U0, V0 = _run(capi, A, noalloc=False)
        s1, U1, V1 = _run(capi, A, noalloc=True)
        for i in range(b):
            tol = 1e-12 * s0[i][0] * max(m, n)
            assert np.max(np.abs(s1[i] - s0[i])) < tol
            # singular vectors are unique up to a phase per column: compare the projectors' action
            rec0 = (U0[i] * s0[i][None, :]) @ V0[i].conj().T
            rec1 = (U1[i] * s1[i][None, :]) @ V1[i].conj().T
            assert np.max(np.abs(rec1 - rec0)) < tol
            assert np.max(np.abs(rec1 - A[i])) < tol
            k = min(m, n)
            assert np.max(np.abs(U1[i].conj().T @ U1[i] - np.eye(k))) < 1e-12 * max(m, n)


def test_noalloc_rejects_a_problem_larger_than_its_static_workspace(capi):
    import ctypes as C
    need = capi.svd_scratch_bytes(2048, 2048, 1)
    assert need > capi.NOALLOC_MAX_BYTES
    rc = capi.lib.pt_svd_f64_noalloc(C.c_void_p(1), 2048, 2048, 1, C.c_void_p(1), C.c_void_p(1),
                                     C.c_void_p(1), 0, None)
    assert rc == -3
    assert b"static array" in capi.lib.pt_tebd_last_error(None)
