"""The whole-GPU Householder QR (explicit Q) of the outer-block reductions (App. A.2) and of the
fast path's range finder, through pt_qr_f64, against the definition: A = Q R with orthonormal Q and
upper-triangular R, to FP64 accuracy (|A - QR| and |Q^H Q - I| within 1e-13 x m of the scale).
Shapes: single columns, square, tall, tiny blocks of the outer reductions (6 x 4), sizes spanning
several 32-row lane strides with ragged tails, a rank-deficient block and an all-zero column."""
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
    c = pkg.load()
    c.use_torch_allocator()
    return c


@pytest.mark.parametrize("m,n,batch", [(1, 1, 1), (6, 4, 5), (5, 5, 2), (33, 32, 3), (200, 3, 4),
                                       (300, 37, 6), (2048, 160, 10), (129, 128, 2)])
def test_householder_qr_against_definition(capi, m, n, batch):
    import torch
    rng = np.random.default_rng(m * 7 + n)
    A = rng.standard_normal((batch, m, n)) + 1j * rng.standard_normal((batch, m, n))
    A[0] *= 10.0 ** rng.uniform(-8, 4, size=n)[None, :]      # graded columns
    if batch > 1 and n > 2:
        A[1][:, 2] = A[1][:, 0] + A[1][:, 1]                  # rank-deficient
    if batch > 2 and n > 1:
        A[2][:, 1] = 0.0                                      # a zero column
    At = torch.from_numpy(np.ascontiguousarray(A.transpose(0, 2, 1))).cuda()
    Rt = torch.zeros((batch, n, n), dtype=torch.complex128, device="cuda")
    scratch = torch.empty(capi.qr_scratch_bytes(m, n, batch), dtype=torch.uint8, device="cuda")
    capi.qr_f64(At, Rt, scratch)
    torch.cuda.synchronize()
    Q = At.cpu().numpy().transpose(0, 2, 1)
    R = Rt.cpu().numpy().transpose(0, 2, 1)
    for b in range(batch):
        scale = max(1.0, float(np.abs(A[b]).max()))
        assert np.allclose(np.tril(R[b], -1), 0.0)
        assert np.abs(Q[b] @ R[b] - A[b]).max() <= 1e-13 * m * scale
        assert np.abs(Q[b].conj().T @ Q[b] - np.eye(n)).max() <= 1e-13 * m
