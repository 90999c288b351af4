"""The fast path's batched complex GEMM on the tensor cores (pt_zgemm_sliced) against FP64 numpy.

Error bound. Every row of opA(A) and column of opB(B) is scaled by a power of two 2^e (max entry
below 1) and cut into six BF16 fixed-point slices of 7 bits; K is accumulated in chunks of 512 (the
two leading levels exact in FP32 within a chunk) and the chunks are added in FP64. Dropping the
slice pairs of level >= 6 costs at most ~1.3 2^-42 per product term, and the FP32 accumulation of
the deeper levels rounds at a similar or smaller scale, so per entry
  |C - C_exact|_ij <= c K max|row i of opA(A)| max|column j of opB(B)|,  c = 2^-40.
The shapes span several 128 x 64 output tiles with ragged tails, all three operand forms, inner
dimensions on both sides of each slice-width switch, rows and columns whose scales differ by many
orders of magnitude, and all-zero rows.
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
    c = pkg.load()
    c.use_torch_allocator()
    return c


def _op(X, op):
    return X if op == "N" else (X.T if op == "T" else X.conj().T)


def _colmajor(torch, X):
    # [batch, rows, cols] numpy -> [batch, cols, rows] contiguous device tensor (column-major storage)
    return torch.from_numpy(np.ascontiguousarray(X.transpose(0, 2, 1))).cuda()


@pytest.mark.parametrize("m,n,k,opA,opB", [
    (1, 1, 1, "N", "N"),
    (300, 70, 530, "N", "N"),          # ragged tiles, two K chunks
    (129, 65, 17, "H", "N"),
    (257, 200, 512, "N", "H"),         # one full K chunk
    (64, 128, 2049, "T", "T"),         # five K chunks, the last one element
    (1000, 160, 1000, "N", "N"),
    (160, 900, 1000, "H", "N"),        # the shape of a projection Q^H D
])
def test_sliced_zgemm_against_numpy(capi, m, n, k, opA, opB):
    import torch
    rng = np.random.default_rng(m * 131 + n * 7 + k)
    batch = 3
    # opA(A) (m x k) and opB(B) (k x n) with graded scales on the rows of opA(A) and the columns of
    # opB(B), one all-zero row and column; stored as the op requires
    ra = 10.0 ** rng.uniform(-9, 3, size=m)
    cb = 10.0 ** rng.uniform(-6, 6, size=n)
    OA = (rng.standard_normal((batch, m, k)) + 1j * rng.standard_normal((batch, m, k))) * ra[None, :, None]
    OB = (rng.standard_normal((batch, k, n)) + 1j * rng.standard_normal((batch, k, n))) * cb[None, None, :]
    if m > 2:
        OA[:, 1, :] = 0.0
    if n > 2:
        OB[:, :, 2] = 0.0
    store = {"N": lambda X: X, "T": lambda X: X.transpose(0, 2, 1), "H": lambda X: X.conj().transpose(0, 2, 1)}
    A, B = store[opA](OA), store[opB](OB)
    At, Bt = _colmajor(torch, A), _colmajor(torch, B)
    Ct = torch.zeros((batch, n, m), dtype=torch.complex128, device="cuda")
    scratch = torch.empty(capi.zgemm_scratch_bytes(m, n, k, batch), dtype=torch.uint8, device="cuda")
    capi.zgemm_sliced(opA, opB, At, Bt, Ct, m, n, k, scratch)
    torch.cuda.synchronize()
    C = Ct.cpu().numpy().transpose(0, 2, 1)
    cb_ = 2.0 ** -40
    worst = 0.0
    for b in range(batch):
        opa, opb = _op(A[b], opA), _op(B[b], opB)
        assert np.array_equal(opa, OA[b]) and np.array_equal(opb, OB[b])
        ref = opa @ opb
        rmax = np.maximum(np.abs(opa.real), np.abs(opa.imag)).max(axis=1)
        cmax = np.maximum(np.abs(opb.real), np.abs(opb.imag)).max(axis=0)
        scale = k * rmax[:, None] * cmax[None, :]
        err = np.abs(C[b] - ref)
        assert np.all(err <= cb_ * scale), float(np.max(err / np.where(scale > 0, scale, 1)))
        assert np.all(C[b][scale == 0] == 0)
        worst = max(worst, float(np.max(err / np.where(scale > 0, scale, 1))))
    print(f"{m}x{n}x{k} {opA}{opB}: max |err| / (K rowmax colmax) = {worst:.2e} (bound {cb_:.1e})")


def test_sliced_zgemm_rejects_bad_arguments(capi):
    import torch
    A = torch.zeros((1, 4, 4), dtype=torch.complex128, device="cuda")
    scratch = torch.empty(capi.zgemm_scratch_bytes(4, 4, 4, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.PTError) as ei:
        capi.zgemm_sliced("N", "N", A, A, A, 4, 4, 0, scratch)
    assert ei.value.code == -1
