"""Fast path (theta + gate on tcgen05 tensor cores, FP64 Jacobi SVD) against the FP64 oracle.

The PT-TEBD target holds the FP32 tensor-core path to 1e-5 absolute on <sigma^z_n(t)>.

bf16_ozaki (fixed-point BF16 slices whose leading partial sums are exact in the tensor cores' FP32
accumulators) is the fast path that meets it: the theta + gate product is accurate to ~1e-9 of
the rows' scale, so the path follows the oracle as closely as the FP64 GPU path does. It is held to
1e-7 on the three-site chain, and on the five-site chain to the strict 1e-5 until the oracle's own
response to a 1e-13 gate perturbation passes 1e-6 (step ~24: beyond it the chi-capped trajectory
amplifies any rounding difference, FP64 included, to ~1e-4; see test_gpu_parity.py).

The natural-split modes (TF32x3, BF16x3: three pieces of every operand, FP32 accumulation of the
unscaled piece products) carry the accumulators' rounding, ~1e-6 of the row scale per product;
on the five-site chain that drifts ~1e-6 per step, so the strict 1e-5 window is an expected failure
(strict xfail: it fails today, and would be flagged if it started to pass). Every error is printed.
"""
import numpy as np
import pytest

from workloads import workload
from oracle import model, problem as oprob
from tests.gpu_helpers import OPS, oracle_envelope, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

FAST_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_05529_gb300 as pkg
    pkg.build()
    capi = pkg.load()
    capi.use_torch_allocator()
    return capi


def _err(obs, ref, N):
    return np.abs(obs[:, 0, :N, :] - ref.obs).max(axis=(1, 2))


@pytest.fixture(scope="module")
def five_site():
    w = workload("xyz5_twobaths", K=30)
    cis = oprob.build_inputs(w)
    ref = run_oracle(w, cis, OPS)[0]
    env = oracle_envelope(w, cis[0], OPS, scale=1e-13)
    # the strict window: until the oracle's own rounding envelope passes 1e-6
    s_end = int(np.argmax(env > 1e-6)) - 1 if np.any(env > 1e-6) else w.K
    return w, cis, ref, env, s_end


def test_three_site_one_bath_ozaki():
    w = workload("xyz3_onebath")
    cis = oprob.build_inputs(w)
    eng, obs, _ = run_gpu(w, cis, OPS, precision="bf16_ozaki")
    err = _err(obs, run_oracle(w, cis, OPS)[0], 3)
    print(f"bf16_ozaki: max |obs - oracle| per step: {np.array2string(err, precision=2)}")
    assert np.max(err) < 1e-7
    eng.destroy()


def test_five_site_two_baths_ozaki(five_site):
    w, cis, ref, env, s_end = five_site
    eng, obs, _ = run_gpu(w, cis, OPS, precision="bf16_ozaki")
    err = _err(obs, ref, 5)
    print(f"bf16_ozaki: strict window 0..{s_end}; per-step err {np.array2string(err, precision=2)}")
    assert s_end >= 20
    assert np.max(err[:s_end + 1]) < FAST_TOL, np.max(err[:s_end + 1])
    # beyond the strict window: the target plus 10x the oracle's own rounding envelope
    assert np.all(err <= FAST_TOL + 10.0 * env)
    eng.destroy()


def test_ozaki_matches_the_fp64_path_on_the_bench_window():
    # steps 5..25 of the five-site chain (the window the bench times): fast vs FP64 GPU path
    w = workload("xyz5_twobaths", K=25)
    cis = oprob.build_inputs(w)
    _, o64, _ = run_gpu(w, cis, OPS, precision="fp64")
    _, o16, _ = run_gpu(w, cis, OPS, precision="bf16_ozaki")
    d = np.abs(o64[5:, 0, :5, :] - o16[5:, 0, :5, :]).max()
    print(f"bf16_ozaki vs fp64 path, steps 5..25: {d:.2e}")
    assert d < FAST_TOL


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_natural_split_three_site_within_1e4(precision):
    w = workload("xyz3_onebath")
    cis = oprob.build_inputs(w)
    eng, obs, _ = run_gpu(w, cis, OPS, precision=precision)
    err = _err(obs, run_oracle(w, cis, OPS)[0], 3)
    print(f"{precision}: max |obs - oracle| per step: {np.array2string(err, precision=2)}")
    assert np.max(err) < 1e-4
    eng.destroy()


@pytest.mark.xfail(strict=True, reason="FP32 accumulation of unscaled split pieces drifts ~1e-6 per step "
                                       "on the five-site chain; bf16_ozaki is the path that meets 1e-5")
@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_natural_split_five_site_strict_window(precision, five_site):
    w, cis, ref, env, s_end = five_site
    eng, obs, _ = run_gpu(w, cis, OPS, precision=precision)
    err = _err(obs, ref, 5)
    print(f"{precision}: per-step err {np.array2string(err, precision=2)}")
    eng.destroy()
    assert np.max(err[:s_end + 1]) < FAST_TOL


def test_tf32x1_runs_and_is_reported():
    w = workload("xyz3_onebath", K=10)
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS, precision="tf32x1")
    ref = run_oracle(w, cis, OPS)[0]
    err = np.abs(obs[:, 0, :3, :] - ref.obs).max()
    print(f"tf32x1: max |obs - oracle| = {err:.2e}")
    assert err < 1e-2
    eng.destroy()


def test_fast_path_first_steps_match_fp64_path():
    # three steps from a product state: the only difference between the paths is theta + gate
    w = workload("xyz5_twobaths", K=3)
    cis = oprob.build_inputs(w)
    _, o64, _ = run_gpu(w, cis, OPS, precision="fp64")
    _, o16, _ = run_gpu(w, cis, OPS, precision="bf16_ozaki")
    assert np.max(np.abs(o64 - o16)) < 1e-8


@pytest.mark.parametrize("precision", ["bf16_ozaki", "tf32x3"])
def test_fast_path_graph_and_eager_agree_bitwise(precision):
    w = workload("xyz3_onebath", K=8)
    cis = oprob.build_inputs(w)
    _, o1, _ = run_gpu(w, cis, OPS, precision=precision, use_graph=True)
    _, o2, _ = run_gpu(w, cis, OPS, precision=precision, use_graph=False)
    assert np.array_equal(o1, o2)
