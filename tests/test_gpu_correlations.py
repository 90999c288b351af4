"""GPU branching two-time correlations (App. B.2) against the oracle, and their spectra.

The branch is cloned on the device at step k_b, the super-operator applied to the clone, and the
clone propagated; the oracle applies the same super-operator to its own state after step k_b.
FP64 path, a workload whose chi cap never binds: held to the 1e-9 bar at every lag.
"""
import numpy as np
import pytest

from workloads import workload
from oracle import model, problem as oprob, spectra
from tests.gpu_helpers import engine_args_from_oracle

pytestmark = pytest.mark.gpu

TOL = 1e-9


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


@pytest.mark.parametrize("side", ["left", "right"])
def test_branch_correlation_matches_oracle_and_leaves_the_engine_alone(side, _lib):
    from paper_2201_05529_gb300.correlations import branch_correlation
    w = workload("xyz3_onebath")
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    eng = _lib.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
    eng.set_observables([model.SZ])
    kb, n = 10, w.K - 10
    eng.step(kb)
    C = branch_correlation(eng, 0, 1, model.SZ, 1, model.SZ, n, side)
    ref = oprob.simulate_chain(cis[0], w, [model.SZ], insert=(1, model.SZ, side), insert_at=kb)
    Cref = ref.obs[kb:kb + n + 1, 1, 0]
    err = np.max(np.abs(C - Cref))
    print(f"{side}: max |C_gpu - C_oracle| = {err:.2e} over {n + 1} lags")
    assert err < TOL
    # the original engine continues as if nothing had been branched off
    eng.step(w.K - kb)
    obs, _ = eng.read_history(0, w.K + 1)
    plain = oprob.simulate_chain(cis[0], w, [model.SZ])
    assert np.max(np.abs(obs[:, 0, :3, 0] - plain.obs[:, :, 0])) < TOL
    eng.destroy()


def test_spectra_of_the_gpu_correlation():
    # S, chi'' and T from the GPU correlation (library FFT) against the oracle's direct sums of the
    # oracle correlation: the spectra inherit the correlation's agreement
    from paper_2201_05529_gb300 import _capi
    from paper_2201_05529_gb300.correlations import branch_correlation, fdt_spectra
    w = workload("xyz3_onebath")
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    eng = _capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
    kb, n = 8, w.K - 8
    eng.step(kb)
    C = branch_correlation(eng, 0, 1, model.SZ, 1, model.SZ, n, "left")
    eng.destroy()
    ref = oprob.simulate_chain(cis[0], w, [model.SZ], insert=(1, model.SZ, "left"), insert_at=kb)
    Cref = ref.obs[kb:kb + n + 1, 1, 0]
    om, S, chi2, T = fdt_spectra(C, w.dt)
    So, Co, _ = spectra.spectra(Cref, w.dt, om)
    scale = np.max(np.abs(So))
    assert np.max(np.abs(S - So)) < 1e-8 * max(1.0, scale)
    assert np.max(np.abs(chi2 - Co)) < 1e-8 * max(1.0, scale)
