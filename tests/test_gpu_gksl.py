"""GPU path with time-local (GKSL) chain terms (App. A.1) and the two-spin driving network of
Sec. III.A.3, against the oracle; FP64 path, 1e-9 on every observable at every step.

The time step is unchanged: dissipation enters only through the (now non-unitary) two-site gates
exp(L^{K'} tau), so these runs check that nothing in the path assumes unitary gates (truncation,
log-norm, readout, caps with a bath on a dissipative site).
"""
import numpy as np
import pytest

from workloads import workload
from oracle import problem as oprob
from tests.gpu_helpers import OPS, run_gpu, run_oracle

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


@pytest.mark.parametrize("name", ["xyz5_gksl", "xyz7_twospin_drive"])
def test_dissipative_chain_parity(name):
    w = workload(name, K=20)
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS)
    ref = run_oracle(w, cis, OPS)[0]
    N = cis[0].N
    err = np.max(np.abs(obs[:, 0, :N, :] - ref.obs))
    print(f"{name}: max |obs - oracle| = {err:.2e}, trace drift {np.max(np.abs(tr[:, 0] - 1)):.1e}")
    assert err < TOL
    assert np.max(np.abs(tr[:, 0] - ref.trace)) < TOL
    chi, _ = eng.get_dims(0)
    assert list(chi) == list(ref.chis[-1])
    eng.destroy()


def test_library_builder_end_to_end_with_dissipation(_lib):
    # the library's own gate and PT-MPO builders feeding the C ABI, against the oracle's run on
    # the oracle's inputs (the builders agree to ~1e-13 in observables)
    from paper_2201_05529_gb300 import problem as pp
    w = workload("xyz5_gksl", K=20)
    chains, mpos = pp.build_problem(w)
    eng = _lib.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
    eng.set_observables(OPS)
    eng.step(w.K)
    obs, _ = eng.read_history(0, w.K + 1)
    ref = run_oracle(w, oprob.build_inputs(w), OPS)[0]
    assert np.max(np.abs(obs[:, 0, :5, :] - ref.obs)) < TOL
    eng.destroy()
