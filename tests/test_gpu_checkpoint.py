"""Checkpoint and resume (App. B.2: the propagation continues from the full augmented MPS).

A run of the five-site two-bath chain is stopped after step s, its state read to the host
(pt_tebd_get_gamma, pt_tebd_get_lambda, pt_tebd_get_lognorms), and a new handle is initialised
from those host buffers with every PT-MPO cut at step s. The resumed run must reproduce the
continuous run's observables, trace and bond dimensions (to 1e-12; bit for bit when the new
handle's capacities match), and stay within the FP64 bar of the oracle. The steps stay inside the
window where the oracle's own rounding envelope is below 1e-9."""
import numpy as np
import pytest

from workloads import workload
from oracle import problem as oprob
from tests.gpu_helpers import OPS, engine_args_from_oracle, run_oracle

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


@pytest.mark.parametrize("precision", ["fp64", "bf16_ozaki"])
def test_resume_from_host_checkpoint(capi, precision):
    S, K = 5, 12
    w = workload("xyz5_twobaths", K=K)
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    kw = dict(chi_max=w.chi_max, eps=w.eps, precision=precision, multiplet_tol=w.multiplet_tol, max_steps=K)

    full = capi.Engine(chains, mpos, **kw)
    full.set_observables(OPS)
    full.step(K)
    obs_full, tr_full = full.read_history(0, K + 1)
    dims_full = full.get_dims(0)
    full.destroy()

    first = capi.Engine(chains, mpos, **kw)
    first.set_observables(OPS)
    first.step(S)
    ck = first.checkpoint()
    assert ck[0]["step"] == S
    chi, kap = first.get_dims(0)
    for n, g in enumerate(ck[0]["gamma"]):
        assert g.shape == (chi[n], 4, kap[n], chi[n + 1])
    first.destroy()

    rchains, rmpos = capi.resume_problem(chains, mpos, ck)
    assert all(len(P) == K - S for P in rmpos)
    res = capi.Engine(rchains, rmpos, **dict(kw, max_steps=K - S))
    res.set_observables(OPS)
    res.step(K - S)
    obs_r, tr_r = res.read_history(0, K - S + 1)
    dims_r = res.get_dims(0)
    res.destroy()

    # the same tensors, per-bond log-norms and kernels: the continuation is the same run (bit for bit
    # when the new handle's capacities, and so its kernel routes, match; held here to 1e-12)
    d_obs = float(np.max(np.abs(obs_r - obs_full[S:])))
    d_tr = float(np.max(np.abs(tr_r - tr_full[S:])))
    print(f"resume ({precision}): max |obs - continuous| = {d_obs:.3e}, max |trace - continuous| = {d_tr:.3e}, "
          f"bitwise: {np.array_equal(obs_r, obs_full[S:]) and np.array_equal(tr_r, tr_full[S:])}")
    assert d_obs <= 1e-12 and d_tr <= 1e-12
    assert np.array_equal(dims_r[0], dims_full[0]) and np.array_equal(dims_r[1], dims_full[1])
    if precision == "fp64":
        ref = run_oracle(w, cis, OPS, K=K)[0]
        assert np.max(np.abs(obs_r[:, 0, :, :] - ref.obs[S:])) < 1e-9


def test_get_gamma_rejects_small_buffer(capi):
    w = workload("xyz3_onebath", K=4)
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=4)
    e.step(2)
    import ctypes as C
    n = capi.lib.pt_tebd_get_gamma(e.h, 0, 1, None, 0)
    assert n > 0
    buf = np.zeros(max(1, n - 1), dtype=np.complex128)
    rc = capi.lib.pt_tebd_get_gamma(e.h, 0, 1, buf.ctypes.data_as(C.POINTER(C.c_double)), n - 1)
    assert rc == -1                                                   # PT_ERR_ARG
    assert capi.lib.pt_tebd_get_gamma(e.h, 0, 3, None, 0) == -1      # no such site
    e.destroy()
