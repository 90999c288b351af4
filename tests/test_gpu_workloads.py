"""GPU checks of the other workloads: the 21-site XY chain (a bath on every site), the ensemble
of independent chains, and the random augmented-MPS stress case.

Element-by-element parity with the oracle runs at sizes the oracle finishes in seconds; the
full-size runs check properties that hold at any size (trace, conservation of sum_n <s^z_n> for the
isotropic XY chain with s^z baths, real expectation values, bond caps).
"""
import numpy as np
import pytest

from workloads import workload
from workloads.configs import ChainSpec, Workload, BathSpec
from oracle import model, problem as oprob
from tests.gpu_helpers import OPS, oracle_envelope, run_gpu, run_oracle

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


def _xy_chain(N, bath):
    init = "".join("u" if n == N // 2 else "d" for n in range(N))
    return ChainSpec(N=N, eps=(0.0,) * N, J=((1.0, 1.0, 0.0),) * (N - 1), init=init, baths=(bath,) * N)


def test_xy_chain_with_a_bath_on_every_site_parity():
    # the 21-site workload's bath (alpha=0.05, wc=3, T=0.8), kappa <= 16, chi <= 128, eps = 1e-6,
    # dt = 0.1, on 9 sites for 5 steps (every bond runs the QR and LQ reductions)
    w0 = workload("xy21_allbaths")
    w = Workload("xy9", (_xy_chain(9, w0.chains[0].baths[0]),), dt=w0.dt, K=5, chi_max=w0.chi_max,
                 eps=w0.eps, kappa_max=w0.kappa_max)
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS)
    ref = run_oracle(w, cis, OPS)[0]
    err = np.abs(obs[:, 0, :9, :] - ref.obs).max(axis=(1, 2))
    env = oracle_envelope(w, cis[0], OPS)
    bad = np.nonzero(err > TOL + 10 * env)[0]
    assert len(bad) == 0, (err, env)
    eng.destroy()


def test_xy21_full_size_properties():
    # the 21-site workload itself (PT-MPO built by the library's host builder), first 12 steps:
    # sum_n <s^z_n> / Tr rho is conserved, expectation values are real, and Tr rho stays within the
    # PT-MPO compression error of 1 (kappa <= 16 on 21 baths: a few 1e-5 per bath and step)
    import paper_2201_05529_gb300._capi as capi
    from paper_2201_05529_gb300 import problem as pp
    w = workload("xy21_allbaths", K=12)
    chains, mpos = pp.build_problem(w)
    eng = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
    eng.set_observables([model.SZ])
    eng.step(w.K)
    obs, tr = eng.read_history(0, w.K + 1)
    sz = (obs[:, 0, :, 0] / tr[:, 0, None]).real
    tot = sz.sum(axis=1)
    assert abs(tot[0] - (-19.0)) < 1e-12
    assert np.max(np.abs(tot - tot[0])) < 1e-6
    assert np.max(np.abs(obs.imag)) < 1e-8
    assert np.max(np.abs(tr[:, 0] - 1)) < 21 * 2e-4
    chi, kap = eng.get_dims(0)
    assert chi.max() <= w.chi_max and kap.max() <= w.kappa_max
    print("xy21: chi after 12 steps", list(chi))
    eng.destroy()


def test_ensemble_of_four_chains_twenty_steps():
    w = workload("xyz_ensemble64", K=20)
    w.chains = w.chains[:4]
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS)
    refs = run_oracle(w, cis, OPS)
    for c, r in enumerate(refs):
        N = cis[c].N
        err = np.abs(obs[:, c, :N, :] - r.obs).max(axis=(1, 2))
        env = oracle_envelope(w, cis[c], OPS)
        bad = np.nonzero(err > TOL + 10 * env)[0]
        assert len(bad) == 0, (c, err.max())
    eng.destroy()


def test_full_ensemble_of_64_chains_in_one_engine():
    # all 64 chains (N = 4..16, two end baths each, 128 PT-MPOs) in one handle: every layer is one
    # grouped launch over the bonds of every chain. Eight chains spread over the batch (short and
    # long ones) against the oracle element by element (FP64 path, 1e-9, bond dimensions exact);
    # the fast path on the same batch against the FP64 path (1e-5) and the trace of every chain.
    import paper_2201_05529_gb300._capi as capi
    from tests.gpu_helpers import engine_args_from_oracle
    K = 10
    w = workload("xyz_ensemble64", K=K)
    cis = oprob.build_inputs(w)
    assert len(cis) == 64
    chains, mpos = engine_args_from_oracle(cis)
    out = {}
    for prec in ("fp64", "bf16_ozaki"):
        eng = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=prec,
                          multiplet_tol=w.multiplet_tol, max_steps=K)
        eng.set_observables(OPS)
        eng.step(K)
        obs, tr = eng.read_history(0, K + 1)
        dims = [eng.get_dims(c) for c in range(64)]
        eng.destroy()
        out[prec] = (obs, tr, dims)
    obs, tr, dims = out["fp64"]
    sel = [0, 9, 18, 27, 36, 45, 54, 63]
    refs = run_oracle(w, [cis[c] for c in sel], OPS, K=K)
    for c, r in zip(sel, refs):
        N = cis[c].N
        err = float(np.max(np.abs(obs[:, c, :N, :] - r.obs)))
        assert err < TOL, f"chain {c} (N = {N}): max |obs - oracle| = {err:.3e}"
        assert list(dims[c][0]) == list(r.chis[-1]), f"chain {c}: bond dimensions"
        assert np.max(np.abs(tr[:, c] - r.trace)) < TOL
    assert np.max(np.abs(tr - 1.0)) < 1e-3                       # PT-MPO compression only
    fobs, ftr, _ = out["bf16_ozaki"]
    assert np.max(np.abs(fobs - obs)) < 1e-5 and np.max(np.abs(ftr - tr)) < 1e-5


def test_random_stress_state_singular_values():
    # the stress workload's structure (Gaussian augmented MPS, Gaussian PT tensors, Haar gates) at
    # N=8, chi=32, kappa=8 for 2 steps: bond dims and singular values against the oracle
    w = workload("random32_stress", K=2)
    w.random_state = dict(N=8, chi=32, kappa=8, K=2)
    w.chi_max = 32
    w.kappa_max = 8
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS, K=2)
    ref = run_oracle(w, cis, OPS, K=2)[0]
    chi, _ = eng.get_dims(0)
    assert list(chi) == list(ref.chis[-1])
    worst = 0.0
    for b in range(1, 8):
        lam = eng.get_lambda(0, b)
        worst = max(worst, float(np.max(np.abs(lam - ref.final_mps.lam[b]))))
    print(f"random stress N=8: max |lambda - oracle| = {worst:.2e}")
    assert worst < 1e-9
    eng.destroy()


def test_random_stress_full_size_first_step_fast_path():
    # the stress workload at full size (N = 32, chi = 96, kappa = 16 on every site: D up to
    # 1536 x 1536) on the fast path, one step, against the oracle's state after that step
    # (tests/golden/random32_step1.json, written by tests/golden/make_random32_step1.py from the
    # oracle alone). Checked: every bond update ran at full size without a fault flag, the bond
    # dimensions equal the oracle's, and the singular values agree to what a randomized range finder
    # can give on this state. Its D have flat spectra (on bond 2 of the first layer
    # sigma_96 / sigma_1 = 0.38 and sigma_129 / sigma_96 = 0.83, so the range finder's subspace
    # error at the cut, (sigma_{l+1} / sigma_chi)^(2q+1) with l = 128, q = 2, is ~0.4): a CPU run of
    # the same algorithm in FP64 on that D leaves the normalised singular values 1.6e-3 off, and the
    # step has six layers. The random state's raw Tr(O rho) underflows to 0 (its caps shrink ~1e-11
    # per site), so observables carry no information here. The FP64 path's exact Jacobi on
    # full-rank D of this size runs minutes per step and is not run.
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "random32_step1.json")))
    w = workload("random32_stress")
    assert g["K"] == w.K and g["chi_max"] == w.chi_max
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, [model.SZ, model.SX], K=1, precision="bf16_ozaki")
    chi, kap = eng.get_dims(0)
    lam_err = max(float(np.max(np.abs(eng.get_lambda(0, b) - np.array(g["lambda"][b])))) for b in range(1, 32))
    blog, _ = eng.read_bond_log(0, 1)
    eng.destroy()
    print(f"random32 full size, fast path, step 1: D up to {blog[..., 0].max()} x {blog[..., 1].max()}, "
          f"max |lambda - oracle| = {lam_err:.2e}")
    assert int(blog[..., 0].max()) == 1536 and int(blog[..., 1].max()) == 1536
    assert not np.any(blog[..., 4])                      # no fault flags
    assert list(chi) == g["chis"] and list(kap) == g["kappas"]
    assert lam_err < 5e-2
    assert np.all(np.isfinite(obs)) and np.all(np.isfinite(tr))


@pytest.fixture(scope="module")
def xy21_ten_steps():
    # the 21-site workload itself, first 10 steps (chi reaches ~85, D up to ~1300 x 1300): the oracle
    # with its own PT-MPOs (tens of seconds on the host cores)
    w = workload("xy21_allbaths", K=10)
    cis = oprob.build_inputs(w)
    return w, cis, run_oracle(w, cis, OPS)[0]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("bf16_ozaki", 1e-5)])
def test_xy21_first_ten_steps_parity(xy21_ten_steps, precision, tol):
    w, cis, ref = xy21_ten_steps
    eng, obs, tr = run_gpu(w, cis, OPS, precision=precision)
    err = np.abs(obs[:, 0, :21, :] - ref.obs).max(axis=(1, 2))
    print(f"xy21 {precision}: max |obs - oracle| per step {np.array2string(err, precision=2)}")
    assert np.max(err) < tol
    assert np.max(np.abs(tr[:, 0] - ref.trace)) < tol
    chi, kap = eng.get_dims(0)
    if precision == "fp64":
        assert list(chi) == list(ref.chis[-1]) and list(kap) == list(ref.kappas[-1])
    # the bond blocks went through the large-matrix routes: D above 256 (cluster pivoted QR) and a
    # rank-revealing stop well below D's size
    log, _ = eng.read_bond_log(0, w.K)
    mD, nD, k = log[..., 0], log[..., 1], log[..., 2]
    big = np.minimum(mD, nD) > 256
    assert np.any(big)
    assert np.all(k[big] < np.minimum(mD, nD)[big])
    eng.destroy()


def test_tuning_at_capacity_leaves_the_state_untouched():
    # the autotuner runs every candidate on a synthetic state at full capacity (the outer-block QR's
    # reflector scalars fill 4 chi_c entries of a bond's scratch, more than its SVD needs on the
    # chain's edge bonds), then restores the initial state: the tuned engine must reproduce, bit for
    # bit, an untuned engine forced onto the same routes
    import paper_2201_05529_gb300._capi as capi
    from paper_2201_05529_gb300 import problem as pp
    w = workload("xy21_allbaths", K=4)
    chains, mpos = pp.build_problem(w)
    runs = []
    for kw in (dict(autotune=True, tune_cache=None), None):
        if kw is None:
            r = runs[0][1]
            kw = dict(autotune=False, route=r["odd"][:2]) if r["odd"][:2] == r["even"][:2] else None
            if kw is None:
                pytest.skip("the tuner chose different routes for the two layers")
        e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K, **kw)
        e.set_observables(OPS)
        routes = e.routes()
        e.step(w.K)
        e.sync()
        obs, tr = e.read_history(0, w.K + 1)
        flags = e.get_svd_sweeps()[:, 1]
        e.destroy()
        assert np.all(flags == 0)
        runs.append(((obs, tr), routes))
    assert runs[0][1]["odd"][2] and not runs[1][1]["odd"][2]         # tuned, then forced
    assert np.array_equal(runs[0][0][0], runs[1][0][0]) and np.array_equal(runs[0][0][1], runs[1][0][1])
