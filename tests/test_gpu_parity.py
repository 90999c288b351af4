"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same inputs.

Tolerance (FP64 path): 1e-9 absolute on every observable at every step, the bar the PT-TEBD
target sets for the FP64 GPU path; bond dimensions must agree exactly and singular values to 1e-9.
Where the chi cap binds, the truncated trajectory amplifies rounding differences (the lambda^-1 of
App. A.2 on singular values down to ~1e-9 of the largest), so there the bar is
1e-9 + 10 x the oracle's own sensitivity to a 1e-13 relative perturbation of its gates, measured
per step on the same inputs (``oracle_envelope``).
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


def _state_matches(eng, c, N, chis, kappas, lams, lognorm, tol):
    chi, kap = eng.get_dims(c)
    assert list(chi) == list(chis), (list(chi), chis)
    assert list(kap) == list(kappas)
    for b in range(1, N):
        lam = eng.get_lambda(c, b)
        assert np.max(np.abs(lam - lams[b])) < tol
    assert abs(eng.get_lognorm(c) - lognorm) < tol


def _compare(w, cis, K=None, insert=None, tol=TOL, chis=True, envelope=False):
    K = w.K if K is None else K
    eng, obs, tr = run_gpu(w, cis, OPS, K=K, insert=insert)
    ref = run_oracle(w, cis, OPS, K=K, insert=insert)
    strict_windows = []
    for c, r in enumerate(ref):
        N = cis[c].N
        err = np.abs(obs[:, c, :N, :] - r.obs).max(axis=(1, 2))
        if envelope:
            ins = insert if (insert is not None and insert[0] == c) else None
            bar = tol + 10.0 * oracle_envelope(w, cis[c], OPS, K=K, insert=ins)
            bad = np.nonzero(err > bar)[0]
            assert len(bad) == 0, f"chain {c}: step {bad[0]}: |obs - oracle| = {err[bad[0]]:.3e} > {bar[bad[0]]:.3e}"
            # the strict window: every step before the oracle's own envelope passes the bar
            s_end = int(np.argmax(bar > 2 * tol)) - 1 if np.any(bar > 2 * tol) else K
            assert s_end >= 1
            assert np.max(err[:s_end + 1]) < tol, f"chain {c}: strict window 0..{s_end}: {np.max(err[:s_end + 1]):.3e}"
            assert np.max(np.abs(tr[:s_end + 1, c] - r.trace[:s_end + 1])) < tol
            strict_windows.append((c, s_end))
            continue
        assert np.max(err) < tol, f"chain {c}: max |obs - oracle| = {np.max(err):.3e}"
        assert np.max(np.abs(tr[:, c] - r.trace)) < tol
        if chis:
            _state_matches(eng, c, N, r.chis[-1], r.kappas[-1], r.final_mps.lam, r.lognorm[-1], tol)
    eng.destroy()
    # envelope runs: bond dims, lambdas and log-norm at the end of each strict window, from a run
    # stopped there (the oracle keeps every step's state)
    for c, s_end in strict_windows:
        if s_end >= K:
            s_end = K
        e2, _, _ = run_gpu(w, cis, OPS, K=s_end, insert=insert)
        r = ref[c]
        _state_matches(e2, c, cis[c].N, r.chis[s_end], r.kappas[s_end], r.lambdas[s_end - 1],
                       r.lognorm[s_end], tol)
        e2.destroy()
    return obs, ref


def test_three_site_one_bath_full():
    # XYZ N=3, one Ohmic bath (alpha=0.1, wc=4, T=1), dt=0.1, 20 steps, kappa<=16, chi<=64
    w = workload("xyz3_onebath")
    _compare(w, oprob.build_inputs(w))


def test_markovian_four_sites_odd_and_even_layers():
    ch = ChainSpec(N=4, eps=(0.5, 0.2, -0.3, 0.1), J=((1.3, 0.7, 1.2),) * 3, init="udud", baths=(None,) * 4)
    w = Workload("t", (ch,), dt=0.05, K=25, chi_max=64, eps=1e-12, kappa_max=1)
    _compare(w, oprob.build_inputs(w))


def test_five_site_two_baths_forty_steps():
    # chi reaches the cap 64 near step 10; strict 1e-9 on observables and trace until the oracle's
    # own response to a 1e-13 gate perturbation passes 2e-9 (step ~17), then the envelope; bond
    # dims, lambdas and log-norm checked at the end of the strict window
    w = workload("xyz5_twobaths", K=40)
    _compare(w, oprob.build_inputs(w), envelope=True)


def test_five_site_two_baths_uncapped_window():
    # the same chain with a cap that never binds: 1e-9 at every step, singular values, dims
    w = workload("xyz5_twobaths", K=12, chi_max=256)
    _compare(w, oprob.build_inputs(w))


def test_two_time_correlation_five_sites():
    # <s^x_3(t) s^x_3(0)>: A^L = sigma^x inserted on site 3 at t = 0, raw readout (App. A.4)
    w = workload("xyz5_twobaths", K=30)
    cis = oprob.build_inputs(w)
    _compare(w, cis, insert=(0, 2, model.SX, "left"), envelope=True)


def test_qr_reduced_path_all_sites_with_baths():
    # every site has a bath: B_L is taller than wide and B_R wider than tall, so both the QR and
    # the LQ reductions of App. A.2 run
    b = BathSpec(0.05, 3.0, 0.8)
    ch = ChainSpec(N=5, eps=(0.0,) * 5, J=((1.0, 1.0, 0.0),) * 4, init="ddudd", baths=(b,) * 5)
    w = Workload("t", (ch,), dt=0.1, K=8, chi_max=48, eps=1e-8, kappa_max=6)
    _compare(w, oprob.build_inputs(w))


def test_ragged_batch_of_chains():
    w = workload("xyz_ensemble64", K=12)
    w.chains = w.chains[:6]
    _compare(w, oprob.build_inputs(w))


def test_random_state_singular_values():
    w = workload("random32_stress", K=2)
    w.random_state = dict(N=6, chi=12, kappa=4, K=2)
    w.chi_max = 12
    w.kappa_max = 4
    cis = oprob.build_inputs(w)
    eng, obs, tr = run_gpu(w, cis, OPS, K=2)
    ref = run_oracle(w, cis, OPS, K=2)[0]
    chi, _ = eng.get_dims(0)
    assert list(chi) == list(ref.chis[-1])
    for b in range(1, 6):
        lam = eng.get_lambda(0, b)
        assert np.max(np.abs(lam - ref.final_mps.lam[b])) < 1e-9
    eng.destroy()


def test_clone_continues_identically():
    import paper_2201_05529_gb300._capi as capi
    from tests.gpu_helpers import engine_args_from_oracle
    w = workload("xyz3_onebath")
    cis = oprob.build_inputs(w)
    chains, mpos = engine_args_from_oracle(cis)
    e1 = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K)
    e1.step(7)
    e2 = e1.clone()
    e1.step(5)
    e2.step(5)
    a, _ = e1.observe([model.SZ])
    b, _ = e2.observe([model.SZ])
    assert np.max(np.abs(a - b)) == 0.0
    e1.destroy()
    e2.destroy()


def test_graph_and_eager_agree_bitwise():
    w = workload("xyz3_onebath", K=10)
    cis = oprob.build_inputs(w)
    _, o1, _ = run_gpu(w, cis, OPS, K=10, use_graph=True)
    _, o2, _ = run_gpu(w, cis, OPS, K=10, use_graph=False)
    assert np.array_equal(o1, o2)


def test_stepping_past_the_pt_mpo_is_an_error():
    import paper_2201_05529_gb300._capi as capi
    from tests.gpu_helpers import engine_args_from_oracle
    w = workload("xyz3_onebath", K=5)
    chains, mpos = engine_args_from_oracle(oprob.build_inputs(w))
    e = capi.Engine(chains, mpos, chi_max=8, eps=1e-10)
    e.step(5)
    with pytest.raises(capi.PTError) as ei:
        e.step(1)
    assert ei.value.code == -8
    e.destroy()


def test_standalone_svd_against_lapack():
    import torch
    import paper_2201_05529_gb300._capi as capi
    rng = np.random.default_rng(7)
    for (m, n, b) in [(37, 23, 3), (16, 64, 2), (130, 130, 1), (1, 5, 2)]:
        A = rng.standard_normal((b, m, n)) + 1j * rng.standard_normal((b, m, n))
        k = min(m, n)
        dA = torch.from_numpy(A).cuda()
        s = torch.zeros((b, k), dtype=torch.float64, device="cuda")
        U = torch.zeros((b, m, k), dtype=torch.complex128, device="cuda")
        V = torch.zeros((b, n, k), dtype=torch.complex128, device="cuda")
        scr = torch.zeros(capi.svd_scratch_bytes(m, n, b), dtype=torch.uint8, device="cuda")
        capi.svd_f64(dA, s, U, V, scr)
        torch.cuda.synchronize()
        s, U, V = s.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
        for i in range(b):
            ref = np.linalg.svd(A[i], compute_uv=False)
            assert np.max(np.abs(s[i] - ref)) < 1e-12 * ref[0] * max(m, n)
            rec = (U[i] * s[i][None, :]) @ V[i].conj().T
            assert np.max(np.abs(rec - A[i])) < 1e-12 * ref[0] * max(m, n)
            assert np.max(np.abs(U[i].conj().T @ U[i] - np.eye(k))) < 1e-12 * max(m, n)


@pytest.mark.parametrize("route", [("grid", "grid"), ("cluster_smem", "grid"), ("cluster_global", "grid"),
                                   ("grid", "cta"), ("cluster_global", "cta")])
@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("bf16_ozaki", 1e-5)])
def test_every_route_the_tuner_can_pick(route, precision, tol):
    # every candidate of the autotuner (pivoted QR of the SVD on the whole GPU, in cluster shared
    # memory, in cluster global memory; outer-block QR on the whole GPU or one CTA per block) forced
    # on a twelve-step window of the five-site chain (chi_max 64: every route fits), against the oracle
    import paper_2201_05529_gb300._capi as capi
    w = workload("xyz5_twobaths", K=12, chi_max=64)
    cis = oprob.build_inputs(w)
    try:
        eng, obs, tr = run_gpu(w, cis, OPS, precision=precision, route=route)
    except capi.PTError as ex:
        # a route this device cannot co-schedule (cluster shared memory needs 16-CTA clusters)
        assert ex.code == -1 and "does not fit" in str(ex) and route[0] == "cluster_smem", ex
        pytest.skip(f"route {route} does not fit on this device")
    r = eng.routes()
    assert r["odd"][:2] == route and r["even"][:2] == route
    ref = run_oracle(w, cis, OPS)[0]
    err = np.abs(obs[:, 0, :5, :] - ref.obs).max(axis=(1, 2))
    assert np.max(err) < tol, err
    eng.destroy()


def test_tuner_times_once_then_reads_its_cache(tmp_path):
    import paper_2201_05529_gb300._capi as capi
    from tests.gpu_helpers import engine_args_from_oracle
    w = workload("xyz5_twobaths", K=4)
    chains, mpos = engine_args_from_oracle(oprob.build_inputs(w))
    cache = str(tmp_path / "tune.tsv")
    e1 = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K, autotune=True, tune_cache=cache)
    r1 = e1.routes()
    assert r1["odd"][2] and not r1["odd"][3]                  # timed, not from the cache
    assert min(t for t in r1["odd"][4] if t >= 0) > 0
    e1.step(4)
    e1.sync()
    e1.destroy()
    e2 = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, max_steps=w.K, autotune=True, tune_cache=cache)
    r2 = e2.routes()
    assert r2["odd"][3] and r2["odd"][:2] == r1["odd"][:2] and r2["even"][:2] == r1["even"][:2]
    e2.destroy()
    assert len(open(cache).read().splitlines()) == 2           # one line per layer shape
