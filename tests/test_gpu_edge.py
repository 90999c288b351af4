"""GPU edge cases against the oracle: a single site (no bond; its field in the per-site propagator
that the engine fuses into the PT-MPO at init), a two-site chain (one odd bond, no even layer)
with propagators on a bath site and on a bath-free site, a ragged batch of N = 1, 2, 5 chains, and
a zero-step call. FP64 path, 1e-9."""
import numpy as np
import pytest
import scipy.linalg as sla

from workloads import workload
from workloads.configs import BathSpec, ChainSpec, Workload
from oracle import model, problem as oprob, pttebd, tempo
from tests.gpu_helpers import OPS

pytestmark = pytest.mark.gpu

TOL = 1e-9
B = BathSpec(0.16, 4.0, 1.0)


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


def _field(eps, dt):
    return sla.expm(model.hamiltonian_liouvillian(model.onsite_hamiltonian(eps)) * dt)


def _case(N, dt, K, fields, baths):
    """(oracle ChainInputs with fused PT-MPOs, engine chain dict with unfused ones + local_prop,
    engine PT-MPO list)."""
    J = ((1.3, 0.7, 1.2),) * (N - 1)
    init = "".join("u" if n % 2 == 0 else "d" for n in range(N))
    ch = ChainSpec(N=N, eps=(0.0,) * N, J=J, init=init, baths=tuple(baths))
    gq, gh = oprob.chain_gates(ch, dt) if N > 1 else ([], [])
    P = tempo.build_pt_mpo(B, dt, K, 1e-9, 16)
    loc = [_field(f, dt) for f in fields]
    ident = [np.eye(4, dtype=complex).reshape(1, 4, 4, 1)] * K
    pts = [[pttebd.fuse_local(Pk, loc[n]) for Pk in (P if baths[n] else ident)] for n in range(N)]
    rho0 = [model.product_state_vector(c) for c in init]
    ci = oprob.ChainInputs(N, rho0, gq, gh, pts)
    d = dict(N=N, rho0=np.array(rho0), gates_q=np.array(gq) if N > 1 else None,
             gates_h=np.array(gh) if N > 1 else None, ptmpo_id=[0 if b else -1 for b in baths],
             local_prop=np.array(loc))
    return ch, ci, d, P


def _oracle(ci, ch, dt, K, chi_max=64, eps=1e-12):
    w = Workload("t", (ch,), dt=dt, K=K, chi_max=chi_max, eps=eps, kappa_max=16)
    return oprob.simulate_chain(ci, w, OPS)


def test_single_site_and_two_sites_with_local_propagators(_lib):
    dt, K = 0.1, 12
    for N, fields, baths in ((1, [0.8], [B]), (2, [0.5, -0.3], [B, None])):
        ch, ci, d, P = _case(N, dt, K, fields, baths)
        eng = _lib.Engine([d], [P], chi_max=64, eps=1e-12, max_steps=K)
        eng.set_observables(OPS)
        eng.step(K)
        obs, tr = eng.read_history(0, K + 1)
        ref = _oracle(ci, ch, dt, K)
        err = np.max(np.abs(obs[:, 0, :N, :] - ref.obs))
        print(f"N={N}: max |obs - oracle| = {err:.2e}")
        assert err < TOL
        assert np.max(np.abs(tr[:, 0] - ref.trace)) < TOL
        eng.destroy()


def test_ragged_batch_of_one_two_and_five_sites(_lib):
    dt, K = 0.1, 10
    c1 = _case(1, dt, K, [0.8], [B])
    c2 = _case(2, dt, K, [0.5, -0.3], [B, None])
    w5 = workload("xyz5_twobaths", K=K, dt=dt)
    ci5 = oprob.build_inputs(w5)[0]
    mpos = [c1[3], c2[3]]
    ids5 = []
    for Pn in ci5.pt:
        if Pn is None:
            ids5.append(-1)
        else:
            mpos.append(Pn)
            ids5.append(len(mpos) - 1)
    d1, d2 = dict(c1[2]), dict(c2[2])
    d2["ptmpo_id"] = [1, -1]
    d5 = dict(N=5, rho0=np.array(ci5.rho0), gates_q=np.array(ci5.gates_q), gates_h=np.array(ci5.gates_h),
              ptmpo_id=ids5, local_prop=np.array([np.eye(4)] * 5, dtype=complex))
    # chi uncapped (256) and the five-site workload's eps (1e-8): with a binding cap, or with
    # eps = 1e-12 keeping singular values near 1e-12 of the largest, the lambda^-1 of the recovery
    # amplifies rounding differences between the two SVDs beyond 1e-9 within a few steps
    eng = _lib.Engine([d1, d2, d5], mpos, chi_max=256, eps=1e-8, max_steps=K)
    eng.set_observables(OPS)
    eng.step(K)
    obs, _ = eng.read_history(0, K + 1)
    refs = [_oracle(c1[1], c1[0], dt, K, 256, 1e-8), _oracle(c2[1], c2[0], dt, K, 256, 1e-8)]
    w5b = Workload("t", w5.chains, dt=dt, K=K, chi_max=256, eps=1e-8, kappa_max=w5.kappa_max)
    refs.append(oprob.simulate_chain(ci5, w5b, OPS))
    for c, (N, r) in enumerate(zip((1, 2, 5), refs)):
        assert np.max(np.abs(obs[:, c, :N, :] - r.obs)) < TOL, c
    eng.destroy()


def test_zero_steps_change_nothing(_lib):
    dt, K = 0.1, 6
    ch, ci, d, P = _case(2, dt, K, [0.5, -0.3], [B, None])
    eng = _lib.Engine([d], [P], chi_max=64, eps=1e-12, max_steps=K)
    eng.set_observables(OPS)
    a, _ = eng.observe(OPS)
    eng.step(0)
    assert eng.steps_done() == 0
    b, _ = eng.observe(OPS)
    assert np.array_equal(a, b)
    eng.step(K)
    assert eng.steps_done() == K
    eng.destroy()
