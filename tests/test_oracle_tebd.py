"""Pins of the oracle's PT-TEBD: exact Liouvillian / Trotter product (alpha = 0), brute-force
influence-functional path sums, an exact single-mode bath, the pure-dephasing closed form,
PT-MPO causality, and the trace / hermiticity / conservation invariants."""
import numpy as np
import pytest

from workloads import BathSpec, workload
from workloads.configs import ChainSpec, Workload
from oracle import bath, exact, model, pttebd, problem, tempo

OPS = [model.SZ, model.SX, model.SY]


def _closed_chain(N, eps, init, J=(1.3, 0.7, 1.2)):
    return ChainSpec(N=N, eps=tuple(eps), J=tuple([J] * (N - 1)), init=init, baths=(None,) * N)


@pytest.mark.parametrize("N,init", [(2, "ud"), (3, "udu"), (4, "uudd")])
def test_markovian_limit_equals_full_trotter_product(N, init):
    # alpha = 0: PT-TEBD is Liouville TEBD (Sec. II.A); without truncation it must reproduce the
    # product of the same gates as full 4^N matrices to rounding.
    ch = _closed_chain(N, [0.5, 0.2, -0.3, 0.1][:N], init)
    w = Workload("t", (ch,), dt=0.05, K=20, chi_max=4 ** N, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    r = problem.simulate_chain(ci, w, OPS)
    ft = exact.full_trotter_run(N, ci.rho0, ci.gates_q, ci.gates_h, w.K, OPS)
    assert np.max(np.abs(r.obs - ft)) < 1e-12


@pytest.mark.parametrize("N", [3, 4])
def test_markovian_limit_converges_to_expm_at_second_order(N):
    ch = _closed_chain(N, [0.5, 0.2, -0.3, 0.1][:N], "udud"[:N])
    errs = []
    for dt, K in [(0.05, 20), (0.025, 40)]:
        w = Workload("t", (ch,), dt=dt, K=K, chi_max=4 ** N, eps=1e-14, kappa_max=1)
        ci = problem.build_inputs(w)[0]
        r = problem.simulate_chain(ci, w, OPS)
        ex = exact.full_liouvillian_run(ch, dt, K, OPS)
        errs.append(np.max(np.abs(r.obs[-1] - ex[-1])))
    assert errs[0] < 1e-3
    assert 3.6 < errs[0] / errs[1] < 4.4          # O(dt^2): halving dt divides the error by 4


def test_qr_and_svd_reductions_agree_without_truncation():
    # The paper's truncated SVDs of the outer blocks and the exact QR reductions give the same D up to a unitary
    # change of basis, hence the same singular values and observables when nothing is truncated.
    w = workload("xyz3_onebath", K=8, kappa_max=64, eps=1e-13)
    ci = problem.build_inputs(w)[0]
    a = problem.simulate_chain(ci, w, OPS, variant="qr", keep_lambdas=True)
    b = problem.simulate_chain(ci, w, OPS, variant="svd", keep_lambdas=True)
    assert np.max(np.abs(a.obs - b.obs)) < 1e-10
    for la, lb in zip(a.lambdas[-1], b.lambdas[-1]):
        n = min(len(la), len(lb))
        assert np.max(np.abs(la[:n] - lb[:n])) < 1e-10


def test_two_time_insertion_matches_full_trotter_product():
    # App. A.4: a left-acting super-operator inserted at t = 0, raw (untraced-normalised) readout.
    ch = _closed_chain(4, [0.5, 0, 0, 0], "udud")
    w = Workload("t", (ch,), dt=0.05, K=15, chi_max=256, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    for side in ("left", "right"):
        ins = (2, model.SX, side)
        r = problem.simulate_chain(ci, w, [model.SX], insert=ins)
        ft = exact.full_trotter_run(4, ci.rho0, ci.gates_q, ci.gates_h, w.K, [model.SX], insert=ins)
        assert np.max(np.abs(r.obs - ft)) < 1e-12


def _two_site_bath_chain():
    return ChainSpec(N=2, eps=(0.5, 0.3), J=((1.3, 0.7, 1.2),), init="ud", baths=(None, None))


def test_single_mode_bath_exact_equals_path_sum():
    # Pins the influence functional (signs and imaginary parts of eta, slot ordering): an exact
    # simulation of chain (x) one harmonic mode equals the discretised Feynman-Vernon path sum.
    ch = _two_site_bath_chain()
    g, w0, T, dt, K = 0.7, 1.3, 0.8, 0.2, 5
    sm = exact.single_mode_run(ch, g, w0, T, dt, K, OPS, nmax=40)
    eta = bath.eta_from_G(lambda t: bath.single_mode_G(g * g, w0, T, t), dt, K)
    gq, _ = problem.chain_gates(ch, dt)
    rho0 = [model.product_state_vector(c) for c in ch.init]
    ps = exact.path_sum_run(rho0, gq, eta, K, OPS)
    assert np.max(np.abs(sm - ps)) < 1e-12


@pytest.mark.parametrize("b", [BathSpec(0.16, 4.0, 5.0), BathSpec(0.32, 4.0, 0.5)])
def test_pt_tebd_equals_brute_force_path_sum(b):
    # TEMPO-compressed PT-MPO (eps_TEMPO -> 0) + PT-TEBD == uncompressed path sum, N = 2, K = 6.
    ch = _two_site_bath_chain()
    dt, K = 0.1, 6
    eta = bath.eta_coefficients(b, dt, K)
    gq, gh = problem.chain_gates(ch, dt)
    rho0 = [model.product_state_vector(c) for c in ch.init]
    ps = exact.path_sum_run(rho0, gq, eta, K, OPS)
    P = tempo.build_pt_mpo_from_eta(eta, K, 1e-14, 4 ** K)
    ci = problem.ChainInputs(2, rho0, gq, gh, [P, None])
    w = Workload("t", (ch,), dt=dt, K=K, chi_max=4 ** 4, eps=1e-14, kappa_max=4 ** K)
    r = problem.simulate_chain(ci, w, OPS)
    assert np.max(np.abs(r.obs - ps)) < 1e-10


def test_pure_dephasing_closed_form():
    # H = eps s^z coupled via s^z: rho_ud(t) = rho_ud(0) e^{-i eps t} e^{-Re G(t)} (independent boson
    # model). Exact under the discretisation because sum eta = G (full memory).
    b = BathSpec(0.16, 4.0, 1.0)
    eps0, dt, K = 0.8, 0.2, 12
    ch = ChainSpec(N=2, eps=(eps0, 0.0), J=((0.0, 0.0, 0.0),), init="uu", baths=(b, None))
    gq, gh = problem.chain_gates(ch, dt)
    plus = model.vec(np.full((2, 2), 0.5, dtype=complex))
    P = tempo.build_pt_mpo(b, dt, K, 1e-11, 128)
    ci = problem.ChainInputs(2, [plus, model.product_state_vector("u")], gq, gh, [P, None])
    w = Workload("t", (ch,), dt=dt, K=K, chi_max=64, eps=1e-14, kappa_max=128)
    r = problem.simulate_chain(ci, w, [model.SX, model.SY])
    rho_ud = (r.obs[:, 0, 0] - 1j * r.obs[:, 0, 1]) / 2
    t = np.arange(K + 1) * dt
    want = 0.5 * np.exp(-1j * eps0 * t) * np.exp(-bath.G_closed(b, t).real)
    assert np.max(np.abs(rho_ud - want)) < 1e-9


def test_pt_mpo_causality_and_cap_gauge():
    # App. A.3 containment: tracing the output of P^(k) against the next cap gives tau_i C^(k-1)[a]
    # (any normalised input gives the same reduced past). Caps have unit norm after the gauge.
    b = BathSpec(0.1, 4.0, 1.0)
    P = tempo.build_pt_mpo(b, 0.1, 20, 1e-9, 64)
    C = pttebd.caps(P)
    for k in range(1, len(P) + 1):
        t = np.einsum("aiob,o,b->ai", P[k - 1], pttebd.TAU, C[k])
        assert np.max(np.abs(t - np.outer(C[k - 1], pttebd.TAU))) < 1e-6
        if k < len(P):
            assert abs(np.linalg.norm(C[k]) - 1) < 1e-12


def test_cap_gauge_leaves_observables_unchanged():
    b = BathSpec(0.1, 4.0, 1.0)
    w = workload("xyz3_onebath", K=10)
    ch = w.chains[0]
    eta = bath.eta_coefficients(b, w.dt, w.K)
    A = tempo.build_influence_mps(eta, w.K, w.K, 1e-9, 64)
    raw = tempo.pt_mpo_from_influence(A)
    gauged = tempo.cap_gauge(raw)
    gq, gh = problem.chain_gates(ch, w.dt)
    rho0 = [model.product_state_vector(c) for c in ch.init]
    r1 = problem.simulate_chain(problem.ChainInputs(3, rho0, gq, gh, [raw, None, None]), w, OPS)
    r2 = problem.simulate_chain(problem.ChainInputs(3, rho0, gq, gh, [gauged, None, None]), w, OPS)
    assert np.max(np.abs(r1.obs - r2.obs)) < 1e-12


def test_invariants_on_three_site_workload():
    w = workload("xyz3_onebath")
    ci = problem.build_inputs(w)[0]
    r = problem.simulate_chain(ci, w, OPS)
    assert np.max(np.abs(r.trace - 1)) < 1e-4                  # Tr rho = 1 up to PT-MPO compression
    assert np.max(np.abs(r.obs.imag)) < 1e-10                  # Hermitian rho: real <sigma^a>
    assert np.max(np.abs(r.obs.real)) <= 1 + 1e-6


def test_isotropic_xy_conserves_total_sz():
    # XY coupling and s^z baths commute with sum_n s^z_n (Sec. IV).
    b = BathSpec(0.05, 3.0, 0.8)
    N = 5
    ch = ChainSpec(N=N, eps=(0.0,) * N, J=((1.0, 1.0, 0.0),) * (N - 1), init="ddudd", baths=(b,) * N)
    w = Workload("t", (ch,), dt=0.1, K=10, chi_max=64, eps=1e-10, kappa_max=8)
    ci = problem.build_inputs(w)[0]
    r = problem.simulate_chain(ci, w, [model.SZ], normalize=True)
    tot = r.obs[:, :, 0].real.sum(axis=1)
    assert np.max(np.abs(tot - tot[0])) < 1e-6
    assert abs(tot[0] - (-3.0)) < 1e-12


def test_planted_sign_error_in_eta_is_caught(monkeypatch):
    # A plausible mistake (conjugated eta in the influence factors) must fail the single-mode pin.
    orig = tempo.influence_factors
    monkeypatch.setattr(tempo, "influence_factors", lambda eta: orig(np.conj(eta)))
    ch = _two_site_bath_chain()
    g, w0, T, dt, K = 0.7, 1.3, 0.8, 0.2, 4
    sm = exact.single_mode_run(ch, g, w0, T, dt, K, OPS, nmax=40)
    eta = bath.eta_from_G(lambda t: bath.single_mode_G(g * g, w0, T, t), dt, K)
    gq, _ = problem.chain_gates(ch, dt)
    rho0 = [model.product_state_vector(c) for c in ch.init]
    ps = exact.path_sum_run(rho0, gq, eta, K, OPS)
    assert np.max(np.abs(sm - ps)) > 1e-4


def test_planted_transposed_gate_is_caught():
    # Swapping the two sites inside the grouped gate (a plausible index-order slip) must fail the
    # exact Trotter pin.
    ch = _closed_chain(3, [0.5, 0.2, -0.3], "udu")
    w = Workload("t", (ch,), dt=0.05, K=10, chi_max=64, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    ft = exact.full_trotter_run(3, ci.rho0, ci.gates_q, ci.gates_h, w.K, OPS)
    def swap(g):
        return g.reshape(4, 4, 4, 4).transpose(1, 0, 3, 2).reshape(16, 16)
    bad = problem.ChainInputs(3, ci.rho0, [swap(g) for g in ci.gates_q], [swap(g) for g in ci.gates_h],
                              ci.pt)
    r = problem.simulate_chain(bad, w, OPS)
    assert np.max(np.abs(r.obs - ft)) > 1e-3
