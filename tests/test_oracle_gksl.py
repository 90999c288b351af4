"""Pins of the time-local (GKSL) chain terms (App. A.1) and of the two-spin driving generator
(Sec. III.A.3) in the oracle (CPU)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import exact, gksl, model, problem
from workloads import workload
from workloads.configs import ChainSpec, DriveSpec, Workload

XYZ = (1.3, 0.7, 1.2)


def test_damped_dephased_coherence_closed_form():
    # one spin, H = eps s^z, decay rate g and dephasing rate gp: rho_du(t) = e^{(i eps - g/2 - 2 gp) t}
    # and rho_uu(t) = e^{-g t}. N = 2 with J = 0 makes the splitting exact (commuting on-site terms).
    eps0, g, gp, dt, K = 0.8, 0.3, 0.05, 0.1, 30
    ch = ChainSpec(N=2, eps=(eps0, 0.2), J=((0.0, 0.0, 0.0),), init="uu", baths=(None, None),
                   gksl=((0, "minus", g), (0, "z", gp), (1, "plus", 0.1)))
    w = Workload("t", (ch,), dt=dt, K=K, chi_max=16, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    t = dt * np.arange(K + 1)
    r = problem.simulate_chain(ci, w, [model.SZ])
    assert np.max(np.abs(r.obs[:, 0, 0] - (2 * np.exp(-g * t) - 1))) < 1e-12
    # sigma^x inserted on the left at t = 0 turns |u><u| into |d><u|; <sigma^x> = rho_du + rho_ud
    r = problem.simulate_chain(ci, w, [model.SX], insert=(0, model.SX, "left"))
    assert np.max(np.abs(r.obs[:, 0, 0] - np.exp((1j * eps0 - g / 2 - 2 * gp) * t))) < 1e-12
    assert np.max(np.abs(r.trace - 0.0)) < 1e-12          # Tr(sigma^x rho) insertion is traceless


def test_gksl_chain_converges_to_the_full_lindbladian():
    # N = 3 XYZ chain with decay, dephasing and pumping on different sites: PT-TEBD without
    # truncation -> expm of the whole Lindbladian (each term added once), error O(dt^2)
    ch = ChainSpec(N=3, eps=(0.5, 0.0, -0.3), J=(XYZ, XYZ), init="udu", baths=(None,) * 3,
                   gksl=((0, "minus", 0.2), (1, "z", 0.1), (2, "plus", 0.15)))
    errs = []
    for dt, K in ((0.1, 10), (0.05, 20)):
        w = Workload("t", (ch,), dt=dt, K=K, chi_max=64, eps=1e-14, kappa_max=1)
        ci = problem.build_inputs(w)[0]
        r = problem.simulate_chain(ci, w, [model.SZ, model.SX])
        ex = exact.full_liouvillian_run(ch, dt, K, [model.SZ, model.SX])
        errs.append(np.max(np.abs(r.obs[-1] - ex[-1])))
        ft = exact.full_trotter_run(3, ci.rho0, ci.gates_q, ci.gates_h, K, [model.SZ, model.SX])
        assert np.max(np.abs(r.obs - ft)) < 1e-12
        assert np.max(np.abs(r.trace - 1.0)) < 1e-12      # GKSL generators preserve the trace
    assert errs[0] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_planted_wrong_absorption_weight_is_caught(monkeypatch):
    # halving the end sites' dissipators (a plausible slip in the absorption) breaks convergence
    ch = ChainSpec(N=3, eps=(0.5, 0.0, -0.3), J=(XYZ, XYZ), init="udu", baths=(None,) * 3,
                   gksl=((0, "minus", 0.4),))
    real = gksl.onsite_dissipators
    monkeypatch.setattr(gksl, "onsite_dissipators",
                        lambda c: [0.5 * d if n == 0 else d for n, d in enumerate(real(c))])
    w = Workload("t", (ch,), dt=0.05, K=20, chi_max=64, eps=1e-14, kappa_max=1)
    ci = problem.build_inputs(w)[0]
    r = problem.simulate_chain(ci, w, [model.SZ])
    monkeypatch.setattr(gksl, "onsite_dissipators", real)
    ex = exact.full_liouvillian_run(ch, 0.05, 20, [model.SZ])
    assert np.max(np.abs(r.obs[-1] - ex[-1])) > 1e-2


def test_drive_generator_relaxes_the_pair_to_its_gibbs_state():
    ch = workload("xyz7_twospin_drive").chains[0]
    L = gksl.drive_generator(ch)
    tau = np.kron(model.trace_vector(), model.trace_vector())          # grouped trace vector
    assert np.max(np.abs(tau @ L)) < 1e-14                               # trace preserving
    g = gksl.gibbs_pair_vector(ch)
    assert np.max(np.abs(L @ g)) < 1e-14                                 # Gibbs state is stationary
    w_ = np.sort(np.abs(np.linalg.eigvals(L)))
    assert w_[0] < 1e-13 and w_[1] > 1e-3                                # and the only one
    # from any pair state the generator alone reaches it
    v0 = np.kron(model.product_state_vector("u"), model.product_state_vector("d"))
    v = sla.expm(L * 60.0) @ v0
    assert np.max(np.abs(v - g)) < 1e-10
    # Gibbs weights: <s^z_0> of the pair equals the thermal value from H_B's spectrum
    H = gksl.drive_pair_hamiltonian(ch)
    E, V = np.linalg.eigh(H)
    p = np.exp(-E / ch.drive.T)
    p /= p.sum()
    sz0 = np.kron(model.SZ, model.ID2)
    thermal = np.sum(p * np.real(np.einsum("ia,ij,ja->a", V.conj(), sz0, V)))
    rho = g.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(4, 4)
    assert abs(np.trace(sz0 @ rho).real - thermal) < 1e-12


def test_driven_chain_matches_full_lindbladian_and_relaxes():
    # the comparison network with 3 sites (pair + one chain spin): O(dt^2) convergence to the full
    # generator, trace 1
    ch = ChainSpec(N=3, eps=(0.0, 0.0, 0.0), J=(XYZ, XYZ), init="udu", baths=(None,) * 3,
                   drive=DriveSpec(T=1.6, rate=1.0))
    errs = []
    for dt, K in ((0.1, 10), (0.05, 20)):
        w = Workload("t", (ch,), dt=dt, K=K, chi_max=64, eps=1e-14, kappa_max=1)
        ci = problem.build_inputs(w)[0]
        r = problem.simulate_chain(ci, w, [model.SZ])
        ex = exact.full_liouvillian_run(ch, dt, K, [model.SZ])
        errs.append(np.max(np.abs(r.obs[-1] - ex[-1])))
        assert np.max(np.abs(r.trace - 1.0)) < 1e-12
    assert errs[0] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5
