"""Edge cases of the oracle (CPU): a single site (no bond, so its on-site term travels in the
per-site propagator fused into the PT-MPO, App. A.1) and the per-site propagator itself."""
import numpy as np
import scipy.linalg as sla

from oracle import bath, model, problem, pttebd, tempo
from workloads.configs import BathSpec, ChainSpec, Workload


def _local_field(eps, dt):
    # exp(L dt) of L = -i[eps s^z, .] on one site (row-major vec)
    return sla.expm(model.hamiltonian_liouvillian(model.onsite_hamiltonian(eps)) * dt)


def test_single_site_field_in_the_local_propagator_closed_form():
    # N = 1 with a dephasing bath: no bond carries the field, the per-site propagator does
    # (fused into the PT-MPO). sigma^x inserted on |u><u| gives rho_du(0) = 1 and
    # <sigma^x>(t) = rho_du(t) = e^{i eps t} e^{-Re G(t)} (independent-boson model, exact here:
    # the field and the coupling commute and sum eta = G).
    b = BathSpec(0.16, 4.0, 1.0)
    eps0, dt, K = 0.8, 0.2, 12
    ch = ChainSpec(N=1, eps=(eps0,), J=(), init="u", baths=(b,))
    P = tempo.build_pt_mpo(b, dt, K, 1e-11, 128)
    Pf = [pttebd.fuse_local(Pk, _local_field(eps0, dt)) for Pk in P]
    ci = problem.ChainInputs(1, [model.product_state_vector("u")], [], [], [Pf])
    w = Workload("t", (ch,), dt=dt, K=K, chi_max=8, eps=1e-14, kappa_max=128)
    r = problem.simulate_chain(ci, w, [model.SX], insert=(0, model.SX, "left"))
    t = np.arange(K + 1) * dt
    want = np.exp(1j * eps0 * t) * np.exp(-bath.G_closed(b, t).real)
    assert np.max(np.abs(r.obs[:, 0, 0] - want)) < 1e-9


def test_local_propagator_on_a_site_without_bath_equals_absorbing_the_field():
    # a field applied once per step by the site propagator (identity PT-MPO, kappa = 1) gives the
    # same result as the field absorbed into the bond gates when it commutes with the bond (J = 0)
    dt, K = 0.1, 10
    ch_a = ChainSpec(N=2, eps=(0.0, 0.7), J=((0.0, 0.0, 0.0),), init="uu", baths=(None, None))
    ch_b = ChainSpec(N=2, eps=(0.0, 0.0), J=((0.0, 0.0, 0.0),), init="uu", baths=(None, None))
    w = Workload("t", (ch_a,), dt=dt, K=K, chi_max=16, eps=1e-14, kappa_max=1)
    ci_a = problem.build_inputs(w)[0]
    wb = Workload("t", (ch_b,), dt=dt, K=K, chi_max=16, eps=1e-14, kappa_max=1)
    ci_b = problem.build_inputs(wb)[0]
    ident = [np.eye(4, dtype=complex).reshape(1, 4, 4, 1)] * K
    ci_b.pt = [None, [pttebd.fuse_local(P, _local_field(0.7, dt)) for P in ident]]
    ins = (1, model.SX, "left")
    a = problem.simulate_chain(ci_a, w, [model.SX, model.SY], insert=ins)
    b_ = problem.simulate_chain(ci_b, wb, [model.SX, model.SY], insert=ins)
    assert np.max(np.abs(a.obs - b_.obs)) < 1e-12
