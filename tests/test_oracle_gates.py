"""Pins of the oracle's Liouville conventions and two-site gates (Sec. II.A, App. A.1)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import model
from oracle.truncation import truncation_rank


def _rand_herm(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (a + a.conj().T) / 2


def _rand_rho(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    r = a @ a.conj().T
    return r / np.trace(r)


def test_vec_conventions():
    rng = np.random.default_rng(1)
    A, B, R = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2)) for _ in range(3))
    assert np.allclose(model.vec(A @ R @ B), np.kron(A, B.T) @ model.vec(R))
    assert np.allclose(model.left_superop(A) @ model.vec(R), model.vec(A @ R))
    assert np.allclose(model.right_superop(A) @ model.vec(R), model.vec(R @ A))
    assert np.isclose(model.op_vector(A) @ model.vec(R), np.trace(A @ R))
    assert np.isclose(model.trace_vector() @ model.vec(R), np.trace(R))


@pytest.mark.parametrize("tau", [0.025, 0.05, 0.3])
def test_gate_expm_equals_unitary_conjugation(tau):
    rng = np.random.default_rng(2)
    Kp = _rand_herm(rng, 4)
    assert np.max(np.abs(model.gate_expm(Kp, tau) - model.gate_unitary(Kp, tau))) < 1e-13


def test_gate_acts_as_unitary_conjugation_on_product_states():
    # grouped gate on vec(rho1) (x) vec(rho2) == vec of U (rho1 (x) rho2) U^dag regrouped per site
    rng = np.random.default_rng(3)
    Kp = _rand_herm(rng, 4)
    tau = 0.37
    U = sla.expm(-1j * Kp * tau)
    r1, r2 = _rand_rho(rng, 2), _rand_rho(rng, 2)
    out = model.gate_expm(Kp, tau) @ np.kron(model.vec(r1), model.vec(r2))
    full = U @ np.kron(r1, r2) @ U.conj().T           # [(i1 i2),(j1 j2)]
    grouped = full.reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(-1)
    assert np.max(np.abs(out - grouped)) < 1e-14


def test_absorbed_bond_hamiltonians_sum_to_chain():
    # sum_b K'_b embedded == full chain Hamiltonian (App. A.1: L_chain = sum_b L^{K'}_b)
    eps = (0.5, -0.2, 0.7, 0.1)
    J = ((1.3, 0.7, 1.2), (0.9, 1.1, 0.4), (0.2, 0.3, 1.5))
    Kp = model.absorbed_bond_hamiltonians(eps, J)
    N = 4
    tot = sum(np.kron(np.kron(np.eye(2 ** b), Kp[b]), np.eye(2 ** (N - b - 2))) for b in range(N - 1))
    assert np.allclose(tot, model.chain_hamiltonian(eps, J), atol=1e-14)
    # N = 2: one bond takes both on-site terms in full
    Kp2 = model.absorbed_bond_hamiltonians((0.5, 0.3), ((1, 1, 1),))
    assert np.allclose(Kp2[0], model.chain_hamiltonian((0.5, 0.3), ((1, 1, 1),)))


def test_gate_preserves_trace_and_hermiticity():
    rng = np.random.default_rng(4)
    Kp = _rand_herm(rng, 4)
    G = model.gate_expm(Kp, 0.2)
    tt = np.kron(model.trace_vector(), model.trace_vector())
    assert np.allclose(tt @ G, tt, atol=1e-14)


def test_truncation_rule_brute_force():
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        s = np.sort(rng.random(n) * 10.0 ** (-rng.integers(0, 12, n)))[::-1]
        eps = 10.0 ** (-float(rng.integers(1, 10)))
        chi_max = int(rng.integers(1, 14))
        got = truncation_rank(s, eps, chi_max, multiplet_tol=0.0)
        # brute force: smallest chi with discarded norm < eps * s_max, then cap
        want = n
        for c in range(1, n + 1):
            if np.sqrt(np.sum(s[c:] ** 2)) < eps * s[0]:
                want = c
                break
        want = max(1, min(want, chi_max))
        assert got == want


def test_truncation_keeps_multiplets_whole():
    s = np.array([1.0, 0.5, 0.5, 0.5, 1e-9])
    assert truncation_rank(s, 0.6, 10) == 4          # eps cut at 2 -> extended over the triplet
    assert truncation_rank(s, 1e-12, 3) == 1          # cap at 3 splits the triplet -> drop it
    assert truncation_rank(np.array([1.0, 0.0, 0.0]), 1e-30, 5) == 1   # exact zeros dropped
