"""Time-local (GKSL) terms of the chain Liouvillian (oracle; test infrastructure).

ORACLE: imported only by tests/, __graft_entry__.smoke() and bench.py's CPU baseline.

App. A.1 allows the system Liouvillians L^S_n to carry GKSL dissipators
    D[L] rho = L rho L^dag - (1/2) {L^dag L, rho}
with operators L on site n; like the on-site Hamiltonians they are absorbed into the bond
Liouvillians L^{K'}_{n,n+1} (whole on the end bonds' outer sites, half elsewhere), and the gates
become exp(L^{K'} tau) of a non-Hermitian generator. Sec. III.A.3's comparison network adds a
two-spin driving generator L_B to the first bond, L^{K'}_{0,1} -> L^{K'}_{0,1} + L_B. The paper
takes L_B from the cited two-spin bath protocol without stating it; the reading here (listed in
the design notes) is a detailed-balance generator in the eigenbasis |a> of the pair's own
Hamiltonian H_B = eps_0 s^z_0 + eps_1 s^z_1 + K_{0,1}: jumps |b> -> |a> with
L_ab = sqrt(rate r_ab) |a><b|, r_ab = 1 / (1 + exp((E_a - E_b) / T)), whose unique steady state
is the Gibbs state exp(-H_B / T) / Z.

All superoperators use the oracle's row-major vectorisation (vec(A rho B) = (A kron B^T) vec rho);
two-site ones are returned in per-site grouping like the gates.
"""
from __future__ import annotations

import numpy as np

from . import model

JUMP_OPS = {
    "minus": np.array([[0, 0], [1, 0]], dtype=complex),     # |down><up| (index 0 = up)
    "plus": np.array([[0, 1], [0, 0]], dtype=complex),      # |up><down|
    "z": model.SZ,
}


def dissipator(L):
    """Liouville matrix of D[L]: L kron conj(L) - (1/2)(L^dag L kron I) - (1/2)(I kron (L^dag L)^T)."""
    L = np.asarray(L, dtype=complex)
    n = L.shape[0]
    I = np.eye(n)
    LdL = L.conj().T @ L
    return np.kron(L, L.conj()) - 0.5 * np.kron(LdL, I) - 0.5 * np.kron(I, LdL.T)


def onsite_dissipators(ch):
    """[N] 4x4 Liouville matrices: the sum of the GKSL terms of each site (zero where none)."""
    out = [np.zeros((4, 4), dtype=complex) for _ in range(ch.N)]
    for site, op, rate in ch.gksl:
        out[site] = out[site] + dissipator(np.sqrt(rate) * JUMP_OPS[op])
    return out


def drive_pair_hamiltonian(ch):
    """H_B of the driven pair (sites 0, 1): its own fields and its coupling."""
    return (np.kron(model.onsite_hamiltonian(ch.eps[0]), model.ID2)
            + np.kron(model.ID2, model.onsite_hamiltonian(ch.eps[1])) + model.bond_coupling(ch.J[0]))


def drive_generator(ch):
    """Grouped 16x16 L_B of the driven pair (the detailed-balance reading above)."""
    H = drive_pair_hamiltonian(ch)
    E, V = np.linalg.eigh(H)
    T, rate = ch.drive.T, ch.drive.rate
    L = np.zeros((16, 16), dtype=complex)
    for a in range(4):
        for b in range(4):
            if a == b:
                continue
            r = 1.0 / (1.0 + np.exp((E[a] - E[b]) / T))
            jump = np.sqrt(rate * r) * np.outer(V[:, a], V[:, b].conj())
            L += dissipator(jump)
    return model.group_two_site(L)


def gibbs_pair_vector(ch):
    """Grouped vec of exp(-H_B / T) / Z (the steady state L_B is built to have)."""
    H = drive_pair_hamiltonian(ch)
    E, V = np.linalg.eigh(H)
    p = np.exp(-(E - E.min()) / ch.drive.T)
    rho = (V * (p / p.sum())) @ V.conj().T
    return _group_pair_vec(rho)


def _group_pair_vec(rho):
    # row-major vec of a two-site density matrix ((i1 i2),(j1 j2)) -> grouped (i1 j1, i2 j2)
    return np.asarray(rho).reshape(2, 2, 2, 2).transpose(0, 2, 1, 3).reshape(16)


def bond_liouvillians(ch):
    """Grouped 16x16 L^{K'}_{b,b+1} with the on-site Hamiltonians and dissipators absorbed
    (whole on the chain's end sites, half on interior ones) and L_B added to bond 0."""
    N = ch.N
    Kp = model.absorbed_bond_hamiltonians(ch.eps, ch.J)
    Ds = onsite_dissipators(ch)
    I4 = np.eye(4)
    out = []
    for b in range(N - 1):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b == N - 2 else 0.5
        L = model.group_two_site(model.hamiltonian_liouvillian(Kp[b]))
        L = L + wl * np.kron(Ds[b], I4) + wr * np.kron(I4, Ds[b + 1])
        if b == 0 and ch.drive is not None:
            L = L + drive_generator(ch)
        out.append(L)
    return out


def full_liouvillian(ch):
    """The whole grouped 4^N chain Liouvillian, each term added once (for the exact checks)."""
    N = ch.N
    H = model.chain_hamiltonian(ch.eps, ch.J)
    L = model.group_sites(model.hamiltonian_liouvillian(H), N)
    for n, Dn in enumerate(onsite_dissipators(ch)):
        L = L + np.kron(np.kron(np.eye(4 ** n), Dn), np.eye(4 ** (N - n - 1)))
    if ch.drive is not None:
        L = L + np.kron(drive_generator(ch), np.eye(4 ** (N - 2)))
    return L
