"""Liouville-space conventions, chain Hamiltonians and two-site gates (oracle).

Conventions (the paper fixes Liouville space, Sec. II.A / App. A.1, but not the index order):
  * basis index 0 = up, sigma^z = diag(1, -1); s = sigma / 2 (Sec. III).
  * row-major vectorisation vec(rho)[i*d + j] = rho[i, j], so vec(A rho B) = (A kron B^T) vec(rho).
  * Tr(O rho) = vec(O^T) . vec(rho) (unconjugated dot product); the trace vector is vec(I).
  * two-site Liouville indices are grouped per site: (p_n, p_{n+1}) with p = i*d + j, the gate
    index being p_n * d^2 + p_{n+1}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

D = 2
D2 = 4
SX = np.array([[0, 1], [1, 0]], dtype=complex)
SY = np.array([[0, -1j], [1j, 0]], dtype=complex)
SZ = np.array([[1, 0], [0, -1]], dtype=complex)
ID2 = np.eye(2, dtype=complex)
PAULI = {"x": SX, "y": SY, "z": SZ}
SPIN_HALF = {k: v / 2 for k, v in PAULI.items()}


def vec(rho):
    """Row-major vectorisation vec(rho)[i*d+j] = rho[i,j]."""
    return np.asarray(rho, dtype=complex).reshape(-1)


def unvec(v, d=D):
    return np.asarray(v).reshape(d, d)


def trace_vector(d=D):
    """tau with tau . vec(rho) = Tr(rho)."""
    return np.eye(d, dtype=complex).reshape(-1)


def op_vector(O):
    """vec(O^T): op_vector(O) . vec(rho) = Tr(O rho)."""
    return np.asarray(O, dtype=complex).T.reshape(-1)


def left_superop(A):
    """Liouville matrix of rho -> A rho (App. A.4, the left-acting super-operator)."""
    A = np.asarray(A, dtype=complex)
    return np.kron(A, np.eye(A.shape[0]))


def right_superop(A):
    """Liouville matrix of rho -> rho A (App. A.4, the right-acting super-operator)."""
    A = np.asarray(A, dtype=complex)
    return np.kron(np.eye(A.shape[0]), A.T)


def hamiltonian_liouvillian(H):
    """L = -i [H, .] in row-major vec: -i (H kron I - I kron H^T)  (Sec. II.A)."""
    H = np.asarray(H, dtype=complex)
    n = H.shape[0]
    I = np.eye(n)
    return -1j * (np.kron(H, I) - np.kron(I, H.T))


def product_state_vector(ch):
    """vec of the pure product state |s><s| for 'u'/'d'."""
    if ch == "u":
        return vec(np.array([[1, 0], [0, 0]], dtype=complex))
    if ch == "d":
        return vec(np.array([[0, 0], [0, 1]], dtype=complex))
    raise ValueError(ch)


# --- chain Hamiltonians (Eq. (xyz-spin-chain), Eq. (xy-spin-chain)) -----------------------

def onsite_hamiltonian(eps_n):
    """H^S_n = eps_n s^z."""
    return eps_n * SPIN_HALF["z"]


def bond_coupling(J):
    """K_{n,n+1} = sum_g J^g s^g (x) s^g (two-site Hilbert space, site n is the left factor)."""
    Jx, Jy, Jz = J
    return sum(Jg * np.kron(SPIN_HALF[g], SPIN_HALF[g]) for Jg, g in ((Jx, "x"), (Jy, "y"), (Jz, "z")))


def absorbed_bond_hamiltonians(eps, J):
    """K'_{n,n+1} of App. A.1: on-site terms absorbed into the bonds.

    End bonds take the whole on-site term of their end site and half of the inner one; interior
    bonds take half of each. For N = 2 the single bond takes both on-site terms in full.
    """
    N = len(eps)
    H = [onsite_hamiltonian(e) for e in eps]
    out = []
    for b in range(N - 1):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b == N - 2 else 0.5
        Kp = bond_coupling(J[b]) + wl * np.kron(H[b], ID2) + wr * np.kron(ID2, H[b + 1])
        out.append(Kp)
    return out


def chain_hamiltonian(eps, J):
    """Full N-site chain Hamiltonian sum_n H^S_n + sum_n K_{n,n+1} (for exact checks)."""
    N = len(eps)
    dim = 2 ** N
    Hc = np.zeros((dim, dim), dtype=complex)
    for n in range(N):
        Hc += np.kron(np.kron(np.eye(2 ** n), onsite_hamiltonian(eps[n])), np.eye(2 ** (N - n - 1)))
    for b in range(N - 1):
        Hc += np.kron(np.kron(np.eye(2 ** b), bond_coupling(J[b])), np.eye(2 ** (N - b - 2)))
    return Hc


# --- two-site Liouville gates -----------------------------------------------------------

def group_two_site(M):
    """Permute a 16x16 two-site Liouville matrix from ((i1 i2),(j1 j2)) row-major vec order to
    per-site grouping (p1, p2) with p = i*2 + j."""
    T = np.asarray(M).reshape(2, 2, 2, 2, 2, 2, 2, 2)   # out: i1 i2 j1 j2 ; in: i1 i2 j1 j2
    T = T.transpose(0, 2, 1, 3, 4, 6, 5, 7)              # out: i1 j1 i2 j2 ; in: i1 j1 i2 j2
    return T.reshape(16, 16)


def group_sites(M, N):
    """Permute an N-site Liouville matrix (row-major vec of the 2^N x 2^N density matrix) to
    per-site grouping p_0 p_1 ... p_{N-1}."""
    T = np.asarray(M).reshape([2] * (4 * N))
    perm_half = []
    for n in range(N):
        perm_half += [n, N + n]
    perm = perm_half + [2 * N + q for q in perm_half]
    return T.transpose(perm).reshape(4 ** N, 4 ** N)


def gate_expm(Kp, tau):
    """G = exp(L^{K'} tau) by scipy's matrix exponential of the 16x16 Liouvillian, grouped."""
    return group_two_site(sla.expm(hamiltonian_liouvillian(Kp) * tau))


def gate_unitary(Kp, tau):
    """Closed form of the same gate: rho -> U rho U^dagger with U = exp(-i K' tau) from eigh,
    i.e. U kron conj(U) in row-major vec, grouped."""
    w, V = np.linalg.eigh(Kp)
    U = (V * np.exp(-1j * w * tau)[None, :]) @ V.conj().T
    return group_two_site(np.kron(U, U.conj()))


def gate_from_unitary(U):
    """Liouville gate of a two-site unitary U (4x4): U kron conj(U), grouped."""
    return group_two_site(np.kron(U, np.conj(U)))
