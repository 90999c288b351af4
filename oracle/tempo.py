"""Discretised influence functional and its PT-MPO (oracle).

The paper takes PT-MPOs for Gaussian bosonic baths from PT-TEMPO (Sec. II.A; App. B.1, whose
parameters are dt, Delta K_max and eps_TEMPO) without restating the algorithm. The oracle builds
them from the standard quasi-adiabatic influence functional written in the eigenbasis of the
coupling operator S = s^z (eigenvalues s(up) = +1/2, s(down) = -1/2). For the Liouville index
p = i*2 + j of the bath site, s+ = s(i), s- = s(j), and for a path p_1 .. p_K
    F = prod_k I_0(p_k) prod_{0 < k-k' <= DK} I_{k-k'}(p_k, p_k'),
    I_0(p)      = exp[-(s+ - s-)(eta_0 s+ - conj(eta_0) s-)],
    I_D(p, p')  = exp[-(s+ - s-)(eta_D s'+ - conj(eta_D) s'-)],
with eta from ``oracle.bath``. F is assembled as an MPS over the K time slots (physical index p_k)
by multiplying in one "influence line" per source time k' -- the MPO that copies p_k' forward and
multiplies in I_{k-k'}(p_k, p_k') at each later slot -- and compressing after each line with the
relative SVD rule (eps_TEMPO) and the bond cap kappa_max. Because the influence functional only
multiplies the path weight, the PT-MPO tensors are diagonal in (input, output):
    P^(k)[a, i, o, b] = delta_io F_k[a, i, b].
Finally each tensor is rescaled so that the cap tensors of App. A.3 have unit norm (a gauge that
keeps intermediate states O(1) and leaves every observable unchanged).
"""
from __future__ import annotations

import numpy as np

from .truncation import truncation_rank
from . import bath as _bath

S_EIG = np.array([0.5, -0.5])
SP = S_EIG[np.arange(4) // 2]     # s+ of Liouville index p = i*2 + j
SM = S_EIG[np.arange(4) % 2]      # s- of p


def influence_factors(eta):
    """I_0[p] and I_D[p_later, p_earlier] for D = 1..len(eta)-1."""
    I0 = np.exp(-(SP - SM) * (eta[0] * SP - np.conj(eta[0]) * SM))
    ID = [None]
    for D in range(1, len(eta)):
        ID.append(np.exp(-(SP - SM)[:, None] * (eta[D] * SP[None, :] - np.conj(eta[D]) * SM[None, :])))
    return I0, ID


def influence_functional_value(path, eta, n_memory):
    """F for one explicit path (p_1 .. p_K): the definition, used by brute-force checks."""
    I0, ID = influence_factors(eta)
    K = len(path)
    f = 1.0 + 0j
    for k in range(K):
        f *= I0[path[k]]
        for kp in range(k):
            D = k - kp
            if D <= n_memory:
                f *= ID[D][path[k], path[kp]]
    return f


def _right_canonicalise(A):
    """QR sweep right -> left; returns the MPS with the centre (all weight) at site 0."""
    A = [a.copy() for a in A]
    for k in range(len(A) - 1, 0, -1):
        kl, d, kr = A[k].shape
        q, r = np.linalg.qr(A[k].reshape(kl, d * kr).T)        # A^T = q r  ->  A = r^T q^T
        A[k] = q.T.reshape(-1, d, kr)
        A[k - 1] = np.einsum("apb,bc->apc", A[k - 1], r.T)
    return A


def _move_centre_right(A, k):
    kl, d, kr = A[k].shape
    q, r = np.linalg.qr(A[k].reshape(kl * d, kr))
    A[k] = q.reshape(kl, d, -1)
    A[k + 1] = np.einsum("ab,bpc->apc", r, A[k + 1])


def build_influence_mps(eta, K, n_memory, eps, kappa_max):
    """The influence functional of K time slots as a compressed MPS [F_1 .. F_K], F_k[a, p, b]."""
    I0, ID = influence_factors(eta)
    A = [I0.reshape(1, 4, 1).astype(complex) for _ in range(K)]
    A = _right_canonicalise(A)                                   # centre at 0
    delta = np.eye(4, dtype=complex)
    for src in range(K):
        end = min(K - 1, src + n_memory)
        if end > src:
            # -- multiply in the influence line of source slot `src` on slots src .. end
            kl, _, kr = A[src].shape
            A[src] = np.einsum("apb,pc->apbc", A[src], delta).reshape(kl, 4, kr * 4)
            for k in range(src + 1, end + 1):
                F = ID[k - src]                                   # [p_k, p_src]
                kl, _, kr = A[k].shape
                if k < end:
                    t = np.einsum("apb,pc,cd->acpbd", A[k], F, delta)
                    A[k] = t.reshape(kl * 4, 4, kr * 4)
                else:
                    A[k] = np.einsum("apb,pc->acpb", A[k], F).reshape(kl * 4, 4, kr)
            # -- restore canonical form over the span and truncate right -> left
            for k in range(src, end):
                _move_centre_right(A, k)
            for k in range(end, src, -1):
                kl, d, kr = A[k].shape
                u, s, vh = np.linalg.svd(A[k].reshape(kl, d * kr), full_matrices=False)
                chi = truncation_rank(s, eps, kappa_max)
                A[k] = vh[:chi].reshape(chi, d, kr)
                A[k - 1] = np.einsum("apb,bc->apc", A[k - 1], u[:, :chi] * s[:chi][None, :])
        if src < K - 1:
            _move_centre_right(A, src)
    return A


def pt_mpo_from_influence(A):
    """P^(k)[a, i, o, b] = delta_io F_k[a, i, b] (influence-functional PT-MPO, diagonal in i,o)."""
    out = []
    for F in A:
        kl, _, kr = F.shape
        P = np.zeros((kl, 4, 4, kr), dtype=complex)
        for p in range(4):
            P[:, p, p, :] = F[:, p, :]
        out.append(P)
    return out


def cap_gauge(P):
    """Rescale P^(k) so every cap C^(k) (App. A.3) has unit 2-norm; observables are unchanged.

    The raw caps obey C^(k-1) = T_k C^(k) with T_k the traced tensor; dividing P^(k) by
    s_k = |T_k c^(k)| (c the normalised caps) makes the rescaled caps exactly c. The product of
    all s_k equals |C^(0)| (1 for a trace-preserving PT); the leftover scalar C^(0)_raw/|...| and
    the product are put back on P^(1) so the overall normalisation is that of the raw tensors.
    """
    iota_over_d = np.array([1, 0, 0, 1], dtype=complex) / 2.0
    tau = np.array([1, 0, 0, 1], dtype=complex)
    P = [p.copy() for p in P]
    c = np.ones(P[-1].shape[3], dtype=complex)
    total = 1.0 + 0j
    for k in range(len(P) - 1, -1, -1):
        raw = np.einsum("aiob,i,o,b->a", P[k], iota_over_d, tau, c)
        s = np.linalg.norm(raw)
        P[k] = P[k] / s
        c = raw / s
        total *= s
    # state after step k picks up prod_{1<j<=k} 1/s_j, its cap prod_{j>k} 1/s_j: restore on P^(1)
    P[0] = P[0] * total
    return P


def build_pt_mpo(bathspec, dt, K, eps_tempo, kappa_max, n_memory=None):
    """PT-MPO of one bath for K steps: list of P^(k) [kappa_{k-1}][4][4][kappa_k], k = 1..K."""
    if n_memory is None or n_memory <= 0:
        n_memory = K
    eta = _bath.eta_coefficients(bathspec, dt, n_memory)
    A = build_influence_mps(eta, K, n_memory, eps_tempo, kappa_max)
    return cap_gauge(pt_mpo_from_influence(A))


def build_pt_mpo_from_eta(eta, K, eps_tempo, kappa_max, n_memory=None):
    if n_memory is None or n_memory <= 0:
        n_memory = K
    A = build_influence_mps(eta, K, n_memory, eps_tempo, kappa_max)
    return cap_gauge(pt_mpo_from_influence(A))
