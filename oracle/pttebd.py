"""Augmented-MPS PT-TEBD (oracle), App. A.1-A.4.

State (App. A.1, "augmented MPS"): Vidal form with an extra leg per site,
    Gamma_n[chi_{n-1}, p, kappa_n, chi_n]   (p = Liouville index, d^2 = 4),
    lambda_n[chi_n] for the N+1 bonds, lambda_0 = lambda_N = [1],
plus a scalar log-norm: the true state is exp(lognorm) times the network (Liouville-space
2-norms are not conserved, so lambda is kept at unit 2-norm and the factor carried separately).
Sites are 0-based here: site i sits between bonds i and i+1.

Bond update (App. A.2), for sites (i, i+1) and a two-site gate G, in four moves:
  reduce   -- the outer blocks B_L = lambda_i Gamma_i (rows (l, a), columns (p, c)) and
              B_R = Gamma_{i+1} lambda_{i+2} (rows (c, q), columns (b, r)) are reduced exactly by
              QR and LQ, B_L = Q_L R_L, B_R = L_R Q_R (the paper reduces them by truncated SVDs;
              both variants are implemented and agree without truncation);
  contract -- D[(u,p'),(q',v)] = sum G[p'q',pq] R_L[u,p,c] lambda_{i+1,c} L_R[c,q,v];
  split    -- truncated SVD of D with the paper's relative rule; the kept singular values,
              normalised, become lambda_{i+1}, their norm goes into the log-norm;
  recover  -- Gamma_i = lambda_i^{-1} Q_L U and Gamma_{i+1} = V^dagger Q_R lambda_{i+2}^{-1}.
Site contraction (App. A.2): Gamma'[l,p',b,r] = sum_{a,p} Gamma[l,p,a,r] P[a,p,p',b].
Caps (App. A.3): C^(K) = 1, C^(k-1)[a] = sum_{i,o,b} P^(k)[a,i,o,b] (iota_i/d) tau_o C^(k)[b].
Readout: contract each augmented leg with its cap, close Liouville legs with vec(I) (trace) or
vec(O^T) (observable), including the lambdas; observables are raw Tr(O rho) unless normalised.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .truncation import truncation_rank, MULTIPLET_TOL
from .model import left_superop, right_superop

TAU = np.array([1, 0, 0, 1], dtype=complex)          # vec(I)
IOTA_OVER_D = TAU / 2.0                                # vec(I)/d: the identity input of App. A.3


@dataclass
class AugmentedMPS:
    gam: List[np.ndarray]
    lam: List[np.ndarray]
    lognorm: float = 0.0
    trunc_log: list = field(default_factory=list)      # (bond, chi, discarded 2-norm / s_max)

    @property
    def N(self):
        return len(self.gam)

    def copy(self):
        return AugmentedMPS([g.copy() for g in self.gam], [l.copy() for l in self.lam], self.lognorm,
                            list(self.trunc_log))

    def chis(self):
        return [len(l) for l in self.lam]

    def kappas(self):
        return [g.shape[2] for g in self.gam]


def product_state(vectors):
    """Augmented MPS of a product state with dummy augmented legs of dimension 1 (App. A.1)."""
    gam = [np.asarray(v, dtype=complex).reshape(1, 4, 1, 1).copy() for v in vectors]
    lam = [np.ones(1) for _ in range(len(vectors) + 1)]
    return AugmentedMPS(gam, lam, 0.0)


def _reduce_qr(BL, BR):
    """Exact reductions: B_L = Q_L R_L (if taller than wide), B_R = L_R Q_R (if wider than tall)."""
    mL, nL = BL.shape
    if mL > nL:
        QL, RL = np.linalg.qr(BL)
    else:
        QL, RL = np.eye(mL, dtype=complex), BL
    mR, nR = BR.shape
    if nR > mR:
        q, r = np.linalg.qr(BR.conj().T)
        LR, QR = r.conj().T, q.conj().T
    else:
        LR, QR = BR, np.eye(nR, dtype=complex)
    return QL, RL, LR, QR


def _reduce_svd(BL, BR, eps):
    """The paper's reduction: truncated SVDs U_L (S_L V_L^dag) and (U_R S_R) V_R^dag of B_L and B_R."""
    u, s, vh = np.linalg.svd(BL, full_matrices=False)
    c = truncation_rank(s, eps, len(s))
    QL, RL = u[:, :c], s[:c, None] * vh[:c]
    u, s, vh = np.linalg.svd(BR, full_matrices=False)
    c = truncation_rank(s, eps, len(s))
    LR, QR = u[:, :c] * s[None, :c], vh[:c]
    return QL, RL, LR, QR


def bond_update(m: AugmentedMPS, i: int, G: np.ndarray, chi_max: int, eps: float,
                variant: str = "qr", multiplet_tol: float = MULTIPLET_TOL):
    """Apply the two-site Liouville gate G (16x16, grouped (p_i, p_{i+1})) to sites i, i+1."""
    GL, GR = m.gam[i], m.gam[i + 1]
    lamL, lamC, lamR = m.lam[i], m.lam[i + 1], m.lam[i + 2]
    chl, _, kl, chc = GL.shape
    _, _, kr, chr_ = GR.shape
    # reduce: the outer blocks
    BL = (lamL[:, None, None, None] * GL).transpose(0, 2, 1, 3).reshape(chl * kl, 4 * chc)
    BR = (GR * lamR[None, None, None, :]).reshape(chc * 4, kr * chr_)
    if variant == "qr":
        QL, RL, LR, QR = _reduce_qr(BL, BR)
    elif variant == "svd":
        QL, RL, LR, QR = _reduce_svd(BL, BR, eps)
    else:
        raise ValueError(variant)
    rL, rR = RL.shape[0], LR.shape[1]
    # contract: theta and the gate
    theta = np.einsum("upc,c,cqv->upqv", RL.reshape(rL, 4, chc), lamC, LR.reshape(chc, 4, rR))
    theta = np.einsum("PQpq,upqv->uPQv", np.asarray(G).reshape(4, 4, 4, 4), theta)
    Dm = theta.reshape(rL * 4, 4 * rR)
    # split: truncated SVD
    try:
        U, S, Vh = np.linalg.svd(Dm, full_matrices=False)
    except np.linalg.LinAlgError:                       # zgesdd failure: fall back to zgesvd
        import scipy.linalg as sla
        U, S, Vh = sla.svd(Dm, full_matrices=False, lapack_driver="gesvd")
    chi = truncation_rank(S, eps, chi_max, multiplet_tol)
    disc = float(np.sqrt(np.sum(S[chi:] ** 2)) / S[0]) if S[0] > 0 else 0.0
    U, S, Vh = U[:, :chi], S[:chi], Vh[:chi]
    nrm = float(np.linalg.norm(S))
    m.lam[i + 1] = S / nrm
    m.lognorm += np.log(nrm)
    m.trunc_log.append((i, chi, disc))
    # recover the site tensors
    newL = (QL @ U.reshape(rL, 4 * chi)).reshape(chl, kl, 4, chi).transpose(0, 2, 1, 3)
    m.gam[i] = newL / lamL[:, None, None, None]
    newR = (Vh.reshape(chi * 4, rR) @ QR).reshape(chi, 4, kr, chr_)
    m.gam[i + 1] = newR / lamR[None, None, None, :]
    return S


def site_contract(m: AugmentedMPS, i: int, P: np.ndarray):
    """PT site contraction (App. A.2): Gamma'[l,p',b,r] = sum_{a,p} Gamma[l,p,a,r] P[a,p,p',b]."""
    m.gam[i] = np.einsum("lpar,apqb->lqbr", m.gam[i], P)


def fuse_local(P, local_prop):
    """P~[a,p,p',b] = sum_q LP[p',q] P[a,p,q,b]: the on-site propagator applied after P."""
    if local_prop is None:
        return P
    return np.einsum("Qq,apqb->apQb", np.asarray(local_prop), P)


def caps(P_list, final_cap=None):
    """Cap tensors C^(0..K) of one PT-MPO (App. A.3), with C^(K) = 1 (all-ones if kappa_K > 1)."""
    K = len(P_list)
    C = [None] * (K + 1)
    C[K] = np.ones(P_list[-1].shape[3], dtype=complex) if final_cap is None else final_cap
    for k in range(K, 0, -1):
        C[k - 1] = np.einsum("aiob,i,o,b->a", P_list[k - 1], IOTA_OVER_D, TAU, C[k])
    return C


def apply_local(m: AugmentedMPS, i: int, A, side: str = "left"):
    """Insert the super-operator A . (left) or . A (right) on site i's Liouville leg (App. A.4)."""
    S = left_superop(A) if side == "left" else right_superop(A)
    m.gam[i] = np.einsum("qp,lpar->lqar", S, m.gam[i])


def observe(m: AugmentedMPS, site_caps, op_vectors, normalize=False):
    """<O>_n for every site n and every operator vector o = vec(O^T); returns [N, n_ops] and trace.

    site_caps[n] is the cap vector for site n's augmented leg at the current step.
    """
    N = m.N
    M = [np.einsum("lpar,a->lpr", m.gam[n], site_caps[n]) for n in range(N)]
    V = [np.einsum("lpr,p->lr", M[n], TAU) for n in range(N)]
    Lp = [None] * (N + 1)
    Lp[0] = m.lam[0].astype(complex)
    for n in range(N):
        Lp[n + 1] = (Lp[n] @ V[n]) * m.lam[n + 1]
    Rs = [None] * (N + 1)
    Rs[N] = np.ones(1, dtype=complex)
    for n in range(N - 1, -1, -1):
        Rs[n] = V[n] @ (m.lam[n + 1] * Rs[n + 1])
    scale = np.exp(m.lognorm)
    trace = complex(Lp[N][0] * scale)
    out = np.zeros((N, len(op_vectors)), dtype=complex)
    for n in range(N):
        right = m.lam[n + 1] * Rs[n + 1]
        for j, o in enumerate(op_vectors):
            On = np.einsum("lpr,p->lr", M[n], o)
            out[n, j] = (Lp[n] @ On @ right) * scale
    if normalize:
        out = out / trace
    return out, trace


def chain_half(m: AugmentedMPS, gates_q, gates_h, chi_max, eps, variant="qr",
               multiplet_tol=MULTIPLET_TOL):
    """e^{L_chain dt/2} by second-order splitting among sites: O(dt/4) E(dt/2) O(dt/4).

    Odd bonds (1,2),(3,4),.. (1-based; 0-based bonds 0,2,..) get exp(L dt/4), even bonds exp(L dt/2).
    """
    nb = m.N - 1
    odd = list(range(0, nb, 2))
    even = list(range(1, nb, 2))
    for b in odd:
        bond_update(m, b, gates_q[b], chi_max, eps, variant, multiplet_tol)
    for b in even:
        bond_update(m, b, gates_h[b], chi_max, eps, variant, multiplet_tol)
    for b in odd:
        bond_update(m, b, gates_q[b], chi_max, eps, variant, multiplet_tol)


def pt_step(m: AugmentedMPS, k: int, gates_q, gates_h, site_P, chi_max, eps, variant="qr",
            multiplet_tol=MULTIPLET_TOL):
    """One full step k (1-based), Eq. (propagator-env): chain half, PT site layer, chain half.

    site_P[n] is None (no bath, no on-site propagator) or the list P^(1..K) of site n.
    """
    chain_half(m, gates_q, gates_h, chi_max, eps, variant, multiplet_tol)
    for n in range(m.N):
        if site_P[n] is not None:
            site_contract(m, n, site_P[n][k - 1])
    chain_half(m, gates_q, gates_h, chi_max, eps, variant, multiplet_tol)
