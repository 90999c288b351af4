"""Host-side construction of PT-TEBD inputs: two-site Liouville gates and bath PT-MPOs.

These are the inputs of pt_tebd_init (they are not part of the time step). They are built here
with NumPy, independently of the test oracle, from the physics of a workload:

* gates (App. A.1): K'_{n,n+1} absorbs the on-site terms (whole end-site terms on the end bonds,
  halves elsewhere); G(tau) = U (x) conj(U), U = exp(-i K' tau) from an eigendecomposition, in the
  per-site grouped Liouville index (p_n, p_{n+1}), p = i*2 + j (row-major vectorisation). With
  time-local GKSL terms (or the two-spin driving of Sec. III.A.3) the bond generator is assembled
  by applying it to each basis operator and G(tau) is its matrix exponential.
* PT-MPOs for Gaussian baths coupled to s^z (App. B.1): the discretised influence functional with
  memory coefficients eta_D built from G(t) = int_0^t int_0^s C(u) du ds, compressed slot by slot
  into an MPO (relative SVD threshold eps_tempo, bond cap kappa_max), diagonal in (input, output),
  and rescaled so that every cap tensor has unit norm.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import asdict

import numpy as np
from scipy.special import loggamma

_SIG = {
    "x": np.array([[0, 1], [1, 0]], dtype=complex),
    "y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "z": np.array([[1, 0], [0, -1]], dtype=complex),
}
_S = {k: v / 2 for k, v in _SIG.items()}
_I2 = np.eye(2, dtype=complex)

CACHE_DIR = os.environ.get("PT_TEBD_CACHE",
                           os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_cache"))


def pauli(name):
    return _SIG[name].copy()


def state_vec(ch):
    """vec(|s><s|) of 'u' or 'd' (row-major)."""
    v = np.zeros(4, dtype=complex)
    v[0 if ch == "u" else 3] = 1.0
    return v


# ------------------------------------------------------------------------------------ gates
def _bond_hamiltonians(eps, J):
    N = len(eps)
    Hs = [e * _S["z"] for e in eps]
    out = []
    for b in range(N - 1):
        K = sum(J[b][g] * np.kron(_S[n], _S[n]) for g, n in enumerate("xyz"))
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b == N - 2 else 0.5
        out.append(K + wl * np.kron(Hs[b], _I2) + wr * np.kron(_I2, Hs[b + 1]))
    return out


def liouville_gate(U):
    """Grouped 16x16 Liouville matrix of rho -> U rho U^dag for a two-site unitary U (4x4)."""
    M = np.kron(U, U.conj())                     # rows (i1 i2 j1 j2), cols likewise
    idx = np.arange(16)
    i1, i2, j1, j2 = (idx >> 3) & 1, (idx >> 2) & 1, (idx >> 1) & 1, idx & 1
    grouped = (i1 * 2 + j1) * 4 + (i2 * 2 + j2)  # position of each row-major index in grouped order
    G = np.zeros((16, 16), dtype=complex)
    G[np.ix_(grouped, grouped)] = M
    return G


_JUMP = {"minus": np.array([[0, 0], [1, 0]], dtype=complex), "plus": np.array([[0, 1], [0, 0]], dtype=complex),
         "z": _SIG["z"]}


def _grouped_superop(action):
    """16x16 matrix, in the grouped two-site index (i1 j1, i2 j2), of a linear map on 4x4 two-site
    operators X[(i1 i2), (j1 j2)], found by applying it to each basis operator."""
    M = np.zeros((16, 16), dtype=complex)
    for i1 in range(2):
        for j1 in range(2):
            for i2 in range(2):
                for j2 in range(2):
                    E = np.zeros((4, 4), dtype=complex)
                    E[i1 * 2 + i2, j1 * 2 + j2] = 1.0
                    Y = action(E)
                    col = (i1 * 2 + j1) * 4 + (i2 * 2 + j2)
                    for a1 in range(2):
                        for b1 in range(2):
                            for a2 in range(2):
                                for b2 in range(2):
                                    M[(a1 * 2 + b1) * 4 + (a2 * 2 + b2), col] = Y[a1 * 2 + a2, b1 * 2 + b2]
    return M


def _lindblad_term(L):
    """X -> L X L^dag - (L^dag L X + X L^dag L) / 2 for a two-site operator L (4x4)."""
    LdL = L.conj().T @ L
    return lambda X: L @ X @ L.conj().T - 0.5 * (LdL @ X + X @ LdL)


def _bond_generators(ch):
    """Bond generators of App. A.1 with time-local dissipation: -i[K', .] plus the sites' GKSL
    terms (whole on the chain's end sites, half elsewhere), plus the two-spin driving generator of
    Sec. III.A.3 on the first bond (jumps between eigenstates of the pair's own Hamiltonian with
    rates 1 / (1 + e^{(E_a - E_b)/T}), whose steady state is the pair's Gibbs state)."""
    N = ch.N
    Kps = _bond_hamiltonians(ch.eps, ch.J)
    jumps = [[] for _ in range(N)]
    for site, op, rate in ch.gksl:
        jumps[site].append(np.sqrt(rate) * _JUMP[op])
    gens = []
    for b in range(N - 1):
        wl = 1.0 if b == 0 else 0.5
        wr = 1.0 if b == N - 2 else 0.5
        terms = [(1.0, -1j, Kps[b])]
        ops = [(wl, np.kron(L, _I2)) for L in jumps[b]] + [(wr, np.kron(_I2, L)) for L in jumps[b + 1]]
        if b == 0 and ch.drive is not None:
            HB = ch.eps[0] * np.kron(_S["z"], _I2) + ch.eps[1] * np.kron(_I2, _S["z"]) + \
                sum(ch.J[0][g] * np.kron(_S[n], _S[n]) for g, n in enumerate("xyz"))
            E, V = np.linalg.eigh(HB)
            for a in range(4):
                for c in range(4):
                    if a != c:
                        r = ch.drive.rate / (1.0 + np.exp((E[a] - E[c]) / ch.drive.T))
                        ops.append((1.0, np.sqrt(r) * np.outer(V[:, a], V[:, c].conj())))
        Kp = Kps[b]

        def action(X, Kp=Kp, ops=ops):
            Y = -1j * (Kp @ X - X @ Kp)
            for wgt, L in ops:
                Y = Y + wgt * _lindblad_term(L)(X)
            return Y
        gens.append(_grouped_superop(action))
    return gens


def chain_gates(ch, dt):
    if ch.gksl or ch.drive is not None:
        from scipy.linalg import expm
        gens = _bond_generators(ch)
        return (np.array([expm(Lg * (dt / 4)) for Lg in gens]), np.array([expm(Lg * (dt / 2)) for Lg in gens]))
    gq, gh = [], []
    for Kp in _bond_hamiltonians(ch.eps, ch.J):
        w, V = np.linalg.eigh(Kp)
        for tau, dst in ((dt / 4, gq), (dt / 2, gh)):
            U = (V * np.exp(-1j * w * tau)) @ V.conj().T
            dst.append(liouville_gate(U))
    return np.array(gq), np.array(gh)


# ------------------------------------------------------------------------------------ baths
def bath_G(bath, t):
    """G(t) for J(w) = 2 alpha w exp(-w/wc) (closed form: coth expanded as a geometric series)."""
    if bath.cutoff != "exponential":
        raise NotImplementedError("only the exponential cutoff has a closed-form G(t) here")
    t = np.asarray(t, dtype=float)
    g = 2 * bath.alpha * (np.log1p(1j * bath.omega_c * t) - 1j * bath.omega_c * t)
    if bath.T > 0:
        x = 1.0 + bath.T / bath.omega_c
        g = g + 4 * bath.alpha * (loggamma(x).real - loggamma(x + 1j * bath.T * t).real)
    return g


def eta_list(bath, dt, n):
    G = bath_G(bath, dt * np.arange(n + 2))
    eta = np.empty(n + 1, dtype=complex)
    eta[0] = G[1]
    eta[1:] = G[2:n + 2] - 2 * G[1:n + 1] + G[0:n]
    return eta


def _keep(s, eps, cap, mtol=1e-12):
    """Relative truncation: smallest chi with ||dropped|| < eps * s0, capped, multiplets whole."""
    n = len(s)
    if n == 0 or s[0] <= 0:
        return 1
    tail = np.sqrt(np.cumsum((s * s)[::-1])[::-1])
    ok = np.nonzero(np.append(tail, 0.0)[1:] < eps * s[0])[0]
    chi = int(ok[0]) + 1 if len(ok) else n
    chi = max(1, min(chi, int(np.count_nonzero(s > 0))))

    def split(c):
        return 0 < c < n and s[c - 1] - s[c] <= mtol * s[0]

    if chi <= cap:
        while split(chi) and chi < cap and s[chi] > 0:
            chi += 1
        if not split(chi):
            return chi
    chi = min(chi, cap)
    while chi > 1 and split(chi):
        chi -= 1
    return chi


def influence_mpo(eta, K, eps, cap, memory=None):
    """Compressed influence functional over K slots: list of F_k[a, p, b] (p = Liouville index)."""
    memory = K if not memory else memory
    sgn = np.array([0.5, -0.5])
    sp, sm = sgn[np.arange(4) // 2], sgn[np.arange(4) % 2]
    d = sp - sm
    first = np.exp(-d * (eta[0] * sp - np.conj(eta[0]) * sm))
    lines = [None] + [np.exp(-np.outer(d, eta[D] * sp - np.conj(eta[D]) * sm)) for D in range(1, len(eta))]
    # start: product MPS, orthogonality centre at slot 0 (all other slots unit vectors)
    F = [(first / np.linalg.norm(first)).reshape(1, 4, 1) for _ in range(K)]
    F[0] = F[0] * np.linalg.norm(first) ** K
    for src in range(K):
        last = min(K - 1, src + memory)
        if last > src:
            a, _, b = F[src].shape
            T = np.zeros((a, 4, b, 4), dtype=complex)
            for p in range(4):
                T[:, p, :, p] = F[src][:, p, :]
            F[src] = T.reshape(a, 4, b * 4)
            for k in range(src + 1, last + 1):
                L = lines[k - src]
                a, _, b = F[k].shape
                if k < last:
                    T = F[k][:, None, :, :, None] * L.T[None, :, :, None, None] * np.eye(4)[None, :, None, None, :]
                    F[k] = T.reshape(a * 4, 4, b * 4)
                else:
                    F[k] = (F[k][:, None, :, :] * L.T[None, :, :, None]).reshape(a * 4, 4, b)
            # left-orthonormalise src..last-1, then compress last..src+1 from the right
            for k in range(src, last):
                a, p, b = F[k].shape
                q, r = np.linalg.qr(F[k].reshape(a * p, b))
                F[k] = q.reshape(a, p, -1)
                F[k + 1] = np.tensordot(r, F[k + 1], axes=(1, 0))
            for k in range(last, src, -1):
                a, p, b = F[k].shape
                u, s, vh = np.linalg.svd(F[k].reshape(a, p * b), full_matrices=False)
                c = _keep(s, eps, cap)
                F[k] = vh[:c].reshape(c, p, b)
                F[k - 1] = np.tensordot(F[k - 1], u[:, :c] * s[:c], axes=(2, 0))
        if src + 1 < K:
            a, p, b = F[src].shape
            q, r = np.linalg.qr(F[src].reshape(a * p, b))
            F[src] = q.reshape(a, p, -1)
            F[src + 1] = np.tensordot(r, F[src + 1], axes=(1, 0))
    return F


def pt_mpo_tensors(F):
    """P^(k)[a, i, o, b] = delta_io F_k[a, i, b], rescaled to unit-norm caps (observables unchanged)."""
    P = []
    for Fk in F:
        a, _, b = Fk.shape
        T = np.zeros((a, 4, 4, b), dtype=complex)
        for p in range(4):
            T[:, p, p, :] = Fk[:, p, :]
        P.append(T)
    cap = np.ones(P[-1].shape[3], dtype=complex)
    prod = 1.0
    for k in range(len(P) - 1, -1, -1):
        raw = 0.5 * (P[k][:, 0, 0, :] + P[k][:, 3, 3, :]) @ cap
        s = np.linalg.norm(raw)
        P[k] = P[k] / s
        cap = raw / s
        prod *= s
    P[0] = P[0] * prod
    return P


def bath_pt_mpo(bath, dt, K, eps_tempo, kappa_max, memory=0, cache=True):
    key = hashlib.sha256(json.dumps(dict(b=asdict(bath), dt=dt, K=K, e=eps_tempo, c=kappa_max, m=memory,
                                         v=1), sort_keys=True).encode()).hexdigest()[:20]
    path = os.path.join(CACHE_DIR, f"product_ptmpo_{key}.npz")
    if cache and os.path.exists(path):
        z = np.load(path)
        return [z[f"P{k}"] for k in range(K)]
    F = influence_mpo(eta_list(bath, dt, memory or K), K, eps_tempo, kappa_max, memory or K)
    P = pt_mpo_tensors(F)
    if cache:
        try:
            os.makedirs(CACHE_DIR, exist_ok=True)
            tmp = path + f".tmp{os.getpid()}.npz"
            np.savez_compressed(tmp, **{f"P{k}": P[k] for k in range(K)})
            os.replace(tmp, path)
        except OSError:
            pass
    return P


# ------------------------------------------------------------------------------------ workloads
def build_problem(w):
    """(chains, pt_mpos) for pt_tebd_init from a workloads.Workload (PT-MPOs deduplicated per bath)."""
    if w.random_state is not None:
        return _random_problem(w)
    mpos, index = [], {}
    chains = []
    for ch in w.chains:
        gq, gh = chain_gates(ch, w.dt) if ch.N > 1 else (None, None)
        ids = []
        for b in ch.baths:
            if b is None:
                ids.append(-1)
                continue
            if b not in index:
                index[b] = len(mpos)
                mpos.append(bath_pt_mpo(b, w.dt, w.K, w.eps_tempo, w.kappa_max, w.memory_steps))
            ids.append(index[b])
        chains.append(dict(N=ch.N, rho0=np.array([state_vec(c) for c in ch.init]), gates_q=gq,
                           gates_h=gh, ptmpo_id=ids))
    return chains, mpos


def _random_problem(w):
    from workloads.configs import random_state_draws
    rs = random_state_draws(**w.random_state)
    N = w.random_state["N"]
    lam = [l / np.linalg.norm(l) for l in rs["lam"]]
    pts = []
    for P in rs["pt"]:
        k = P.shape[0]
        pts.append(P / np.linalg.norm(P.reshape(4 * k, 4 * k), 2))
    gq = np.array([liouville_gate(u) for u in rs["u_q"]])
    gh = np.array([liouville_gate(u) for u in rs["u_h"]])
    chi0 = [g.shape[0] for g in rs["gamma"]] + [1]
    kap0 = [g.shape[2] for g in rs["gamma"]]
    chain = dict(N=N, rho0=None, gates_q=gq, gates_h=gh, ptmpo_id=[0] * N, chi0=chi0, kappa0=kap0,
                 gamma0=rs["gamma"], lambda0=lam)
    return [chain], [pts]
