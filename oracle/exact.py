"""Exact references that pin the oracle (test infrastructure).

* ``full_liouvillian_run``: rho(t) = expm(L_chain t) rho(0) with the whole 4^N x 4^N Liouvillian of
  the chain without baths (alpha = 0; GKSL terms included when the chain has them). PT-TEBD reduces to Liouville-space TEBD there (Sec. II.A), so it
  must match this up to its O(dt^2) Trotter error.
* ``full_trotter_run``: the same gate sequence as PT-TEBD, each gate embedded as a full 4^N
  matrix: PT-TEBD without truncation must equal it to rounding.
* ``path_sum_run``: N = 2 with a bath on site 0; sum over every Liouville path (p_1 .. p_K) of site
  0 of the influence functional times the projected chain propagation -- the uncompressed network
  of Fig. (tensor-network-construction)(a/c), evaluated by brute force (4^K paths).
* ``single_mode_run``: the same N = 2 chain with a bath of ONE harmonic mode, simulated exactly in
  the chain (x) truncated-Fock Hilbert space with the same splitting e^{L_c dt/2} e^{L_E dt}
  e^{L_c dt/2}. For piecewise-constant system paths the Gaussian influence functional is exact,
  so this pins the influence functional (both signs, real and imaginary parts of eta).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla

from . import model, tempo


def _embed_two_site(G, b, N):
    """Embed a grouped 16x16 gate on sites (b, b+1) into the grouped 4^N Liouville space."""
    return np.kron(np.kron(np.eye(4 ** b), G), np.eye(4 ** (N - b - 2)))


def _product_vector(vectors):
    v = np.ones(1, dtype=complex)
    for x in vectors:
        v = np.kron(v, x)
    return v


def _site_observables(v, N, ops):
    """Tr(O_n rho) for a grouped 4^N Liouville vector, every site n, every op."""
    tau = model.trace_vector()
    out = np.zeros((N, len(ops)), dtype=complex)
    for n in range(N):
        for j, O in enumerate(ops):
            vecs = [tau] * N
            vecs[n] = model.op_vector(O)
            out[n, j] = _product_vector(vecs) @ v
    return out


def full_liouvillian_run(ch, dt, K, ops):
    """<O_n>(k dt), k = 0..K, from expm of the whole closed-chain Liouvillian."""
    from . import gksl
    N = ch.N
    L = gksl.full_liouvillian(ch)           # Hamiltonian part, plus GKSL terms if the chain has any
    v0 = _product_vector([model.product_state_vector(c) for c in ch.init])
    step = sla.expm(L * dt)
    v = v0.copy()
    out = [_site_observables(v, N, ops)]
    for _ in range(K):
        v = step @ v
        out.append(_site_observables(v, N, ops))
    return np.array(out)


def full_trotter_run(N, rho0, gates_q, gates_h, K, ops, insert=None, insert_at=0):
    """Same schedule as PT-TEBD (chain half O(dt/4) E(dt/2) O(dt/4), twice per step), no baths.

    insert = (site, A, side) applies A. or .A on that site after step insert_at."""
    nb = N - 1
    Gq = [_embed_two_site(gates_q[b], b, N) for b in range(nb)]
    Gh = [_embed_two_site(gates_h[b], b, N) for b in range(nb)]
    half = np.eye(4 ** N, dtype=complex)
    for b in range(0, nb, 2):
        half = Gq[b] @ half
    for b in range(1, nb, 2):
        half = Gh[b] @ half
    for b in range(0, nb, 2):
        half = Gq[b] @ half
    v = _product_vector(rho0)
    ins = None
    if insert is not None:
        n, A, side = insert
        S = model.left_superop(A) if side == "left" else model.right_superop(A)
        ins = np.kron(np.kron(np.eye(4 ** n), S), np.eye(4 ** (N - n - 1)))
    if ins is not None and insert_at == 0:
        v = ins @ v
    out = [_site_observables(v, N, ops)]
    for k in range(1, K + 1):
        v = half @ (half @ v)
        if ins is not None and insert_at == k:
            v = ins @ v
        out.append(_site_observables(v, N, ops))
    return np.array(out)


def _two_site_half(gates_q):
    # N = 2: one odd bond, no even bonds: O(dt/4) O(dt/4)
    return gates_q[0] @ gates_q[0]


def path_sum_run(rho0, gates_q, eta, K, ops, n_memory=None):
    """Brute-force influence-functional path sum, N = 2, bath on site 0 (see module docstring)."""
    if n_memory is None:
        n_memory = K
    half = _two_site_half(gates_q)
    v0 = _product_vector(rho0)
    proj = []
    for p in range(4):
        P = np.zeros((16, 16))
        for q in range(4):
            P[p * 4 + q, p * 4 + q] = 1.0
        proj.append(P)
    out = [_site_observables(v0, 2, ops)]
    for k in range(1, K + 1):
        acc = np.zeros(16, dtype=complex)
        for path in itertools.product(range(4), repeat=k):
            f = tempo.influence_functional_value(path, eta, n_memory)
            if f == 0:
                continue
            v = v0
            for p in path:
                v = half @ (proj[p] @ (half @ v))
            acc += f * v
        out.append(_site_observables(acc, 2, ops))
    return np.array(out)


def single_mode_run(ch, g, w0, T, dt, K, ops, nmax=40):
    """Exact Trotterised dynamics of an N = 2 chain whose site 0 couples via s^z to one mode.

    H_E = s^z_0 (g b^dag + conj(g) b) + w0 b^dag b; the mode starts thermal at temperature T.
    Each step: U_c (dt/2), U_E (dt), U_c (dt/2) on the chain (x) mode density matrix, with U_c the
    product of the chain-half gates (for N = 2: exp(-i K' dt/2)).
    """
    assert ch.N == 2
    Kp = model.absorbed_bond_hamiltonians(ch.eps, ch.J)[0]
    Uc = sla.expm(-1j * Kp * dt / 2)
    b = np.diag(np.sqrt(np.arange(1, nmax)), 1).astype(complex)
    nop = b.conj().T @ b
    sz0 = np.kron(model.SPIN_HALF["z"], model.ID2)
    HE = np.kron(sz0, g * b.conj().T + np.conj(g) * b) + np.kron(np.eye(4), w0 * nop)
    UE = sla.expm(-1j * HE * dt)
    Uc_full = np.kron(Uc, np.eye(nmax))
    if T > 0:
        th = np.diag(np.exp(-w0 * np.arange(nmax) / T))
    else:
        th = np.zeros((nmax, nmax)); th[0, 0] = 1
    th = th / np.trace(th)
    rho_c = np.kron(model.unvec(model.product_state_vector(ch.init[0])),
                    model.unvec(model.product_state_vector(ch.init[1])))
    rho = np.kron(rho_c, th).astype(complex)

    def obs(r):
        rc = np.einsum("imjm->ij", r.reshape(4, nmax, 4, nmax))
        out = np.zeros((2, len(ops)), dtype=complex)
        for j, O in enumerate(ops):
            out[0, j] = np.trace(np.kron(O, model.ID2) @ rc)
            out[1, j] = np.trace(np.kron(model.ID2, O) @ rc)
        return out

    res = [obs(rho)]
    for _ in range(K):
        rho = Uc_full @ rho @ Uc_full.conj().T
        rho = UE @ rho @ UE.conj().T
        rho = Uc_full @ rho @ Uc_full.conj().T
        res.append(obs(rho))
    return np.array(res)
