"""Oracle-side assembly of a workload: gates, PT-MPOs, initial states, and a full FP64 run.

Gates follow App. A.1: K'_{n,n+1} absorbs the on-site terms, G_b(tau) = exp(L^{K'}_b tau) with
tau = dt/4 (odd bonds) and dt/2 (even bonds). Each gate is computed twice -- matrix exponential of
the Liouvillian and the closed form U (x) conj(U) -- and the two must agree to 1e-12.
PT-MPOs come from ``oracle.tempo`` (one per distinct bath, shared by identical sites as in
App. A.1) and are cached on disk as .npz, keyed by every parameter that defines them.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import asdict, dataclass, field
from typing import List, Optional

import numpy as np

import scipy.linalg as sla

from . import gksl, model, tempo, pttebd
from .truncation import MULTIPLET_TOL

CACHE_DIR = os.environ.get("PT_TEBD_CACHE",
                           os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                        "_cache"))


@dataclass
class ChainInputs:
    N: int
    rho0: List[np.ndarray]                 # per site vec(rho_n) (4,)
    gates_q: List[np.ndarray]              # per bond 16x16
    gates_h: List[np.ndarray]
    pt: List[Optional[List[np.ndarray]]]   # per site: None or P^(1..K)
    init_mps: Optional[pttebd.AugmentedMPS] = None


def chain_gates(ch, dt, check=True):
    if ch.gksl or ch.drive is not None:
        # time-local dissipation (App. A.1, Sec. III.A.3): gates of the non-Hermitian bond
        # generators, by scipy's matrix exponential
        Ls = gksl.bond_liouvillians(ch)
        return ([sla.expm(L * (dt / 4)) for L in Ls], [sla.expm(L * (dt / 2)) for L in Ls])
    Kp = model.absorbed_bond_hamiltonians(ch.eps, ch.J)
    gq, gh = [], []
    for Kb in Kp:
        a = model.gate_expm(Kb, dt / 4)
        b = model.gate_expm(Kb, dt / 2)
        if check:
            assert np.max(np.abs(a - model.gate_unitary(Kb, dt / 4))) < 1e-12
            assert np.max(np.abs(b - model.gate_unitary(Kb, dt / 2))) < 1e-12
        gq.append(a)
        gh.append(b)
    return gq, gh


def _ptmpo_key(bath, dt, K, eps_tempo, kappa_max, n_memory):
    d = dict(bath=asdict(bath), dt=dt, K=K, eps_tempo=eps_tempo, kappa_max=kappa_max,
             n_memory=n_memory, v=2)
    return hashlib.sha256(json.dumps(d, sort_keys=True).encode()).hexdigest()[:20]


def pt_mpo_cached(bath, dt, K, eps_tempo, kappa_max, n_memory=0):
    key = _ptmpo_key(bath, dt, K, eps_tempo, kappa_max, n_memory)
    path = os.path.join(CACHE_DIR, f"oracle_ptmpo_{key}.npz")
    if os.path.exists(path):
        z = np.load(path)
        return [z[f"P{k}"] for k in range(K)]
    P = tempo.build_pt_mpo(bath, dt, K, eps_tempo, kappa_max, n_memory)
    try:
        os.makedirs(CACHE_DIR, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez_compressed(tmp, **{f"P{k}": P[k] for k in range(K)})
        os.replace(tmp, path)
    except OSError:
        pass
    return P


def build_inputs(w) -> List[ChainInputs]:
    """Oracle inputs for every chain of workload w."""
    if w.random_state is not None:
        return [_random_inputs(w)]
    out = []
    for ch in w.chains:
        gq, gh = chain_gates(ch, w.dt)
        pts = []
        for b in ch.baths:
            if b is None:
                pts.append(None)
            else:
                pts.append(pt_mpo_cached(b, w.dt, w.K, w.eps_tempo, w.kappa_max, w.memory_steps))
        rho0 = [model.product_state_vector(c) for c in ch.init]
        out.append(ChainInputs(ch.N, rho0, gq, gh, pts))
    return out


def _random_inputs(w):
    from workloads.configs import random_state_draws
    rs = random_state_draws(**w.random_state)
    N = w.random_state["N"]
    gam = [g.copy() for g in rs["gamma"]]
    lam = [l / np.linalg.norm(l) for l in rs["lam"]]
    m = pttebd.AugmentedMPS(gam, lam, 0.0)
    pts = []
    for P in rs["pt"]:
        k = P.shape[0]
        s = np.linalg.norm(P.reshape(4 * k, 4 * k), 2)   # rows (a,p), cols (p',b)
        pts.append(P / s)
    gq = [model.gate_from_unitary(u) for u in rs["u_q"]]
    gh = [model.gate_from_unitary(u) for u in rs["u_h"]]
    return ChainInputs(N, [None] * N, gq, gh, [pts] * N, init_mps=m)


@dataclass
class RunResult:
    obs: np.ndarray            # [K+1, N, n_ops] raw (or trace-normalised) observables
    trace: np.ndarray          # [K+1]
    chis: list                 # per step: list of bond dims
    kappas: list
    lognorm: np.ndarray
    final_mps: Optional[pttebd.AugmentedMPS] = None
    lambdas: list = field(default_factory=list)


def simulate_chain(ci: ChainInputs, w, ops, K=None, variant="qr", normalize=False,
                   insert=None, multiplet_tol=None, keep_lambdas=False, insert_at=0):
    """Run the PT-TEBD schedule for one chain; observe every op on every site after each step.

    insert = (site, 2x2 operator, 'left'|'right') applies that super-operator to the full augmented
    MPS after step insert_at (0: the initial state), before that step's readout (App. A.4; the
    branching at a later time follows the two-time correlation procedure of App. B.2).
    multiplet_tol: the truncation's multiplet tolerance (None: the workload's).
    """
    K = w.K if K is None else K
    if multiplet_tol is None:
        multiplet_tol = getattr(w, "multiplet_tol", MULTIPLET_TOL)
    m = ci.init_mps.copy() if ci.init_mps is not None else pttebd.product_state(ci.rho0)
    site_caps = []
    for n in range(ci.N):
        if ci.pt[n] is None:
            site_caps.append(None)
        else:
            site_caps.append(pttebd.caps(ci.pt[n]))
    if insert is not None and insert_at == 0:
        pttebd.apply_local(m, insert[0], insert[1], insert[2])
    opv = [model.op_vector(o) for o in ops]

    def caps_at(k):
        return [np.ones(1, dtype=complex) if c is None else c[k] for c in site_caps]

    obs, tr, chis, kaps, lns, lams = [], [], [], [], [], []
    o, t = pttebd.observe(m, caps_at(0), opv, normalize)
    obs.append(o); tr.append(t); chis.append(m.chis()); kaps.append(m.kappas()); lns.append(m.lognorm)
    for k in range(1, K + 1):
        pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps, variant, multiplet_tol)
        if insert is not None and insert_at == k:
            pttebd.apply_local(m, insert[0], insert[1], insert[2])
        o, t = pttebd.observe(m, caps_at(k), opv, normalize)
        obs.append(o); tr.append(t); chis.append(m.chis()); kaps.append(m.kappas()); lns.append(m.lognorm)
        if keep_lambdas:
            lams.append([l.copy() for l in m.lam])
    return RunResult(np.array(obs), np.array(tr), chis, kaps, np.array(lns), m, lams)
