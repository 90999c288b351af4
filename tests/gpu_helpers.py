"""Shared helpers of the GPU parity tests: feed oracle-built inputs through the C ABI."""
import numpy as np

from oracle import model, problem as oprob


def engine_args_from_oracle(cis):
    """(chains, pt_mpos) in the C-ABI form from oracle ChainInputs (PT-MPOs shared by identity)."""
    mpos, index = [], {}
    chains = []
    for ci in cis:
        ids = []
        for P in ci.pt:
            if P is None:
                ids.append(-1)
                continue
            if id(P) not in index:
                index[id(P)] = len(mpos)
                mpos.append(P)
            ids.append(index[id(P)])
        d = dict(N=ci.N, gates_q=np.array(ci.gates_q) if ci.N > 1 else None,
                 gates_h=np.array(ci.gates_h) if ci.N > 1 else None, ptmpo_id=ids)
        if ci.init_mps is not None:
            m = ci.init_mps
            d.update(rho0=None, chi0=m.chis(), kappa0=m.kappas(), gamma0=m.gam, lambda0=m.lam)
        else:
            d["rho0"] = np.array(ci.rho0)
        chains.append(d)
    return chains, mpos


def run_gpu(w, cis, ops, K=None, precision="fp64", insert=None, use_graph=True, multiplet_tol=None, route=None):
    import paper_2201_05529_gb300._capi as capi
    K = w.K if K is None else K
    multiplet_tol = w.multiplet_tol if multiplet_tol is None else multiplet_tol
    chains, mpos = engine_args_from_oracle(cis)
    eng = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=precision,
                      multiplet_tol=multiplet_tol, max_steps=K, use_graph=use_graph, route=route)
    if insert is not None:
        c, n, A, side = insert
        eng.apply_local(c, n, A, side)
    eng.set_observables(ops)
    eng.step(K)
    obs, tr = eng.read_history(0, K + 1)
    return eng, obs, tr


def run_oracle(w, cis, ops, K=None, insert=None, multiplet_tol=None):
    multiplet_tol = w.multiplet_tol if multiplet_tol is None else multiplet_tol
    res = []
    for c, ci in enumerate(cis):
        ins = None
        if insert is not None and insert[0] == c:
            ins = (insert[1], insert[2], insert[3])
        res.append(oprob.simulate_chain(ci, w, ops, K=K, insert=ins, multiplet_tol=multiplet_tol,
                                        keep_lambdas=True))
    return res


OPS = [model.SZ, model.SX, model.SY]


def oracle_envelope(w, ci, ops, K=None, scale=1e-13, seed=1, insert=None):
    """Rounding sensitivity of the oracle's own trajectory: |run(inputs) - run(inputs perturbed by
    `scale` relative noise on the dt/4 gates)| per step, as a running maximum over steps.

    Once the chi cap binds, the kept singular values reach ~1e-9 of the largest and the lambda^-1
    of the Gamma recovery (App. A.2) amplifies rounding differences step by step, up to the
    accumulated truncation error; two correct FP64 implementations can then differ by this much.
    """
    rng = np.random.default_rng(seed)
    gq = [g * (1 + scale * rng.standard_normal(g.shape)) for g in ci.gates_q]
    ins = None if insert is None else (insert[1], insert[2], insert[3])
    a = oprob.simulate_chain(ci, w, ops, K=K, insert=ins)
    b = oprob.simulate_chain(oprob.ChainInputs(ci.N, ci.rho0, gq, ci.gates_h, ci.pt, ci.init_mps),
                             w, ops, K=K, insert=ins)
    d = np.abs(a.obs - b.obs).max(axis=(1, 2))
    return np.maximum.accumulate(d)
