"""ctypes binding of ``libpttebd.so`` (include/pt_tebd.h): argument marshalling only.

Every computation of the PT-TEBD step runs in the library's CUDA kernels. PyTorch supplies device
memory (its caching allocator is registered as the library's allocator) and the CUDA stream.
There is no CPU fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpttebd.so")

PT_FP64, PT_TF32X3, PT_BF16X3, PT_TF32X1, PT_BF16_OZAKI = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": PT_FP64, "tf32x3": PT_TF32X3, "bf16x3": PT_BF16X3, "tf32x1": PT_TF32X1,
              "bf16_ozaki": PT_BF16_OZAKI}
ERRORS = {-1: "PT_ERR_ARG", -2: "PT_ERR_OOM", -3: "PT_ERR_CAPACITY", -4: "PT_ERR_SVD_NOCONV",
          -5: "PT_ERR_DEVICE_TIMEOUT", -6: "PT_ERR_NAN", -7: "PT_ERR_CUDA", -8: "PT_ERR_STEPS"}

EXPORTS = [
    "pt_tebd_set_allocator", "pt_tebd_init", "pt_tebd_set_observables", "pt_tebd_step",
    "pt_tebd_observe", "pt_tebd_read_history", "pt_tebd_apply_local", "pt_tebd_steps_done",
    "pt_tebd_get_dims", "pt_tebd_get_lambda", "pt_tebd_get_lognorm", "pt_tebd_get_lognorms", "pt_tebd_get_gamma", "pt_tebd_get_svd_sweeps",
    "pt_tebd_clone", "pt_tebd_read_bond_log", "pt_tebd_step_kernels", "pt_tebd_get_routes",
    "pt_tune_cache_lookup", "pt_tune_cache_store",
    "pt_tebd_sync", "pt_tebd_destroy", "pt_tebd_last_error", "pt_tebd_set_timing",
    "pt_tebd_get_timing", "pt_svd_scratch_bytes", "pt_svd_f64", "pt_svd_f64_noalloc",
    "pt_zgemm_scratch_bytes", "pt_zgemm_sliced", "pt_qr_scratch_bytes", "pt_qr_f64", "pt_selftest_grid_barrier",
]


class PTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2201_05529_gb300.build()")
    return C.CDLL(LIB_PATH)


lib = _load()

c_double_p = C.POINTER(C.c_double)
c_int_p = C.POINTER(C.c_int)


class ChainDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("rho0", c_double_p), ("gates_q", c_double_p),
                ("gates_h", c_double_p), ("local_prop", c_double_p), ("ptmpo_id", c_int_p),
                ("chi0", c_int_p), ("kappa0", c_int_p), ("gamma0", C.POINTER(c_double_p)),
                ("lambda0", C.POINTER(c_double_p)), ("lognorm0", c_double_p)]


class MpoDesc(C.Structure):
    _fields_ = [("K", C.c_int), ("kappa", c_int_p), ("P", C.POINTER(c_double_p))]


class Options(C.Structure):
    _fields_ = [("chi_max", C.c_int), ("eps", C.c_double), ("multiplet_tol", C.c_double),
                ("precision", C.c_int), ("max_steps", C.c_int), ("max_sweeps", C.c_int),
                ("use_graph", C.c_int), ("autotune", C.c_int), ("tune_cache", C.c_char_p),
                ("force_route", C.c_int)]


# the tuner's cache of kernel choices per layer shape (in-tree, next to the library)
TUNE_CACHE = os.path.join(HERE, "_tune_cache.tsv")
QR_ROUTES = {"grid": 0, "cluster_smem": 1, "cluster_global": 2}
K2_ROUTES = {"grid": 0, "cta": 1}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

lib.pt_tebd_set_allocator.argtypes = [ALLOC_FN, FREE_FN, C.c_void_p]
lib.pt_tebd_set_allocator.restype = None
lib.pt_tebd_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(ChainDesc), C.c_int,
                             C.POINTER(MpoDesc), C.c_int, C.POINTER(Options), C.c_void_p]
lib.pt_tebd_set_observables.argtypes = [C.c_void_p, c_double_p, C.c_int]
lib.pt_tebd_step.argtypes = [C.c_void_p, C.c_int]
lib.pt_tebd_observe.argtypes = [C.c_void_p, c_double_p, C.c_int, c_double_p, c_double_p, C.c_int]
lib.pt_tebd_read_history.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, c_double_p]
lib.pt_tebd_apply_local.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, C.c_int]
lib.pt_tebd_steps_done.argtypes = [C.c_void_p]
lib.pt_tebd_step_kernels.argtypes = [C.c_void_p]
lib.pt_tebd_get_routes.argtypes = [C.c_void_p, c_int_p, C.POINTER(C.c_float)]
lib.pt_tune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, c_int_p, c_int_p]
lib.pt_tune_cache_store.argtypes = [C.c_char_p, C.c_char_p, C.c_int, C.c_int]
lib.pt_tebd_get_dims.argtypes = [C.c_void_p, C.c_int, c_int_p, c_int_p]
lib.pt_tebd_get_lambda.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, C.c_int]
lib.pt_tebd_get_lognorm.argtypes = [C.c_void_p, C.c_int, c_double_p]
lib.pt_tebd_get_gamma.argtypes = [C.c_void_p, C.c_int, C.c_int, c_double_p, C.c_size_t]
lib.pt_tebd_get_lognorms.argtypes = [C.c_void_p, C.c_int, c_double_p]
lib.pt_tebd_get_svd_sweeps.argtypes = [C.c_void_p, c_int_p, C.c_int]
lib.pt_tebd_clone.argtypes = [C.c_void_p, C.POINTER(C.c_void_p)]
lib.pt_tebd_read_bond_log.argtypes = [C.c_void_p, C.c_int, C.c_int, c_int_p, C.c_size_t]
lib.pt_tebd_sync.argtypes = [C.c_void_p]
lib.pt_tebd_destroy.argtypes = [C.c_void_p]
lib.pt_tebd_last_error.argtypes = [C.c_void_p]
lib.pt_tebd_last_error.restype = C.c_char_p
lib.pt_tebd_set_timing.argtypes = [C.c_void_p, C.c_int]
lib.pt_tebd_get_timing.argtypes = [C.c_void_p, c_double_p]
lib.pt_svd_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
lib.pt_svd_scratch_bytes.restype = C.c_size_t
lib.pt_svd_f64.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_int, C.c_void_p]


lib.pt_zgemm_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
lib.pt_zgemm_scratch_bytes.restype = C.c_size_t
lib.pt_zgemm_sliced.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_longlong,
                                C.c_void_p, C.c_int, C.c_longlong, C.c_void_p, C.c_int, C.c_longlong, C.c_int,
                                C.c_void_p, C.c_void_p]
lib.pt_qr_scratch_bytes.argtypes = [C.c_int, C.c_int, C.c_int]
lib.pt_qr_scratch_bytes.restype = C.c_size_t
lib.pt_qr_f64.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
lib.pt_svd_f64_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_int, C.c_void_p]
NOALLOC_MAX_BYTES = 16 << 20     # PT_SVD_NOALLOC_MAX_BYTES


lib.pt_selftest_grid_barrier.argtypes = [C.c_int, C.c_double, C.POINTER(C.c_int)]
lib.pt_selftest_grid_barrier.restype = C.c_int


def _check(rc, h=None):
    if rc < 0:
        msg = lib.pt_tebd_last_error(h)
        raise PTError(rc, msg.decode() if msg else "")
    return rc


def _dptr(a):
    return a.ctypes.data_as(c_double_p)


def _c128(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.complex128))


_ALLOCATOR_REFS = []


def use_torch_allocator(device=None):
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch

    dev = torch.cuda.current_device() if device is None else device

    def _alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
        except Exception:
            return None

    def _free(ptr, ctx):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    _ALLOCATOR_REFS[:] = [fa, ff]
    lib.pt_tebd_set_allocator(fa, ff, None)


def current_stream_handle():
    import torch

    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Engine:
    """One pt_tebd handle. Arguments mirror pt_tebd_init (host numpy arrays, complex128)."""

    def __init__(self, chains: Sequence[dict], pt_mpos: Sequence[Sequence[np.ndarray]], chi_max: int,
                 eps: float, precision: str = "fp64", multiplet_tol: float = 1e-12,
                 max_steps: int = 0, max_sweeps: int = 0, use_graph: bool = True, stream=None,
                 autotune: bool = True, tune_cache: Optional[str] = TUNE_CACHE, route=None, _handle=None):
        self._keep = []
        self.h = C.c_void_p()
        self.n_chains = len(chains)
        self.N = [int(c["N"]) for c in chains]
        self.n_max = max(self.N)
        self.n_ops = 0
        if _handle is not None:
            self.h = _handle
            return
        descs = (ChainDesc * len(chains))()
        for i, ch in enumerate(chains):
            d = descs[i]
            N = int(ch["N"])
            d.N = N
            if ch.get("rho0") is not None:
                r = _c128(ch["rho0"]).reshape(N, 4)
                self._keep.append(r)
                d.rho0 = _dptr(r)
            if N > 1:
                gq = _c128(ch["gates_q"]).reshape(N - 1, 16, 16)
                gh = _c128(ch["gates_h"]).reshape(N - 1, 16, 16)
                self._keep += [gq, gh]
                d.gates_q, d.gates_h = _dptr(gq), _dptr(gh)
            if ch.get("local_prop") is not None:
                lp = _c128(ch["local_prop"]).reshape(N, 4, 4)
                self._keep.append(lp)
                d.local_prop = _dptr(lp)
            ids = np.ascontiguousarray(np.asarray(ch.get("ptmpo_id", [-1] * N), dtype=np.int32))
            self._keep.append(ids)
            d.ptmpo_id = ids.ctypes.data_as(c_int_p)
            if ch.get("gamma0") is not None:
                chi0 = np.ascontiguousarray(np.asarray(ch["chi0"], dtype=np.int32))
                kap0 = np.ascontiguousarray(np.asarray(ch["kappa0"], dtype=np.int32))
                gams = [_c128(g) for g in ch["gamma0"]]
                lams = [np.ascontiguousarray(np.asarray(l, dtype=np.float64)) for l in ch["lambda0"]]
                gp = (c_double_p * N)(*[_dptr(g) for g in gams])
                lp_ = (c_double_p * (N + 1))(*[_dptr(l) for l in lams])
                self._keep += [chi0, kap0, gams, lams, gp, lp_]
                d.chi0 = chi0.ctypes.data_as(c_int_p)
                d.kappa0 = kap0.ctypes.data_as(c_int_p)
                d.gamma0 = gp
                d.lambda0 = lp_
                if ch.get("lognorm0") is not None:
                    ln = np.ascontiguousarray(np.asarray(ch["lognorm0"], dtype=np.float64).reshape(N + 1))
                    self._keep.append(ln)
                    d.lognorm0 = _dptr(ln)
        mdescs = (MpoDesc * max(1, len(pt_mpos)))()
        for m, Ps in enumerate(pt_mpos):
            K = len(Ps)
            kap = [Ps[0].shape[0]] + [P.shape[3] for P in Ps]
            kap = np.ascontiguousarray(np.asarray(kap, dtype=np.int32))
            arrs = [_c128(P) for P in Ps]
            ptrs = (c_double_p * K)(*[_dptr(a) for a in arrs])
            self._keep += [kap, arrs, ptrs]
            mdescs[m].K = K
            mdescs[m].kappa = kap.ctypes.data_as(c_int_p)
            mdescs[m].P = ptrs
        force = 0
        if route is not None:                     # (qr route, outer-QR route) by name, for tests
            force = 1 + QR_ROUTES[route[0]] + 4 * K2_ROUTES[route[1]]
        cache = tune_cache.encode() if tune_cache else None
        self._keep.append(cache)
        opt = Options(chi_max=int(chi_max), eps=float(eps), multiplet_tol=float(multiplet_tol),
                      precision=PRECISIONS[precision], max_steps=int(max_steps),
                      max_sweeps=int(max_sweeps), use_graph=int(bool(use_graph)),
                      autotune=int(bool(autotune)), tune_cache=cache, force_route=force)
        st = stream if stream is not None else current_stream_handle()
        rc = lib.pt_tebd_init(C.byref(self.h), descs, len(chains), mdescs, len(pt_mpos),
                              C.byref(opt), st)
        _check(rc, None)
        self._keep = []       # the library copied everything

    # --- C ABI wrappers (same names) ---------------------------------------------------
    def set_observables(self, ops):
        ops = _c128(ops).reshape(-1, 2, 2)
        _check(lib.pt_tebd_set_observables(self.h, _dptr(ops), len(ops)), self.h)
        self.n_ops = len(ops)

    def step(self, n_steps=1):
        _check(lib.pt_tebd_step(self.h, int(n_steps)), self.h)

    def observe(self, ops, normalize=False):
        ops = _c128(ops).reshape(-1, 2, 2)
        out = np.zeros((self.n_chains, self.n_max, len(ops)), dtype=np.complex128)
        tr = np.zeros(self.n_chains, dtype=np.complex128)
        _check(lib.pt_tebd_observe(self.h, _dptr(ops), len(ops), _dptr(out), _dptr(tr),
                                   int(bool(normalize))), self.h)
        return out, tr

    def read_history(self, first, count):
        out = np.zeros((count, self.n_chains, self.n_max, self.n_ops), dtype=np.complex128)
        tr = np.zeros((count, self.n_chains), dtype=np.complex128)
        _check(lib.pt_tebd_read_history(self.h, int(first), int(count), _dptr(out), _dptr(tr)), self.h)
        return out, tr

    def apply_local(self, chain, site, op, side="left"):
        op = _c128(op).reshape(2, 2)
        _check(lib.pt_tebd_apply_local(self.h, int(chain), int(site), _dptr(op),
                                       0 if side == "left" else 1), self.h)

    def steps_done(self):
        return _check(lib.pt_tebd_steps_done(self.h), self.h)

    def routes(self):
        """pt_tebd_get_routes: {'odd'|'even': (qr route, outer-QR route, tuned, from cache, timings)}."""
        out = np.zeros(8, dtype=np.int32)
        ms = np.zeros(10, dtype=np.float32)
        _check(lib.pt_tebd_get_routes(self.h, out.ctypes.data_as(c_int_p), ms.ctypes.data_as(C.POINTER(C.c_float))),
               self.h)
        qn = {v: k for k, v in QR_ROUTES.items()}
        kn = {v: k for k, v in K2_ROUTES.items()}
        return {layer: (qn[int(out[4 * l])], kn[int(out[4 * l + 1])], bool(out[4 * l + 2]), bool(out[4 * l + 3]),
                        [float(x) for x in ms[5 * l:5 * l + 5]])
                for l, layer in enumerate(("odd", "even"))}

    def step_kernels(self):
        """pt_tebd_step_kernels: kernel launches per step (nodes of the captured step graph)."""
        return _check(lib.pt_tebd_step_kernels(self.h), self.h)

    def get_dims(self, chain):
        N = self.N[chain]
        chi = np.zeros(N + 1, dtype=np.int32)
        kap = np.zeros(N, dtype=np.int32)
        _check(lib.pt_tebd_get_dims(self.h, int(chain), chi.ctypes.data_as(c_int_p),
                                    kap.ctypes.data_as(c_int_p)), self.h)
        return chi, kap

    def get_lambda(self, chain, bond, cap=4096):
        out = np.zeros(cap, dtype=np.float64)
        n = _check(lib.pt_tebd_get_lambda(self.h, int(chain), int(bond), _dptr(out), cap), self.h)
        return out[:n]

    def get_lognorm(self, chain):
        v = C.c_double()
        _check(lib.pt_tebd_get_lognorm(self.h, int(chain), C.byref(v)), self.h)
        return v.value

    def get_gamma(self, chain, site):
        """pt_tebd_get_gamma: Gamma_n of one site, complex [chi_{n-1}][4][kappa_n][chi_n]."""
        chi, kap = self.get_dims(chain)
        shape = (int(chi[site]), 4, int(kap[site]), int(chi[site + 1]))
        out = np.zeros(shape, dtype=np.complex128)
        n = _check(lib.pt_tebd_get_gamma(self.h, int(chain), int(site), _dptr(out), out.size), self.h)
        assert n == out.size
        return out

    def checkpoint(self):
        """The full augmented MPS of every chain at the current step (App. B.2), on the host:
        [{'step', 'chi', 'kappa', 'gamma': [N], 'lambda': [N + 1], 'lognorm': [N + 1]}]."""
        step = self.steps_done()
        out = []
        for c in range(self.n_chains):
            chi, kap = self.get_dims(c)
            out.append({"step": step, "chi": chi.copy(), "kappa": kap.copy(),
                        "gamma": [self.get_gamma(c, n) for n in range(self.N[c])],
                        "lambda": [self.get_lambda(c, b)[:int(chi[b])].copy() for b in range(self.N[c] + 1)],
                        "lognorm": self.get_lognorms(c)})
        return out

    def get_lognorms(self, chain):
        """pt_tebd_get_lognorms: the log-norm carried by each of the chain's N + 1 bonds."""
        out = np.zeros(self.N[chain] + 1, dtype=np.float64)
        _check(lib.pt_tebd_get_lognorms(self.h, int(chain), _dptr(out)), self.h)
        return out

    def get_svd_sweeps(self, cap=4096):
        """[(Jacobi sweeps, fault flags)] of the latest update of every bond (odd layer first)."""
        out = np.zeros(2 * cap, dtype=np.int32)
        n = _check(lib.pt_tebd_get_svd_sweeps(self.h, out.ctypes.data_as(c_int_p), cap), self.h)
        return out[:2 * min(n, cap)].reshape(-1, 2)

    def read_bond_log(self, first, count, nb_max=4096):
        """pt_tebd_read_bond_log: ([count, 6, nb, 8] int fields 0-7, [count, 6, nb] discarded weight)."""
        n_ints = count * 6 * nb_max * 10
        buf = np.zeros(max(1, n_ints), dtype=np.int32)
        nb = _check(lib.pt_tebd_read_bond_log(self.h, int(first), int(count), buf.ctypes.data_as(c_int_p),
                                              n_ints), self.h)
        rec = buf[:count * 6 * nb * 10].reshape(count, 6, nb, 10)
        disc = np.ascontiguousarray(rec[..., 8:10]).view(np.float64)[..., 0]
        return rec[..., :8].copy(), disc

    def sync(self):
        _check(lib.pt_tebd_sync(self.h), self.h)

    def clone(self):
        h2 = C.c_void_p()
        _check(lib.pt_tebd_clone(self.h, C.byref(h2)), self.h)
        e = Engine.__new__(Engine)
        e._keep, e.h, e.n_chains, e.N, e.n_max, e.n_ops = [], h2, self.n_chains, list(self.N), self.n_max, self.n_ops
        return e

    def set_timing(self, enable=True):
        _check(lib.pt_tebd_set_timing(self.h, int(bool(enable))), self.h)

    def get_timing(self):
        out = np.zeros(9, dtype=np.float64)
        _check(lib.pt_tebd_get_timing(self.h, _dptr(out)), self.h)
        return out

    def destroy(self):
        if self.h:
            lib.pt_tebd_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def resume_problem(chains, pt_mpos, ckpt):
    """Inputs of pt_tebd_init that continue a run from a checkpoint (Engine.checkpoint) taken after
    step s: every chain starts from its augmented MPS and log-norm at step s, and every PT-MPO is cut
    to its tensors P^(s+1), ... (its bond kappa[s] becomes the first). The new handle continues the
    same run (bit for bit when the cut PT-MPOs keep their largest bond, so the new handle has the same
    capacities); its history index 0 is step s of the original run."""
    steps = {int(ck["step"]) for ck in ckpt}
    if len(steps) != 1:
        raise ValueError("checkpoint chains are at different steps")
    s = steps.pop()
    out = []
    for ch, ck in zip(chains, ckpt):
        d = dict(ch)
        d.update(rho0=None, chi0=np.asarray(ck["chi"], dtype=np.int32),
                 kappa0=np.asarray(ck["kappa"], dtype=np.int32),
                 gamma0=[np.array(g, dtype=np.complex128) for g in ck["gamma"]],
                 lambda0=[np.asarray(l, dtype=np.float64) for l in ck["lambda"]],
                 lognorm0=np.asarray(ck["lognorm"], dtype=np.float64).copy())
        out.append(d)
    return out, [list(Ps[s:]) for Ps in pt_mpos]


def svd_scratch_bytes(m, n, batch):
    return int(lib.pt_svd_scratch_bytes(int(m), int(n), int(batch)))


def svd_f64(A, sigma, U, V, scratch, max_sweeps=0, stream=None):
    """Batched FP64 Jacobi SVD on device tensors: A [b,m,n] complex128, sigma [b,k] float64,
    U [b,m,k], V [b,n,k] complex128 (k = min(m,n)); scratch: uint8 tensor of svd_scratch_bytes."""
    b, m, n = A.shape
    st = stream if stream is not None else current_stream_handle()
    rc = lib.pt_svd_f64(C.c_void_p(A.data_ptr()), m, n, b, C.c_void_p(sigma.data_ptr()),
                        C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()),
                        C.c_void_p(scratch.data_ptr()), int(max_sweeps), st)
    _check(rc, None)


ZOPS = {"N": 0, "T": 1, "H": 2}


def zgemm_scratch_bytes(m, n, k, batch):
    return int(lib.pt_zgemm_scratch_bytes(int(m), int(n), int(k), int(batch)))


def zgemm_sliced(opA, opB, A, B, C_out, m, n, k, scratch, stream=None):
    """pt_zgemm_sliced on device tensors: C[b] = opA(A[b]) opB(B[b]) (column-major, complex128).
    A, B, C_out: [batch, cols, rows] contiguous tensors, i.e. each batch entry column-major with its
    row count as leading dimension; opA/opB in "N", "T", "H"; scratch: uint8 tensor of
    zgemm_scratch_bytes(m, n, k, batch)."""
    b = A.shape[0]
    lda, ldb, ldc = A.shape[2], B.shape[2], C_out.shape[2]
    st = stream if stream is not None else current_stream_handle()
    rc = lib.pt_zgemm_sliced(ZOPS[opA], ZOPS[opB], int(m), int(n), int(k), C.c_void_p(A.data_ptr()), lda,
                             A.shape[1] * A.shape[2], C.c_void_p(B.data_ptr()), ldb, B.shape[1] * B.shape[2],
                             C.c_void_p(C_out.data_ptr()), ldc, C_out.shape[1] * C_out.shape[2], int(b),
                             C.c_void_p(scratch.data_ptr()), st)
    _check(rc, None)


def qr_scratch_bytes(m, n, batch):
    return int(lib.pt_qr_scratch_bytes(int(m), int(n), int(batch)))


def qr_f64(A, R, scratch, stream=None):
    """pt_qr_f64 on device tensors: A [batch, n, m] complex128 (each entry column-major m x n) is
    replaced by Q; R [batch, n, n] (column-major) receives the triangular factor."""
    b, n, m = A.shape
    st = stream if stream is not None else current_stream_handle()
    _check(lib.pt_qr_f64(C.c_void_p(A.data_ptr()), int(m), int(n), int(b), C.c_void_p(R.data_ptr()),
                         C.c_void_p(scratch.data_ptr()), st), None)


def svd_f64_noalloc(A, sigma, U, V, max_sweeps=0, stream=None):
    """pt_svd_f64_noalloc: the same SVD as svd_f64 with no workspace argument. For callers that
    cannot allocate device memory; the library's static workspace (NOALLOC_MAX_BYTES) is shared by
    every call, so calls must not overlap on the GPU."""
    b, m, n = A.shape
    st = stream if stream is not None else current_stream_handle()
    rc = lib.pt_svd_f64_noalloc(C.c_void_p(A.data_ptr()), m, n, b, C.c_void_p(sigma.data_ptr()),
                                C.c_void_p(U.data_ptr()), C.c_void_p(V.data_ptr()), int(max_sweeps), st)
    _check(rc, None)


def selftest_grid_barrier(withheld_block=-1, limit_ms=1.0):
    """pt_selftest_grid_barrier: run the cooperative kernels' bounded grid barrier with one CTA
    withheld (-1: none) and a wait limit of limit_ms; returns (return code, device status bits)
    without raising, PT_ERR_DEVICE_TIMEOUT being the expected code when a CTA is withheld."""
    st = C.c_int(0)
    rc = lib.pt_selftest_grid_barrier(int(withheld_block), float(limit_ms), C.byref(st))
    return rc, st.value


def tune_cache_lookup(path, key):
    """pt_tune_cache_lookup: (qr, k2) of the last valid line of `key`, or None."""
    qr, k2 = C.c_int(-1), C.c_int(-1)
    rc = lib.pt_tune_cache_lookup(path.encode(), key.encode(), C.byref(qr), C.byref(k2))
    _check(rc, None)
    return (qr.value, k2.value) if rc == 1 else None


def tune_cache_store(path, key, qr, k2):
    """pt_tune_cache_store: append a choice for `key`."""
    _check(lib.pt_tune_cache_store(path.encode(), key.encode(), int(qr), int(k2)), None)
