#!/usr/bin/env python3
"""Benchmark of the PT-TEBD time step on GB300 (site-steps/s), one JSON line on stdout.

Workload (default): the 21-site isotropic XY chain with an Ohmic bath on every site (alpha=0.05,
w_c=3, T=0.8), one central excitation, dt=0.1, PT-MPO bond <= 16, chi <= 128, eps = 1e-6 (a
100-step trajectory; the largest single-GPU workload). A "step" is one full PT-TEBD time step (three
bond layers, the PT site layer, three bond layers, readout). W warm-up steps run from t = 0, then K
steps are timed, each with CUDA events on the library's stream and an L2 flush (a 256 MiB write)
between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16_ozaki|fp64|tf32x3|bf16x3|tf32x1]
The default times the fast path (theta + gate on tensor cores from exact-accumulation BF16 slices,
FP64 SVD) and, on the same window, the FP64 path; the five-site two-bath chain is reported as a
secondary workload.
  python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores, same metric
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PT-TEBD site-steps/s and TFLOP/s vs roofline, FP32-TC vs FP64 at <=1e-5 obs err"
UNIT = "site-steps/s"
DEFAULT_WORKLOAD = "xy21_allbaths"
SECONDARY_WORKLOAD = "xyz5_twobaths"
SM_COUNT = 152
FP64_FLOPS_PER_CLK_PER_SM = 4.0       # 2 DFMA / clk / SM: 1.26 TFLOP/s at 2.07 GHz x 152 SMs
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16_ozaki",
                    choices=["bf16_ozaki", "fp64", "tf32x3", "bf16x3", "tf32x1"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0)
    # a smaller case of the same kernels (lower bond cap, smaller capacity buffers), for profiling
    ap.add_argument("--chi-max", type=int, default=0)
    ap.add_argument("--no-fp64-path", action="store_true")
    # profiling aid: write the timed handle's bond log of steps 0..W+K ([step][layer][bond][field], .npy)
    ap.add_argument("--bond-log", default="")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons, sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return None
    return None


# ------------------------------------------------------------------------ algorithmic flops
def svd_flops(mD, nD, k):
    """SVD of an m x n complex D of numerical rank k (the pivoted QR's rank), Golub-Van Loan counts:
    Householder QR to rank k, 4(4mnk - 2k^2(m+n) + 4k^3/3); the SVD of the n x k factor with both
    singular-vector sets, 4(4n^2k + 8nk^2 + 9k^3); and U = D V, 8mnk (complex flops = 4 real)."""
    m, n = max(mD, nD), min(mD, nD)
    k = n if k <= 0 else min(k, n)
    qr = 4.0 * (4.0 * m * n * k - 2.0 * k * k * (m + n) + 4.0 * k ** 3 / 3.0)
    small = 4.0 * (4.0 * n * n * k + 8.0 * n * k * k + 9.0 * k ** 3)
    return qr + small + 8.0 * m * n * k


def svd_flops_full(mD, nD):
    """The full-rank Golub-Van Loan count 4(4m^2n + 8mn^2 + 9n^3) x 4 (complex)."""
    m, n = max(mD, nD), min(mD, nD)
    return 4.0 * (4 * m * m * n + 8 * m * n * n + 9 * n ** 3)


def log_flops(rec):
    """SVD flops of every bond update of the window from the device bond log [K, 6, nb, 8]."""
    mD, nD, k = rec[..., 0].astype(np.float64), rec[..., 1].astype(np.float64), rec[..., 2]
    tot = full = 0.0
    for m, n, kk in zip(mD.ravel(), nD.ravel(), k.ravel()):
        if m > 0 and n > 0:
            tot += svd_flops(m, n, int(kk))
            full += svd_flops_full(m, n)
    return tot, full


RSVD_POWER = 2          # the fast path's power iterations (rsvd.cu)


def hqr_flops(m, n):
    """Complex Householder QR of an m x n matrix with the explicit Q: 8(mn^2 - n^3/3) to factor and
    as much again to form Q (Golub-Van Loan, complex = 4 real)."""
    return 16.0 * (m * n * n - n ** 3 / 3.0) if m >= n > 0 else 0.0


def rsvd_flops(rec):
    """The fast path's randomized SVD over the window from the device bond log [K, 6, nb, >=6]
    (rows, columns, range-finder width l, ..., kept chi): the range finder's QRs ((1 + q) of the
    m x l sketches Y, (q + 1) of the n x l sketches Z) and the tensor-core products ((1 + q) D Omega /
    D Qz, (q + 1) D^H Q, the residual D - Q Z^H, the kept vectors Q Wr and Qb Ur; complex MAC = 8)."""
    qr = gemm = 0.0
    q = RSVD_POWER
    for r in rec.reshape(-1, rec.shape[-1]):
        mD, nD, l, chi = int(r[0]), int(r[1]), int(r[2]), int(r[5])
        if mD <= 0 or nD <= 0 or l <= 0:
            continue
        m, n = max(mD, nD), min(mD, nD)
        qr += (1 + q) * hqr_flops(m, l) + (q + 1) * hqr_flops(n, l)
        gemm += 8.0 * m * n * l * ((1 + q) + (q + 1) + 1) + 8.0 * (m + n) * l * chi
    return qr, gemm


def sketch_elements(rec):
    """Sketch elements m l the range finder's QRs factor over the window: (1 + q) m x l sketches Y and
    (q + 1) n x l sketches Z per bond update (bond log [K, 6, nb, >=3])."""
    tot = 0.0
    q = RSVD_POWER
    for r in rec.reshape(-1, rec.shape[-1]):
        mD, nD, l = int(r[0]), int(r[1]), int(r[2])
        if mD > 0 and nD > 0 and l > 0:
            tot += ((1 + q) * max(mD, nD) + (q + 1) * min(mD, nD)) * l
    return tot


def bond_sizes(chis, kaps, N):
    """(m_L, n_L, m_R, n_R, r_L, r_R, chi) of every bond for the given dims (App. A.2)."""
    out = []
    for b in range(N - 1):
        chl, chc, chr_ = chis[b], chis[b + 1], chis[b + 2]
        mL, nL = chl * kaps[b], 4 * chc
        mR, nR = 4 * chc, kaps[b + 1] * chr_
        out.append((mL, nL, mR, nR, min(mL, nL), min(mR, nR), chc))
    return out


def step_flops_rest(chis, kaps, N):
    """Algorithmic flops of one step outside the SVD: the outer-block QR/LQ (with explicit Q), theta
    with the gate, the Gamma recovery (each bond update: odd bonds 4x, even bonds 2x per step), and
    the PT site contractions."""
    other = theta = 0.0
    for b, (mL, nL, mR, nR, rL, rR, chc) in enumerate(bond_sizes(chis, kaps, N)):
        reps = 4 if b % 2 == 0 else 2
        f_qr = (32.0 * (mL * nL * nL - nL ** 3 / 3) if mL > nL else 0.0) + \
               (32.0 * (nR * mR * mR - mR ** 3 / 3) if nR > mR else 0.0)
        f_theta = 128.0 * rL * rR * chc + 2048.0 * rL * rR
        f_rec = 8.0 * (mL * rL * 4 * chc if mL > nL else 0) + 8.0 * (nR * rR * 4 * chc if nR > mR else 0)
        other += reps * (f_qr + f_theta + f_rec)
        theta += reps * f_theta
    for n in range(N):
        chl, chr_ = chis[n], chis[n + 1]
        other += 8.0 * chl * chr_ * 4 * kaps[n] * 4 * kaps[n]
    return other, theta


# ------------------------------------------------------------------------ replicas across ranks
def aggregate(total_ms, site_steps_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: the timed region is the maximum over ranks,
    the work is every rank's site-steps. Returns (value, max_ms)."""
    import torch
    world = 1
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        t = torch.tensor([float(total_ms), float(site_steps_local)], dtype=torch.float64, device=device)
        mx = t.clone()
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        sm = t.clone()
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
        total_ms, work = float(mx[0]), float(sm[1])
    else:
        work = float(site_steps_local)
    return work / (total_ms / 1e3), total_ms


def traffic_record(kernel_src, elements_per_launch=None):
    """DRAM bytes per launch of the dominant stage from a committed ncu capture, or None once the
    kernel source has changed since that capture (the record carries the source's SHA-256). A record
    taken on a smaller case gives bytes per sketch element; it is scaled by this run's elements per
    launch (elements_per_launch)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None, "no ncu capture recorded"
    try:
        rec = json.load(open(TRAFFIC_FILE))
    except Exception:
        return None, "unreadable capture record"
    sha = {}
    for f in rec.get("sources", []):
        p = os.path.join(ROOT, "paper_2201_05529_gb300", "csrc", f)
        sha[f] = hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] if os.path.exists(p) else None
    if any(sha[f] != rec.get("sha", {}).get(f) for f in sha) or not sha or sorted(sha) != sorted(kernel_src):
        return None, "no ncu capture of this kernel's current source"
    if "dram_bytes_per_sketch_element" in rec and elements_per_launch:
        return rec["dram_bytes_per_sketch_element"] * elements_per_launch, rec.get("how", "")
    return rec.get("dram_bytes_per_launch"), rec.get("how", "")


# ------------------------------------------------------------------------ our arm
def _timed_window(eng, K, stream, flush, torch):
    """K single steps, each bracketed by CUDA events on the library's stream, L2 flushed between."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize()
    for i in range(K):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        eng.step(1)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _secondary(capi, pp, workload, torch, stream, flush, prec, W=5, K=20):
    """The five-site two-bath chain (the previous headline): fast path and FP64 path on one window."""
    w = workload(SECONDARY_WORKLOAD)
    chains, mpos = pp.build_problem(w)
    N = sum(c["N"] for c in chains)
    out = {"workload": w.name, "window": f"steps {W}..{W + K} of {w.K}"}
    hist = {}
    for p in (prec, "fp64"):
        e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=p, multiplet_tol=w.multiplet_tol,
                        max_steps=w.K, use_graph=True)
        e.set_observables([pp.pauli("z")])
        e.step(W)
        ms = _timed_window(e, K, stream, flush, torch)
        hist[p], _ = e.read_history(W, K + 1)
        e.destroy()
        out[p] = {"value": N * K / (sum(ms) / 1e3), "ms_per_step": float(np.mean(ms))}
    out["speedup_vs_fp64_path"] = out[prec]["value"] / out["fp64"]["value"]
    out["max_sz_diff_vs_fp64_path"] = float(np.max(np.abs(hist[prec] - hist["fp64"])))
    return out


def _stress(capi, pp, workload, torch, stream, flush, prec, W=1, K=2):
    """The random augmented-MPS stress workload at full size (N = 32, chi = 96, kappa = 16 on every
    site: D up to 1536 x 1536), the fast path only (the FP64 path's exact Jacobi on full-rank D of
    that size runs minutes per step)."""
    w = workload("random32_stress")
    out = {"workload": w.name, "precision": prec, "window": f"steps {W}..{W + K} of {w.K}"}
    try:
        chains, mpos = pp.build_problem(w)
        N = sum(c["N"] for c in chains)
        e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=prec, multiplet_tol=w.multiplet_tol,
                        max_steps=w.K, use_graph=True)
        e.set_observables([pp.pauli("z")])
        e.step(W)
        ms = _timed_window(e, K, stream, flush, torch)
        blog, _ = e.read_bond_log(W, K)
        e.destroy()
        out.update(value=N * K / (sum(ms) / 1e3), ms_per_step=float(np.mean(ms)),
                   max_D=[int(blog[..., 0].max()), int(blog[..., 1].max())])
    except Exception as ex:          # reported, not fatal
        out["error"] = str(ex)[:300]
    return out


def run_ours(args, rank, world, local):
    import torch
    import paper_2201_05529_gb300 as pkg
    from paper_2201_05529_gb300 import problem as pp
    from workloads import workload

    torch.cuda.set_device(local)
    pkg.build()
    capi = pkg.load()
    capi.use_torch_allocator(local)
    w = workload(args.workload) if args.chi_max <= 0 else workload(args.workload, chi_max=args.chi_max)
    chains, mpos = pp.build_problem(w)
    K, W = args.steps, args.warmup
    if W + K > w.K:
        raise SystemExit(f"warmup + steps must be <= {w.K} (the PT-MPO length of {w.name})")
    Z = pp.pauli("z")
    site_steps_per_step = sum(c["N"] for c in chains)
    n_chains = len(chains)

    def make(precision, graph=True):
        e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=precision,
                        multiplet_tol=w.multiplet_tol, max_steps=w.K, use_graph=graph)
        e.set_observables([Z])
        return e

    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # --- main timed run: graph replay, per-step events, L2 flush between steps
    eng = make(args.precision)
    eng.step(W)
    eng.sync()
    stage_eng = eng.clone()                  # the same state at step W, for the per-stage timing
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        step_ms = _timed_window(eng, K, stream, flush, torch)
    if world > 1:
        dist.barrier()
    value, total_ms = aggregate(float(np.sum(step_ms)), site_steps_per_step * K,
                                dist if world > 1 else None, device="cuda")
    eng.sync()
    launches_per_step = eng.step_kernels()
    routes = eng.routes()
    hist_fast, _ = eng.read_history(W, K + 1)
    blog, disc = eng.read_bond_log(W, K)
    if args.bond_log:
        np.save(args.bond_log, eng.read_bond_log(0, W + K)[0])
    dims = [eng.get_dims(c) for c in range(n_chains)]
    eng.destroy()
    fl_rest = fl_theta = 0.0
    for c, (chi, kap) in enumerate(dims):
        o_, t_ = step_flops_rest(list(chi), list(kap), chains[c]["N"])
        fl_rest += o_ * K          # the window's last dims: an upper estimate for the earlier steps
        fl_theta += t_ * K

    # --- per-stage device time over the same window (eager launches with events, on the clone)
    stage_eng.set_timing(True)
    stage = np.zeros(9)
    for i in range(K):
        flush.fill_(float(i))
        stage_eng.step(1)
        stage += stage_eng.get_timing()
    stage_eng.set_timing(False)
    stage_eng.destroy()

    # --- the plain FP64 GPU path on the same window (FP32-TC vs FP64)
    fp64 = None
    fp64_svd = None
    if args.precision != "fp64" and not args.no_fp64_path:
        e64 = make("fp64")
        e64.step(W)
        e64.sync()
        ms64 = _timed_window(e64, K, stream, flush, torch)
        hist64, _ = e64.read_history(W, K + 1)
        blog64, _ = e64.read_bond_log(W, K)
        e64.destroy()
        # its SVD's roofline on a short stage-timed sub-window (a second engine at step W)
        Ks = min(K, 5)
        e64s = make("fp64", graph=False)
        e64s.step(W)
        e64s.sync()
        e64s.set_timing(True)
        st64 = np.zeros(9)
        for i in range(Ks):
            flush.fill_(float(i))
            e64s.step(1)
            st64 += e64s.get_timing()
        e64s.destroy()
        f64, _ = log_flops(blog64[:Ks])
        ms64_svd = (st64[3] + st64[7] + st64[8]) / (Ks * 6)
        ach64 = (f64 / (Ks * 6)) / (ms64_svd / 1e3) / 1e12
        fp64_peak_ = SM_COUNT * FP64_FLOPS_PER_CLK_PER_SM * 2070.0 * 1e6 / 1e12
        fp64_svd = {"kernel": "FP64 path's bond SVD (pivoted QR, Jacobi sweeps on R^H, U = D V)", "bound": "alu",
                    "achieved": ach64, "peak": fp64_peak_, "unit": "TFLOP/s", "frac": ach64 / fp64_peak_,
                    "window": f"steps {W}..{W + Ks}", "ms_per_launch": ms64_svd,
                    "work": "Golub-Van Loan counts with the pivoted QR's rank (bond log)"}
        d = np.abs(hist64 - hist_fast)
        fp64 = {"value": site_steps_per_step * K / (float(np.sum(ms64)) / 1e3),
                "ms_per_step": float(np.mean(ms64)), "steps": K,
                "window": f"steps {W}..{W + K} (the same steps as the fast path)",
                "max_sz_diff_vs_fast_path": float(np.max(d)),
                "max_sz_diff_per_step": [float(x) for x in d.max(axis=(1, 2, 3))]}

    # --- roofline of the dominant kernel
    n_layers = 6
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_peak = SM_COUNT * FP64_FLOPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12
    mp = measured_peaks()
    src = ("MEASURED_PEAKS.json gives HBM copy and bf16 GEMM peaks only" if mp else "MEASURED_PEAKS.json absent")
    peak_src = ("derived: 152 SMs x 4 FP64 flop/clk x median SM clock (of derived; " + src +
                "; a DFMA probe measured 1.20 TFLOP/s)")
    bf16 = float(mp["bf16_tflops"]) if mp and "bf16_tflops" in mp else 1900.0
    sweeps = blog[..., 3]
    stage_ms = {"site": stage[0] / K, "blocks_qr": stage[1] / K, "theta": stage[2] / K,
                "svd_jacobi_sweeps": stage[3] / K, "svd_range_finder_qr": stage[7] / K,
                "svd_products_or_precond": stage[8] / K, "truncate": stage[4] / K,
                "recover": stage[5] / K, "readout": stage[6] / K}
    if args.precision == "bf16_ozaki":
        fl_qr, fl_gemm = rsvd_flops(blog)
        fl_path = fl_qr + fl_gemm
        n_qr = (1 + RSVD_POWER) + (RSVD_POWER + 1)          # QR launches per layer
        qr_ms = stage[7] / K / n_layers / n_qr              # per launch
        achieved = (fl_qr / (K * n_layers * n_qr)) / (qr_ms / 1e3) / 1e12
        traffic, tsrc = traffic_record(["hqr_grid.cu"], sketch_elements(blog) / (K * n_layers * n_qr))
        roofline = {"bound": "alu", "kernel": "k_hqr_items: whole-GPU Householder QR (explicit Q) of the randomized "
                                              "range finder's sketches Y (m x l) and Z (n x l) of every bond of a layer",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                    "traffic": traffic, "traffic_source": tsrc,
                    "work": "16 (m l^2 - l^3 / 3) per m x l QR with its explicit Q (GVL, complex = 4 real), "
                            f"{n_qr} QRs per bond update, m, n, l read from the device bond log",
                    "work_tflop_window": fl_qr / 1e12, "peak_source": peak_src,
                    "ms_per_launch": qr_ms, "launches_per_layer": n_qr,
                    "jacobi_sweeps_mean": float(np.mean(sweeps[sweeps > 0])) if np.any(sweeps > 0) else 0.0,
                    "range_width_over_n_mean": float(np.mean((blog[..., 2] / np.maximum(1, np.minimum(blog[..., 0], blog[..., 1])))
                                                             [blog[..., 0] > 0])),
                    "stage_ms_per_step": stage_ms}
        # the sliced tensor-core products (the fast path's dense contractions)
        gemm_s = stage[8] / 1e3
        roofline["tensor_products"] = {
            "kernel": "k_zgemm (+ k_zg_rowexp / k_zg_pack): D Omega, D^H Q, D Qz, D - Q Z^H, Q Wr, Qb Ur",
            "bound": "tensor", "achieved": fl_gemm / gemm_s / 1e12, "peak": bf16, "unit": "TFLOP/s",
            "frac": fl_gemm / gemm_s / 1e12 / bf16,
            "achieved_executed_bf16": 21.0 * fl_gemm / gemm_s / 1e12,
            "work": "complex products at 8 flops per MAC (algorithmic); each runs as 21 slice-pair x 4 real "
                    "BF16 products, the executed rate is 21 x the algorithmic one; stage time includes the "
                    "packing passes and the plan kernels",
            "peak_source": "of measured bf16 GEMM burst"}
    else:
        fl_svd, fl_svd_full = log_flops(blog)
        fl_path = fl_svd
        svd_ms = stage[3] + stage[7] + stage[8]
        achieved = (fl_svd / (K * n_layers)) / (svd_ms / K / n_layers / 1e3) / 1e12
        traffic, tsrc = traffic_record(["qrcp.cu", "jacobi_grid.cu", "svd_gemm.cu"])
        roofline = {"bound": "alu", "kernel": "FP64 bond SVD, one launch chain per layer: pivoted QR stopping at "
                                              "D's noise level, one-sided Jacobi sweeps on B = R^H, U = D V",
                    "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                    "traffic": traffic, "traffic_source": tsrc,
                    "work": "Golub-Van Loan counts of the SVD of each m x n D of numerical rank k (the pivoted "
                            "QR's rank, read from the device bond log): QR to rank k + SVD of the n x k factor + U = D V",
                    "work_tflop_window": fl_svd / 1e12, "work_full_rank_tflop_window": fl_svd_full / 1e12,
                    "peak_source": peak_src, "ms_per_launch": svd_ms / K / n_layers,
                    "jacobi_sweeps_mean": float(np.mean(sweeps[sweeps > 0])) if np.any(sweeps > 0) else 0.0,
                    "stage_ms_per_step": stage_ms}
    if args.precision != "fp64" and stage[2] > 0:
        # theta + gate on the tensor cores
        tpeak = bf16 * (1.1 / 2.25) if args.precision in ("tf32x3", "tf32x1") else bf16
        tach = (fl_theta / K) / (stage[2] / K / 1e3) / 1e12
        roofline["theta_tensor"] = {
            "kernel": "k_tc_pack + k_tc_theta (theta + gate as one tcgen05 GEMM, K = 4 chi)", "bound": "tensor",
            "achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
            "work": "128 r^2 chi + 2048 r^2 per bond update (algorithmic, complex MAC = 8)",
            "peak_source": "of measured bf16 GEMM burst" + (" x 1.1/2.25" if "tf32" in args.precision else "")}
    if fp64_svd is not None:
        roofline["fp64_path_svd"] = fp64_svd

    # --- end to end through the C ABI on the same steps W..W+K. The state after the W warm-up steps
    # is read to the host once (a checkpoint, untimed). The timed region then initialises a handle
    # from host buffers only (the augmented MPS at step W, the gates, the PT-MPOs cut at step W: every
    # input of the window goes host -> device), runs the K steps and reads their observables and
    # traces back to the host. One untimed handle of the same shapes is built and destroyed first,
    # so the tuner's cache and the loaded modules are warm, as for a user's repeated job.
    ck_eng = make(args.precision)
    ck_eng.step(W)
    ckpt = ck_eng.checkpoint()
    ck_eng.destroy()
    rchains, rmpos = capi.resume_problem(chains, mpos, ckpt)

    def make_resumed():
        e = capi.Engine(rchains, rmpos, chi_max=w.chi_max, eps=w.eps, precision=args.precision,
                        multiplet_tol=w.multiplet_tol, max_steps=K, use_graph=True)
        e.set_observables([Z])
        return e

    make_resumed().destroy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = make_resumed()
    e2.step(K)
    hist, tr = e2.read_history(0, K + 1)
    t1 = time.perf_counter()
    e2.destroy()
    h2d = 0
    for c in rchains:
        h2d += sum(g.nbytes for g in c["gamma0"]) + sum(l.nbytes for l in c["lambda0"])
        h2d += (c["gates_q"].nbytes + c["gates_h"].nbytes) if c["N"] > 1 else 0
    h2d += sum(P.nbytes for Ps in rmpos for P in Ps)
    d2h = hist.nbytes + tr.nbytes
    e2e = {"value": site_steps_per_step * K / (t1 - t0), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d / K), "d2h_bytes_per_step": int(d2h / K),
           "window": f"steps {W}..{W + K}, the same steps as value; timed: init from host buffers (the "
                     f"checkpointed state at step {W}, gates, PT-MPOs from step {W + 1}) + {K} steps + the "
                     f"history read",
           "max_sz_diff_vs_timed_run": float(np.max(np.abs(hist - hist_fast)))}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "bf16 TC slices (fp32 acc) + f64",
           "data": "synthetic (seeded workload; PT-MPOs built on the host from the stated Ohmic baths)",
           "config": {"workload": w.name, "chains": n_chains, "N": [c["N"] for c in chains],
                      "dt": w.dt, "chi_max": w.chi_max, "kappa_max": w.kappa_max, "eps": w.eps,
                      "precision": args.precision, "window": f"steps {W}..{W + K} of {w.K}",
                      "l2": "flushed between timed steps (256 MiB write)",
                      "parallelism": f"{world} replicas" if world > 1 else "single GPU"},
           "clocks": clocks, "roofline": roofline, "e2e": e2e,
           "routes": {layer: {"svd_pivoted_qr": r[0], "outer_block_qr": r[1], "tuned": r[2], "from_cache": r[3],
                              "candidate_ms": r[4]} for layer, r in routes.items()},
           "gpu_launches": int(launches_per_step) * K,
           "gpu_launches_per_step": int(launches_per_step),
           "algorithmic_tflops": (fl_path + fl_rest) / (total_ms / 1e3) / 1e12,
           "max_discarded_weight": float(np.max(disc)) if disc.size else 0.0}
    if fp64 is not None:
        out["fp64_path"] = fp64
        out["speedup_vs_fp64_path"] = value / fp64["value"]
    if not args.no_secondary and args.workload != SECONDARY_WORKLOAD:
        out["secondary"] = _secondary(capi, pp, workload, torch, stream, flush, args.precision)
        if args.precision == "bf16_ozaki":
            out["stress"] = _stress(capi, pp, workload, torch, stream, flush, args.precision)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds, W, K)
    if world > 1:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------------------ the oracle on the host
def _oracle_prefix(w, W):
    """The FP64 oracle's state after W untimed steps (the start of the GPU's timed window)."""
    from oracle import problem as oprob, pttebd
    cis = oprob.build_inputs(w)
    states = [pttebd.product_state(ci.rho0) if ci.init_mps is None else ci.init_mps.copy() for ci in cis]
    for k in range(1, W + 1):
        for ci, m in zip(cis, states):
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps, multiplet_tol=w.multiplet_tol)
    return cis, states


def _oracle_timed(w, cis, states, first, seconds, max_steps):
    """The oracle as it stands: steps first, first+1, .. timed one by one until `seconds` have passed
    (at least one step) or max_steps were taken."""
    from oracle import pttebd
    done, t_all = 0, 0.0
    for k in range(first, first + max_steps):
        t0 = time.perf_counter()
        for ci, m in zip(cis, states):
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps, multiplet_tol=w.multiplet_tol)
        t_all += time.perf_counter() - t0
        done += 1
        if t_all > seconds:
            break
    return done, t_all, sum(ci.N for ci in cis)


def cpu_baseline(w, seconds, W, K):
    """The oracle as it stands on the host cores, on the GPU's own window: its state after the W
    warm-up steps, then steps W+1.. timed until `seconds` have passed (a bounded sample of the same
    steps), plus the same sample with one BLAS thread (a subprocess starting from that state)."""
    import pickle
    import tempfile
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cis, states = _oracle_prefix(w, W)
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "state.pkl")
        with open(path, "wb") as f:
            pickle.dump((cis, [m.copy() for m in states]), f)
        done, t_all, N = _oracle_timed(w, cis, states, W + 1, seconds, K)
        out = {"value": N * done / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"steps {W + 1}..{W + done} of {w.name} (the first {done} of the GPU's {K} timed steps, "
                         f"from the oracle's own state after the {W} warm-up steps; numpy/LAPACK, "
                         f"{cores} host threads available)"}
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import sys, json, pickle; sys.path.insert(0, %r); import bench; from workloads import workload; "
                "cis, st = pickle.load(open(%r, 'rb')); "
                "d, t, n = bench._oracle_timed(workload(%r), cis, st, %d, %f, 1); print(json.dumps([d, t, n]))"
                % (ROOT, path, w.name, W + 1, seconds))
        try:
            r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
            d1, t1, n1 = json.loads(r.stdout.strip().splitlines()[-1])
            out["single_thread"] = {"value": n1 * d1 / t1, "cores": 1,
                                    "sample": f"step {W + 1} of {w.name}, one BLAS thread"}
        except Exception as ex:          # reported, not fatal
            out["single_thread"] = {"value": None, "error": str(ex)[:200]}
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from workloads import workload
    w = workload(args.workload)
    W, K = args.warmup, args.steps
    from oracle import problem as oprob, pttebd
    cis = oprob.build_inputs(w)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    site_steps = sum(ci.N for ci in cis)
    # the same trajectory: W untimed steps, then up to K timed steps within the time budget (each
    # step is one PT-TEBD step of every chain; later steps cost more, so a cut window is cheaper)
    states = []
    for ci in cis:
        m = pttebd.product_state(ci.rho0) if ci.init_mps is None else ci.init_mps.copy()
        for k in range(1, W + 1):
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps, multiplet_tol=w.multiplet_tol)
        states.append(m)
    ms = []
    t_all = 0.0
    for i in range(K):
        ts = time.perf_counter()
        for ci, m in zip(cis, states):
            pttebd.pt_step(m, W + i + 1, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps,
                           multiplet_tol=w.multiplet_tol)
        ms.append((time.perf_counter() - ts) * 1e3)
        t_all += ms[-1] / 1e3
        if t_all > args.ref_seconds:
            break
    done = len(ms)
    value = site_steps * done / t_all
    sample = (f"steps {W + 1}..{W + done} of {w.name} after {W} untimed steps"
              + ("" if done == K else f" ({done} of the {K} requested within the {args.ref_seconds:.0f} s budget)"))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_all * 1e3 / done, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": "synthetic (seeded workload; PT-MPOs built by the oracle)",
            "config": {"workload": w.name, "chains": len(cis), "precision": "fp64 (numpy/LAPACK)",
                       "window": f"steps {W}..{W + done} of {w.K}", "steps_timed": done},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
