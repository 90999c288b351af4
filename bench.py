#!/usr/bin/env python3
"""Benchmark of the PT-TEBD time step on GB300 (site-steps/s), one JSON line on stdout.

Workload (default): the five-site XYZ chain between a hot (T=5) and a cold (T=0.5) Ohmic bath,
alpha=0.16, w_c=4, dt=0.05, PT-MPO bond <= 32, chi <= 64, eps = 1e-8 (200-step trajectory).
A "step" is one full PT-TEBD time step of every chain (three bond layers, the PT site layer,
three bond layers, readout). W warm-up steps run from t = 0, then K steps are timed, each with
CUDA events on the library's stream and an L2 flush (a 256 MiB write) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision tf32x3|fp64|bf16x3|tf32x1]
The default times the FP32 tensor-core path (TF32x3) and, on the same window, the FP64 path.
  python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores, same metric
"""
from __future__ import annotations

import argparse
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
DEFAULT_WORKLOAD = "xyz5_twobaths"
SM_COUNT = 152
JACOBI_DRAM_BYTES_PER_LAUNCH = 1378048 + 174848   # bytes, ncu capture of the current k_jacobi_grid
FP64_FLOPS_PER_CLK_PER_SM = 4.0       # 2 DFMA / clk / SM: 1.25 TFLOP/s nominal at 2.07 GHz x 152 SMs


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "bf16x3", "tf32x1"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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
def bond_sizes(chis, kaps, N):
    """(m_L, n_L, m_R, n_R, r_L, r_R, chi) of every bond for the given dims (App. A.2)."""
    out = []
    for b in range(N - 1):
        chl, chc, chr_ = chis[b], chis[b + 1], chis[b + 2]
        mL, nL = chl * kaps[b], 4 * chc
        mR, nR = 4 * chc, kaps[b + 1] * chr_
        out.append((mL, nL, mR, nR, min(mL, nL), min(mR, nR), chc))
    return out


def svd_flops(m, n):
    """Golub-Van Loan dense SVD count with U and V, 4m^2n + 8mn^2 + 9n^3, x4 for complex."""
    if m < n:
        m, n = n, m
    return 4.0 * (4 * m * m * n + 8 * m * n * n + 9 * n ** 3)


def step_flops(chis, kaps, N):
    """Algorithmic flops of one step: 3 bond updates per bond (the O layers twice, E once, per
    half step -> odd bonds 4x, even bonds 2x), each QR + theta + SVD + recovery, plus the PT layer."""
    svd = other = theta = 0.0
    for b, (mL, nL, mR, nR, rL, rR, chc) in enumerate(bond_sizes(chis, kaps, N)):
        reps = 4 if b % 2 == 0 else 2
        mD, nD = 4 * rL, 4 * rR
        f_svd = svd_flops(mD, nD)
        f_qr = (16.0 * (mL * nL * nL - nL ** 3 / 3) if mL > nL else 0.0) + \
               (16.0 * (nR * mR * mR - mR ** 3 / 3) if nR > mR else 0.0)
        f_theta = 128.0 * rL * rR * chc + 2048.0 * rL * rR
        f_rec = 8.0 * (mL * rL * 4 * chc if mL > nL else 0) + 8.0 * (nR * rR * 4 * chc if nR > mR else 0)
        svd += reps * f_svd
        other += reps * (f_qr + f_theta + f_rec)
        theta += reps * f_theta
    return svd, other, theta


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


# ------------------------------------------------------------------------ our arm
# kernels per bond layer on the default route: blocks, QR/LQ reductions, theta (FP64: one kernel;
# fast path: two packs + the tcgen05 GEMM), pivoted QR, Jacobi, V_D scatter, U_D GEMM, U_D scale,
# truncation, recovery; per step 5 more (site contraction, swap, the two readout kernels, step counter)
LAUNCHES_PER_LAYER = {"fp64": 10, "fast": 12}


def _timed_window(eng, K, stream, flush, torch, n_chains, clk=None):
    """K single steps, each bracketed by CUDA events on the library's stream, L2 flushed between."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    dims = []
    torch.cuda.synchronize()
    for i in range(K):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        eng.step(1)
        ev[i][1].record(stream)
        dims.append([eng.get_dims(c) for c in range(n_chains)])   # synchronises; outside the events
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], dims


def run_ours(args, rank, world, local):
    import torch
    import paper_2201_05529_gb300 as pkg
    from paper_2201_05529_gb300 import problem as pp
    from workloads import workload

    torch.cuda.set_device(local)
    pkg.build()
    capi = pkg.load()
    capi.use_torch_allocator(local)
    w = workload(args.workload)
    chains, mpos = pp.build_problem(w)
    K, W = args.steps, args.warmup
    if W + K > w.K:
        raise SystemExit(f"warmup + steps must be <= {w.K} (the PT-MPO length of {w.name})")
    Z = pp.pauli("z")
    site_steps_per_step = sum(c["N"] for c in chains)
    n_chains = len(chains)

    def make(precision):
        e = capi.Engine(chains, mpos, chi_max=w.chi_max, eps=w.eps, precision=precision,
                        max_steps=w.K, use_graph=True)
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
    if world > 1:
        dist.barrier()
    with ClockSampler(local) as clk:
        step_ms, dims = _timed_window(eng, K, stream, flush, torch, n_chains)
    if world > 1:
        dist.barrier()
    value, total_ms = aggregate(float(np.sum(step_ms)), site_steps_per_step * K,
                                dist if world > 1 else None, device="cuda")
    eng.sync()
    sweeps = eng.get_svd_sweeps()
    hist_fast, _ = eng.read_history(W, K + 1)
    eng.destroy()
    fl_svd = fl_other = fl_theta = 0.0
    for per_chain in dims:
        for c, (chi, kap) in enumerate(per_chain):
            s_, o_, t_ = step_flops(list(chi), list(kap), chains[c]["N"])
            fl_svd += s_
            fl_other += o_
            fl_theta += t_

    # --- the plain FP64 GPU path on the same window (for the FP32-TC vs FP64 comparison)
    fp64 = None
    if args.precision != "fp64":
        k64 = K
        e64 = make("fp64")
        e64.step(W)
        e64.sync()
        ms64, _ = _timed_window(e64, k64, stream, flush, torch, n_chains)
        hist64, _ = e64.read_history(W, k64 + 1)
        e64.destroy()
        fp64 = {"value": site_steps_per_step * k64 / (float(np.sum(ms64)) / 1e3),
                "ms_per_step": float(np.mean(ms64)), "steps": k64,
                "window": f"steps {W}..{W + k64} (the same steps as the fast path)",
                "max_obs_diff_vs_fast_path": float(np.max(np.abs(hist64 - hist_fast[:k64 + 1])))}

    # --- per-stage timing (eager launches with events) over the same window
    eng = make(args.precision)
    eng.step(W)
    eng.sync()
    eng.set_timing(True)
    stage = np.zeros(9)
    nk = K
    for i in range(nk):
        flush.fill_(float(i))
        eng.step(1)
        stage += eng.get_timing()
    eng.set_timing(False)
    eng.destroy()
    stage /= nk
    n_layers = 6
    svd_ms = stage[3] + stage[7] + stage[8]
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_peak = SM_COUNT * FP64_FLOPS_PER_CLK_PER_SM * sm_mhz * 1e6 / 1e12
    achieved = (fl_svd / K / n_layers) / (svd_ms / n_layers / 1e3) / 1e12
    kernel = ("bond SVD (FP64 in every mode): pivoted QR k_qrcp_grid, one-sided Jacobi on R^H "
              "k_jacobi_grid<double>, U_D = D V_D / sigma k_mix_gemm")
    mp = measured_peaks()
    src = ("MEASURED_PEAKS.json gives HBM copy and bf16 GEMM peaks only" if mp else "MEASURED_PEAKS.json absent")
    roofline = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                # DRAM read + write of one k_jacobi_grid launch on a full-size layer (step 16, two
                # 256x256 bonds) from an ncu capture of this kernel version (profiles/)
                "traffic": JACOBI_DRAM_BYTES_PER_LAUNCH,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one k_jacobi_grid launch "
                                  "at step 16 (full-size layer); the matrices stay in L2 otherwise",
                "work": "Golub-Van Loan SVD flops 4(4m^2n+8mn^2+9n^3) x4 (complex) per bond update",
                "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x median SM clock (of derived; "
                               + src + "; a DFMA probe measured 1.20 TFLOP/s)",
                "svd_ms_per_launch": svd_ms / n_layers,
                "svd_sweeps_last_step": {"fp64": [int(x) for x in sweeps[:, 0]],
                                         "fp32": [int(x) for x in sweeps[:, 1]]},
                "stage_ms_per_step": {"site": stage[0], "blocks_qr": stage[1], "theta": stage[2],
                                      "svd_fp64": stage[3], "svd_fp32": stage[7], "svd_precond": stage[8],
                                      "truncate": stage[4], "recover": stage[5], "readout": stage[6]}}

    if args.precision != "fp64" and stage[2] > 0:
        # the tcgen05 theta GEMM against the TF32 (or bf16) tensor peak: measured bf16 x the nominal
        # dense ratio (TF32 1.1 / bf16 2.25 PFLOP/s), or the fallback figure without the file
        bf16 = float(mp["bf16_tflops"]) if mp and "bf16_tflops" in mp else 1900.0
        tpeak = bf16 * (1.1 / 2.25) if args.precision in ("tf32x3", "tf32x1") else bf16
        tach = (fl_theta / K) / (stage[2] / 1e3) / 1e12
        roofline["theta_tensor"] = {
            "kernel": "k_tc_pack + k_tc_theta (tcgen05 3M complex GEMM, split pieces)", "bound": "tensor",
            "achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
            "work": "128 r^2 chi + 2048 r^2 per bond update (algorithmic, complex MAC = 8)",
            "peak_source": ("of measured: bf16 GEMM burst x 1.1/2.25" if mp else "of fallback: 1.9 PF bf16 x 1.1/2.25")
            if args.precision in ("tf32x3", "tf32x1") else ("of measured: bf16 GEMM burst" if mp else "of fallback")}

    # --- end to end through the C ABI: host inputs -> init (H2D) -> W+K steps -> history (D2H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2 = make(args.precision)
    e2.step(W + K)
    hist, tr = e2.read_history(0, W + K + 1)
    t1 = time.perf_counter()
    e2.destroy()
    h2d = 0
    for c in chains:
        h2d += c["rho0"].nbytes if c.get("rho0") is not None else 0
        h2d += (c["gates_q"].nbytes + c["gates_h"].nbytes) if c["N"] > 1 else 0
    h2d += sum(P.nbytes for Ps in mpos for P in Ps)
    d2h = hist.nbytes + tr.nbytes
    e2e = {"value": site_steps_per_step * (W + K) / (t1 - t0), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d / (W + K)), "d2h_bytes_per_step": int(d2h / (W + K)),
           "window": f"init + steps 0..{W + K} + history read, all timed"}
    path = "fp64" if args.precision == "fp64" else "fast"
    gpu_launches = K * (6 * LAUNCHES_PER_LAYER[path] + 5)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32 (tf32/bf16 TC) + f64",
           "data": "synthetic (seeded workload; PT-MPOs built on the host from the stated Ohmic baths)",
           "config": {"workload": w.name, "chains": n_chains, "N": [c["N"] for c in chains],
                      "dt": w.dt, "chi_max": w.chi_max, "kappa_max": w.kappa_max, "eps": w.eps,
                      "precision": args.precision, "window": f"steps {W}..{W + K} of {w.K}",
                      "l2": "flushed between timed steps (256 MiB write)",
                      "parallelism": f"{world} replicas" if world > 1 else "single GPU"},
           "clocks": clocks, "roofline": roofline, "e2e": e2e, "gpu_launches": gpu_launches,
           "algorithmic_tflops": (fl_svd + fl_other) / (total_ms / 1e3) / 1e12}
    if fp64 is not None:
        out["fp64_path"] = fp64
        out["speedup_vs_fp64_path"] = value / fp64["value"]
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, W, args.cpu_seconds, site_steps_per_step)
    if world > 1:
        dist.destroy_process_group()
    return out


# ------------------------------------------------------------------------ the oracle on the host
def cpu_baseline(w, warm, seconds, site_steps_per_step):
    """Time the FP64 oracle as it stands on the host cores: W untimed steps from t = 0, then as
    many steps as fit in about `seconds` (at least one)."""
    from oracle import problem as oprob, model, pttebd
    cis = oprob.build_inputs(w)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    total_steps = 0
    t_total = 0.0
    for ci in cis:
        m = pttebd.product_state(ci.rho0) if ci.init_mps is None else ci.init_mps.copy()
        for k in range(1, warm + 1):
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps)
        t0 = time.perf_counter()
        k = warm
        while k < w.K:
            k += 1
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps)
            total_steps += 1
            if time.perf_counter() - t0 > seconds / max(1, len(cis)):
                break
        t_total += time.perf_counter() - t0
        if len(cis) > 4 and t_total > seconds:
            break
    n_sites_done = total_steps * (site_steps_per_step / len(cis))
    return {"value": n_sites_done / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{total_steps} steps after {warm} warm-up steps of {w.name} "
                      f"(numpy/LAPACK, {cores} host threads available)"}


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
    # each "step" of the reference arm is one PT-TEBD step of the same trajectory (bounded: K steps)
    ms = []
    states = []
    for ci in cis:
        m = pttebd.product_state(ci.rho0) if ci.init_mps is None else ci.init_mps.copy()
        for k in range(1, W + 1):
            pttebd.pt_step(m, k, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps)
        states.append(m)
    t0 = time.perf_counter()
    for i in range(K):
        ts = time.perf_counter()
        for ci, m in zip(cis, states):
            pttebd.pt_step(m, W + i + 1, ci.gates_q, ci.gates_h, ci.pt, w.chi_max, w.eps)
        ms.append((time.perf_counter() - ts) * 1e3)
    t_all = time.perf_counter() - t0
    value = site_steps * K / t_all
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": t_all * 1e3 / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "impl": "reference",
            "data": "synthetic (seeded workload; PT-MPOs built by the oracle)",
            "config": {"workload": w.name, "chains": len(cis), "precision": "fp64 (numpy/LAPACK)",
                       "window": f"steps {W}..{W + K} of {w.K}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{K} steps after {W} warm-up steps of {w.name}"},
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
