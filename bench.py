#!/usr/bin/env python3
"""Benchmark: FP64-accurate dense solve throughput on one GB300.

Workload (default): dense nonsymmetric system, n = 16384, nrhs = 1, A i.i.d.
N(0,1), x_true i.i.d. U[-1,1], b = A x_true in FP64 (seeded, synthetic).  One
step = one whole mixed-precision solve through the C ABI (mp_gesv): FP64->FP32
conversion, low-precision LU with partial pivoting (default rung fp16x3: the
trailing updates as three fp16 tensor-core products, about FP32 accurate),
FP64 iterative refinement to a normwise backward error <= 1e-14 (and the FP64
fallback, if taken).  --workload chol|batched|adjoint times the secondary
workloads instead (one JSON line each, not the headline).

  value      = (2 n^3 / 3) * N_ranks / (max-over-ranks time per step), GFLOP/s,
               inputs resident in HBM (A is 2.1 GB, larger than L2).
  e2e        = the same metric through mp_gesv_host: host->device copy of A and
               b from pinned memory and device->host copy of x and the pivots
               inside the timed region.
  roofline   = the kernel class with the largest share of the step, timed
               with CUDA events on its own stream by the library's profiler
               during the timed steps.
  cpu_baseline = the CPU oracle (plain C, Algorithm 1 with an FP32 factor)
               timed on this host's cores on a smaller n of the same recipe.

--impl reference times the CPU oracle arm instead (the only reference that
exists for this method is the paper; its CPU restatement is the oracle).
Multi-GPU (torchrun): every rank solves its own independent system
(replicas; weak scaling), no collective on the data path.
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

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


# Nominal FP64 rate of GB300 (dense, CUDA cores): the residual's one FP64 FMA
# per 8-byte element of A runs against it rather than against HBM.
FP64_NOMINAL_TFLOPS = 1.25


def class_rooflines(prof, peaks, prec, n, nrhs):
    """Roofline of every timed kernel class of one solve: prof maps class ->
    (ms, launches, work) as the library's profiler reports it (work in flops
    for the factorization classes, in bytes for the triangular solves, the
    residual and the row exchanges).  Each class gets the bound that applies
    to it on GB300: the tensor pipe for the low-precision trailing update,
    FP32 CUDA cores for the panel and the FP32 updates, HBM for the
    triangular solves and row exchanges, and the FP64 pipe for the residual
    (2 n^2 nrhs FP64 flops per launch, one FMA per element of A and column)."""
    smx = peaks.get("sm_max_mhz", 2070.0)
    fp32 = 152 * 128 * 2 * smx * 1e6 / 1e12
    out = {}
    for cls, (ms, nl, work) in prof.items():
        if ms <= 0 or nl <= 0:
            continue
        if cls == "update" and prec in ("bf16", "fp16", "fp16x3", "e4m3"):
            bound, unit, peak, src = "tensor", "TFLOP/s", peaks.get("bf16_tflops_sustained", 1700.0), peaks["_source"]
            if prec == "fp16x3":
                work = 3.0 * work  # three products per k-step on the tensor pipe
            elif prec == "e4m3":
                peak = 2.0 * peak  # fp8 runs at twice the bf16 rate
            achieved = work / (ms * 1e-3) / 1e12
        elif cls in ("panel", "panelgemm", "trsm", "update"):
            bound, unit, peak, src = "alu", "TFLOP/s", fp32, "sm_max_mhz x 152 SM x 128 lanes x 2"
            achieved = work / (ms * 1e-3) / 1e12
        elif cls == "residual":
            bound, unit, peak, src = "alu", "TFLOP/s", FP64_NOMINAL_TFLOPS, "nominal FP64"
            achieved = nl * 2.0 * n * n * nrhs / (ms * 1e-3) / 1e12
        else:
            bound, unit, peak, src = "hbm", "GB/s", peaks.get("hbm_gbs", 6800.0), peaks["_source"]
            achieved = work / (ms * 1e-3) / 1e9
        out[cls] = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                    "frac": achieved / peak if peak else None, "ms": ms, "launches": nl, "peak_source": src}
    return out


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "-i", str(self.index),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "200"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist, device):
    """The largest of every rank's value (the slowest rank's time); the
    value itself when running alone."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(work_per_rank, world, ms_max):
    """Throughput of the whole job: every rank's work (replicas: the same
    amount each) divided by the slowest rank's time, in units of 1e9/s."""
    return work_per_rank * world / (ms_max * 1e-3) / 1e9


def cpu_oracle_rate(n, seed=0, reps=1):
    """Times the CPU oracle (Algorithm 1, FP32 factor, FP64 refinement) on n."""
    import oracle
    from paper_0808_2794_gb300 import inputs
    cores = oracle.set_threads(os.cpu_count() or 1)
    A, B, _ = inputs.dense_system(n, seed=seed)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        r = oracle.gesv_ir(A, B, factor_prec=32)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    return (2.0 * n ** 3 / 3.0) / best / 1e9, cores, best, r


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.ref_n
    for _ in range(args.warmup):
        cpu_oracle_rate(n)
    times = []
    for _ in range(args.steps):
        rate, cores, dt, r = cpu_oracle_rate(n)
        times.append(dt)
    t = float(np.mean(times))
    value = (2.0 * n ** 3 / 3.0) / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32-factor/f64-refine",
        "data": "synthetic", "config": {"workload": f"dense LU solve, A~N(0,1), nrhs=1, n={n} "
                                                     "(bounded CPU sample of the n=16384 recipe)",
                                         "n": n, "nrhs": 1},
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": f"one CPU-oracle solve (Algorithm 1, FP32 factor) per step at n={n}"},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "bwd_err": r["bwd"], "iter": r["iter"],
    }
    print(json.dumps(line), flush=True)
    return 0


METRIC = "FP64-accurate solve GFLOP/s (2n^3/3) at bwd err <= 1e-14 vs plain FP64 LU, 1 GB300"


def run_secondary(args):
    """Times one of the secondary workloads on one GPU (not the headline
    line): SPD Cholesky solve (n=4096, nrhs=4, prescribed kappa), the batch of
    4096 small systems, or the adjoint solve (n=2048, nrhs=8).  Prints one
    JSON line with the workload's own metric."""
    import ctypes
    import torch
    from paper_0808_2794_gb300 import inputs, solver
    torch.cuda.set_device(0)
    lib = solver.load()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    extra = {}
    if args.workload == "chol":
        n, nrhs = (args.n if args.n != 16384 else 4096), 4
        A, B, _ = inputs.conditioned_system(n, args.kappa, nrhs=nrhs, spd=True, seed=0)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        o = solver.default_opts(prec=args.prec, refine=args.refine)
        work = solver.workspace(lib.mp_posv_workspace_bytes(n, nrhs, ctypes.byref(o)))
        step = lambda: solver.posv(Ad, Bd, prec=args.prec, refine=args.refine, work=work)[1]
        flops = n ** 3 / 3.0
        metric = "FP64-accurate SPD solve GFLOP/s (n^3/3) at bwd err <= 1e-14, 1 GB300"
        cfg = {"workload": f"SPD Cholesky solve, A = U diag(s) U^T, kappa={args.kappa:g}, n={n}, nrhs={nrhs}"}
    elif args.workload == "batched":
        As, Bs, _ = inputs.batched_systems(count=4096, seed=0)
        dA = [torch.from_numpy(a).cuda() for a in As]
        dB = [torch.from_numpy(b).cuda() for b in Bs]
        prec = args.prec if args.prec in ("fp32", "bf16", "fp16") else "fp32"
        flops = sum(2.0 * a.shape[0] ** 3 / 3.0 for a in As)
        plan = solver.BatchedPlan(dA, dB, prec=prec)  # argument tables built once, outside the timing

        def step():
            plan.run()
            it, fl = plan.iter, plan.flags
            return {"iter_max": int(it.max()), "flags_or": int(np.bitwise_or.reduce(fl)),
                    "n_fallback": int(np.sum(it < 0))}
        metric = "batched FP64-accurate solve GFLOP/s (sum 2n^3/3), 1 GB300"
        cfg = {"workload": "4096 systems, n log-uniform [16,512], nrhs 1..4, A = N(0,1) + n I",
               "prec": prec}
    else:  # adjoint
        n, nrhs = (args.n if args.n != 16384 else 2048), 8
        A, B, Wt = inputs.adjoint_problem(n, nrhs, seed=0)
        Ad, Bd, Gd = (torch.from_numpy(x).cuda() for x in (A, B, Wt))
        o = solver.default_opts(prec=args.prec)
        work = solver.workspace(lib.mp_gesv_workspace_bytes(n, nrhs, ctypes.byref(o)))
        adj = solver.workspace(lib.mp_gesv_adjoint_workspace_bytes(n, ctypes.byref(o)))
        X, _, _ = solver.gesv(Ad, Bd, prec=args.prec, work=work)

        def step():
            return solver.gesv_adjoint(Ad, X, Gd, work, prec=args.prec, adj_work=adj)[2]
        flops = 8.0 * n * n  # reported as GB/s of the n x n FP64 Abar write
        metric = "adjoint solve (Bbar = A^-T G, Abar = -Bbar X^T) Abar write GB/s"
        cfg = {"workload": f"adjoint of X = A^-1 B, A = N(0,1) + sqrt(n) I, n={n}, nrhs={nrhs}"}
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches0 = solver.launch_count()
    ev[0].record(stream)
    out = None
    for _ in range(args.steps):
        out = step()
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.steps
    value = flops / (ms * 1e-3) / 1e9
    line = {"metric": metric, "value": value, "unit": "GFLOP/s" if args.workload != "adjoint" else "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": f"{args.prec}-factor/f64-refine", "data": "synthetic",
            "config": cfg, "gpu_launches": solver.launch_count() - launches0,
            "solve": {k: v for k, v in (out or {}).items() if not isinstance(v, list)}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--prec", default="fp16x3")
    ap.add_argument("--refine", default="classical", choices=["classical", "gmres", "auto"])
    ap.add_argument("--workload", default="lu", choices=["lu", "chol", "batched", "adjoint"],
                    help="lu: the headline dense solve; the others time the secondary "
                         "workloads (SPD Cholesky, batched small systems, adjoint solve)")
    ap.add_argument("--kappa", type=float, default=1e4, help="condition number for --workload chol")
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--ref-n", type=int, default=4096)
    ap.add_argument("--cpu-n", type=int, default=8192)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "lu":
        return run_secondary(args)

    import torch
    from paper_0808_2794_gb300 import inputs, solver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    else:
        dist = None

    def barrier():
        if dist is not None:
            dist.barrier()

    n, nrhs = args.n, args.nrhs
    A, B, Xtrue = inputs.dense_system(n, nrhs=nrhs, seed=rank)
    Ad = torch.from_numpy(np.asfortranarray(A)).cuda()
    Bd = torch.from_numpy(np.asfortranarray(B)).cuda()
    opts = dict(prec=args.prec, nb_outer=args.nb, refine=args.refine)
    lib = solver.load()
    import ctypes
    o = solver.default_opts(**opts)
    work = solver.workspace(lib.mp_gesv_workspace_bytes(n, nrhs, ctypes.byref(o)))
    stream = torch.cuda.current_stream()

    # warm-up; the first profiled step finds the dominant kernel class
    solver.profile_enable(solver.KERNEL_CLASSES)
    for i in range(args.warmup):
        X, ipiv, st = solver.gesv(Ad, Bd, work=work, **opts)
        if i == 0:
            torch.cuda.synchronize()
            prof0 = solver.profile_collect()
            solver.profile_enable(())
    torch.cuda.synchronize()
    dom = max(prof0, key=lambda c: prof0[c][0])

    # timed region
    solver.profile_enable([dom])
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = solver.launch_count()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        X, ipiv, st = solver.gesv(Ad, Bd, work=work, **opts)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = solver.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = solver.profile_collect()
    solver.profile_enable(())
    ms_step = max_over_ranks(ms_total / args.steps, dist, "cuda")
    flops = 2.0 * n ** 3 / 3.0
    value = whole_job_rate(flops, ws, ms_step)

    # correctness of the timed solves (library's own FP64 residual, and a check
    # of the final X through the residual entry point)
    worst_bwd = max(s["bwd_err"] for s in stats)
    R = solver.residual(Ad, X.reshape(n, -1), Bd.reshape(n, -1))
    anorm = float(torch.linalg.matrix_norm(Ad, ord=float("inf")))
    xn = float(X.abs().max())
    bn = float(Bd.abs().max())
    bwd_check = float(R.abs().max()) / (anorm * xn + bn)
    fwd_vs_true = float((X.reshape(n, -1).cpu() - torch.from_numpy(Xtrue)).abs().max() /
                        torch.from_numpy(Xtrue).abs().max())

    # roofline of the dominant kernel class
    peaks = load_peaks()
    ms_d, nl_d, work_d = prof[dom]
    if dom in ("update", "trsm", "panelgemm", "panel"):
        tensor = dom == "update" and args.prec in ("bf16", "fp16", "fp16x3")
        if tensor:
            bound, unit, peak = "tensor", "TFLOP/s", peaks.get("bf16_tflops_sustained", 1700.0)
        else:
            smx = peaks.get("sm_max_mhz", 2070.0)
            bound, unit = "alu", "TFLOP/s"
            peak = 152 * 128 * 2 * smx * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x clock
        achieved = work_d / (ms_d * 1e-3) / 1e12 if ms_d > 0 else 0.0
    else:
        bound, unit, peak = "hbm", "GB/s", peaks.get("hbm_gbs", 6800.0)
        achieved = work_d / (ms_d * 1e-3) / 1e9 if ms_d > 0 else 0.0
    share = ms_d / (ms_total) if ms_total > 0 else 0.0
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak if peak else None, "traffic": None,
                "kernel": dom, "share_of_step": share, "launches_timed": nl_d,
                "peak_source": peaks["_source"]}
    breakdown = {c: round(v[0] / max(1, 1), 3) for c, v in prof0.items()}
    by_class = class_rooflines(prof0, peaks, args.prec, n, nrhs)

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(np.asfortranarray(A)).pin_memory()
        hB = torch.from_numpy(np.asfortranarray(B)).pin_memory()
        hX = torch.zeros((nrhs, n), dtype=torch.float64).pin_memory()
        hP = torch.zeros(n, dtype=torch.int32).pin_memory()
        need = lib.mp_gesv_host_workspace_bytes(n, nrhs, ctypes.byref(o))
        wh = solver.workspace(need)
        st_ = solver.mp_stats()
        sp = ctypes.c_void_p(stream.cuda_stream)

        def host_solve():
            r = lib.mp_gesv_host(n, nrhs, hA.data_ptr(), n, hB.data_ptr(), n, hX.data_ptr(), n,
                                 hP.data_ptr(), wh.data_ptr(), wh.numel(), ctypes.byref(o),
                                 ctypes.byref(st_), sp)
            if r < 0:
                raise RuntimeError(solver.last_error())
        host_solve()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_solve()
        torch.cuda.synchronize()
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, dist, "cuda")
        e2e = {"value": whole_job_rate(flops, ws, e2e_ms), "unit": "GFLOP/s",
               "h2d_bytes_per_step": 8 * n * n + 8 * n * nrhs,
               "d2h_bytes_per_step": 8 * n * nrhs + 4 * n, "ms_per_step": e2e_ms}
        del wh

    cpu = None
    if rank == 0 and not args.no_cpu:
        rate, cores, dt, r = cpu_oracle_rate(args.cpu_n)
        cpu = {"value": rate, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
               "sample": f"one CPU-oracle solve (Algorithm 1: FP32 LU + FP64 refinement) at "
                         f"n={args.cpu_n} of the same recipe, {dt:.1f} s"}

    if rank == 0:
        last = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": f"{args.prec}-factor/f64-refine", "data": "synthetic",
            "config": {"workload": f"dense LU solve, A~N(0,1), x~U[-1,1], n={n}, nrhs={nrhs}",
                       "n": n, "nrhs": nrhs, "prec": args.prec, "nb_outer": args.nb,
                       "l2": "inputs larger than L2 (A is %.1f GB)" % (8 * n * n / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
            "solve": {"iter": last["iter"], "flags": last["flags"], "bwd_err": worst_bwd,
                      "bwd_check": bwd_check, "fwd_err_vs_xtrue": fwd_vs_true,
                      "ms_convert": last["ms_convert"], "ms_factor": last["ms_factor"],
                      "ms_refine": last["ms_refine"], "ms_fallback": last["ms_fallback"]},
            "kernel_ms_first_warmup": breakdown,
            "rooflines_by_class": by_class,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
