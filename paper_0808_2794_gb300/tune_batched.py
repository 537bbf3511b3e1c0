"""Autotuner of the batched solver's tile schedule.

The batched solver factors each small system inside one CTA with a blocked
LU whose panel width (8 or 16 columns) trades the latency-bound pivoted
panel against the trailing update.  For every range of n of the built-in
schedule this script times, on the GPU, the systems of the config-4 batch
(4096 systems, n log-uniform in [16, 512], nrhs 1..4) that fall in the range,
once per candidate width (median of `reps` timed launches after one warm-up,
CUDA events), picks the fastest and writes the table to
csrc/batched_schedule.h (or --out), which the library compiles in.

    python -m paper_0808_2794_gb300.tune_batched [--out PATH] [--reps 5]
"""
from __future__ import annotations

import argparse
import datetime
import os

import numpy as np

CANDIDATES = (8, 16)
HERE = os.path.dirname(os.path.abspath(__file__))


def tune(count=4096, seed=0, reps=5, prec="fp32"):
    import torch

    from paper_0808_2794_gb300 import inputs, solver
    As, Bs, _ = inputs.batched_systems(count=count, seed=seed)
    ns = np.array([a.shape[0] for a in As])
    solver.set_batched_schedule(None)
    ranges = [nm for nm, _ in solver.batched_schedule()]
    rows = []
    lo = 0
    try:
        for nmax in ranges:
            idx = [i for i in range(count) if lo < ns[i] <= nmax]
            times = {}
            if idx:
                dA = [torch.from_numpy(As[i]).cuda() for i in idx]
                dB = [torch.from_numpy(Bs[i]).cuda() for i in idx]
                plan = solver.BatchedPlan(dA, dB, prec=prec)
                for nb in CANDIDATES:
                    solver.set_batched_schedule([(solver.BATCH_MAX_N, nb)])
                    plan.run()
                    ms = []
                    for _ in range(reps):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        torch.cuda.synchronize()
                        e0.record()
                        plan.run()
                        e1.record()
                        torch.cuda.synchronize()
                        ms.append(e0.elapsed_time(e1))
                    times[nb] = float(np.median(ms))
                best = min(times, key=times.get)
            else:
                best = 32
            rows.append((lo, nmax, len(idx), best, times))
            lo = nmax
    finally:
        solver.set_batched_schedule(None)
    return rows


def write_header(rows, path, gpu_name=""):
    stamp = datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%d")
    lines = ["// batched_schedule.h -- panel width of the batched solver's FP32 factorization",
             "// per range of n, as chosen by the autotuner (paper_0808_2794_gb300/tune_batched.py,",
             "// which times every candidate width on each range of the batch of 4096 systems",
             "// and rewrites this file).  Entry i covers kBatchedNmax[i-1] < n <= kBatchedNmax[i].",
             f"// Tuned {stamp} on {gpu_name or 'the GPU'}: milliseconds per launch of the range's systems",
             "// for panel widths " + ", ".join(str(c) for c in CANDIDATES) + ":"]
    for lo, hi, cnt, best, times in rows:
        t = ", ".join(f"{times[c]:.3f}" for c in CANDIDATES) if times else "no systems"
        lines.append(f"//   n in ({lo}, {hi}]: {cnt} systems: {t} -> {best}")
    lines += ["#pragma once",
              f"static const int kBatchedRanges = {len(rows)};",
              "static const int kBatchedNmax[kBatchedRanges] = {" + ", ".join(str(r[1]) for r in rows) + "};",
              "static const int kBatchedNb[kBatchedRanges] = {" + ", ".join(str(r[3]) for r in rows) + "};"]
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "csrc", "batched_schedule.h"))
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    import torch
    rows = tune(reps=args.reps)
    write_header(rows, args.out, torch.cuda.get_device_name(0))
    for r in rows:
        print(r)


if __name__ == "__main__":
    main()
