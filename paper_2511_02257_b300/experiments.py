"""Scheduler comparisons on the device (the paper's Sec. IV-B measurements).

For one synthetic workload and a device budget, every policy (naive
topological order, sibling, tree) is scheduled, planned and executed; the
line per policy reports the paper's figures -- peak memory of the model,
evictions, host<->device transfers (count and bytes, planned and actually
copied) -- and the measured time-to-solution of a full execution with the
leaves starting in pinned host memory.  Correlators of all policies are
compared bit for bit (each node's arithmetic is fixed; an eviction is a
copy), so a schedule can change the time but never a result.

  python -m paper_2511_02257_b300.experiments [--workload memory_pressure]
         [--precision tf32x3] [--evict lru] [--steps 2] [--budget-gib 24]

Prints one JSON line per policy, then a summary line with ratios to the
naive order.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="memory_pressure")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--evict", default="lru")
    ap.add_argument("--policies", default="naive,sibling,tree")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--budget-gib", type=float, default=None)
    ap.add_argument("--graph", type=int, default=1)
    args = ap.parse_args()

    import torch
    import paper_2511_02257_b300 as L
    import synth

    wl = synth.make_workload(args.workload)
    budget = int(args.budget_gib * 2 ** 30) if args.budget_gib is not None else wl.budget_bytes
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        leaves = list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))
    t_gen = time.perf_counter() - t0
    nd, _ = L.build_dag(wl, precision=args.precision, leaf_data_fn=lambda li: leaves[li])
    del leaves
    stream = torch.cuda.current_stream().cuda_stream
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
    ref = None
    rows = []
    for pol in args.policies.split(","):
        nd.schedule(pol, args.evict, budget)  # also releases the previous plan's memory
        ts = time.perf_counter()
        planned = nd.schedule(pol, args.evict, budget)
        t_sched = time.perf_counter() - ts
        nd.execute(stream)          # warm-up (graph capture, arena allocation)
        nd.wait(600000)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            nd.execute(stream)
            vals = nd.read_all_correlators()
            times.append(time.perf_counter() - t1)
        info = nd.exec_info()
        st = nd.stats()
        if ref is None:
            ref = vals.copy()
            same = True
        else:
            same = bool(np.array_equal(vals.view(np.float64), ref.view(np.float64)))
        row = {
            "workload": args.workload, "precision": args.precision, "policy": pol,
            "evict": args.evict, "budget_bytes": budget, "contractions": len(nd.order()),
            "schedule_ms": 1e3 * t_sched,
            "peak_paper_gib": planned["peak_paper"] / 2 ** 30,
            "peak_exec_gib": planned["peak_exec"] / 2 ** 30,
            "n_evict": planned["n_evict"], "n_h2d": planned["n_h2d"], "n_d2h": planned["n_d2h"],
            "h2d_gib": planned["h2d_bytes"] / 2 ** 30, "d2h_gib": planned["d2h_bytes"] / 2 ** 30,
            "copied_h2d_gib": info["copied_h2d"] / 2 ** 30,
            "copied_d2h_gib": info["copied_d2h"] / 2 ** 30,
            "measured_equals_planned": st == planned,
            "arena_gib": info["arena_bytes"] / 2 ** 30,
            "host_arena_gib": info["host_arena_bytes"] / 2 ** 30,
            "time_to_solution_s": min(times), "tflops": info["flops"] / min(times) / 1e12,
            "correlators_bit_identical_to_first_policy": same,
            "leaf_generation_s": t_gen,
        }
        rows.append(row)
        print(json.dumps(row), flush=True)
    base = rows[0]
    summary = {"summary": "ratios to %s" % base["policy"]}
    for r in rows[1:]:
        summary[r["policy"]] = {
            k: (base[k] / r[k] if r[k] else None)
            for k in ("peak_paper_gib", "n_evict", "h2d_gib", "time_to_solution_s")}
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
