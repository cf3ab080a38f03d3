"""Benchmark: execute a correlation-function contraction DAG on B300.

One step = one execution of the whole DAG (every contraction of every
correlation function, in the tree scheduler's order, then the correlators),
i.e. all rows of the hot path over one synthetic workload.  The default
workload is the 200-function multi-meson DAG (Lt=64, N=64, ~2,100
contractions, FP64 path, unlimited budget).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` = algorithmic complex TFLOP/s
(8 real flops per complex multiply-add) with leaves already resident in
device memory; ``e2e`` = the same metric through the public C ABI with the
leaves loaded from the library's pinned host store every step and all
correlators read back to the host.  N>1 runs independent replicas (one DAG
per rank, weak scaling), or with ``--shard lt`` one DAG split over the ranks
along the time-slice axis (each rank executes its slices of every tensor
under its share of the budget; the root values are gathered at the end of
every end-to-end step; strong scaling).  ``--impl reference`` times the CPU
oracle on this host's cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

# DRAM bytes (read + write) per launch of the dominant FP64 kernel from one
# ncu capture of the default workload: 300 launches of k_contract_fp64<1,1>,
# the 64x64x64 x Lt 64 contraction that makes 86 % of its launches (reads
# its two 4.2 MB inputs once; the output stays in L2).  Algorithmic bytes of
# that launch: 12.58 MB.
TRAFFIC_PER_LAUNCH = 8.34e6
TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of 300 launches of "
                "k_contract_fp64<1,1> (64x64x64 x Lt 64, 86 % of the launches); algorithmic "
                "12.58 MB per such launch")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=8.0,
                    help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--workload", default="multi_meson")
    ap.add_argument("--policy", default="tree")
    ap.add_argument("--evict", default="lru")
    ap.add_argument("--precision", default="fp64")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: replay the whole execute as one CUDA graph")
    ap.add_argument("--window", type=int, default=64,
                    help="grouped-window size of the mixed path (0 = one contraction at a time)")
    ap.add_argument("--compare", default="tf32x3",
                    help="with --precision fp64: also time this mixed precision on the same "
                         "workload (grouped windows, graphs) and report its speedup and "
                         "error against the FP64 path; 'none' skips it")
    ap.add_argument("--autotune", type=int, default=1,
                    help="mixed precisions: pick window / fused-form limit / split policy by "
                         "timing every candidate on this DAG before the timed steps")
    ap.add_argument("--fused-max-n", type=int, default=64,
                    help="with --autotune 0: LQC_OPT_FUSED_MAX_N of the mixed path")
    ap.add_argument("--split-policy", type=int, default=0,
                    help="with --autotune 0: LQC_OPT_SPLIT_POLICY of the mixed path")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "lt"],
                    help="N>1: independent replicas, or one DAG split over the time slices")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def max_over_ranks(x: float, ws: int) -> float:
    """Largest value of x over the ranks (the job's time is its slowest
    rank's): a MAX all-reduce on the process group's device (CUDA under
    NCCL, the host under gloo)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws: int):
    """Sum over the ranks of a number or of a list of numbers, element by
    element (same device rule as max_over_ranks)."""
    many = isinstance(x, (list, tuple))
    if ws <= 1:
        return [float(v) for v in x] if many else float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in x] if many else [float(x)], dtype=torch.float64,
                     device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().tolist() if many else float(t.item())


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _blas_all_cores():
    """Context in which the oracle's BLAS pool spans every host core
    (threadpoolctl where installed; otherwise the BLAS default, which is
    one thread per core unless the environment limits it)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(limits=os.cpu_count(), user_api="blas")
    except ImportError:
        return contextlib.nullcontext()


def blas_threads():
    """Threads of the BLAS pool the oracle runs on."""
    try:
        from threadpoolctl import threadpool_info
    except ImportError:
        env = [os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")]
        env = [int(v) for v in env if v and v.isdigit()]
        return env[0] if env else len(os.sched_getaffinity(0))
    with _blas_all_cores():
        n = [p.get("num_threads", 0) for p in threadpool_info() if p.get("user_api") == "blas"]
    return max(n) if n else 1


def node_flops(od, u):
    nd = od.nodes[u]
    L, R = od.nodes[nd.left], od.nodes[nd.right]
    K = int(np.prod([L.extents[a] for a in nd.la], dtype=np.int64))
    M = int(np.prod(L.extents, dtype=np.int64)) // K
    N = int(np.prod(R.extents, dtype=np.int64)) // K
    return 8 * nd.lt * M * N * K


def oracle_sample(wl, seconds, rng_seed=0):
    """Time the CPU oracle on a random subset of correlation functions
    (their descendant closures), sized to about ``seconds`` of work, with
    the BLAS thread pool spanning every host core."""
    with _blas_all_cores():
        return _oracle_sample(wl, seconds, rng_seed)


def _oracle_sample(wl, seconds, rng_seed):
    from oracle import contract as C
    from oracle import dag as D
    import synth
    od, ids = D.build_from_workload(wl)
    cache = {}

    def lf(u):
        li = od.nodes[u].leaf_index
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    for u in od.used_leaves():   # input generation is not part of the timed work
        lf(u)
    rng = np.random.default_rng(rng_seed)
    roots = od.roots()
    perm = rng.permutation(len(roots))
    # calibrate on a few roots, then size the sample
    cal = [roots[i] for i in perm[:12]]
    t0 = time.perf_counter()
    C.evaluate(od, lf, cal)
    dt = max(time.perf_counter() - t0, 1e-3)
    calf = sum(node_flops(od, u) for u in C.closure(od, cal) if not od.nodes[u].is_leaf)
    rate = calf / dt
    chosen, fl = [], 0
    for i in perm:
        chosen.append(roots[i])
        fl = sum(node_flops(od, u) for u in C.closure(od, chosen) if not od.nodes[u].is_leaf)
        if fl >= rate * seconds:
            break
    t0 = time.perf_counter()
    C.evaluate(od, lf, chosen)
    el = time.perf_counter() - t0
    return fl, el, len(chosen), len(roots)


def run_reference(args, ws, rank):
    import synth
    if rank != 0:
        return
    wl = synth.make_workload(args.workload)
    per_step = args.ref_seconds
    oracle_sample(wl, min(1.0, per_step))  # warm caches
    total_f, total_t = 0, 0.0
    for w in range(args.warmup):
        oracle_sample(wl, per_step, rng_seed=100 + w)
    samples = []
    for k in range(args.steps):
        f, t, nr, nt = oracle_sample(wl, per_step, rng_seed=k)
        total_f += f
        total_t += t
        samples.append((nr, nt))
    v = total_f / total_t / 1e12
    cores = blas_threads()
    line = {
        "impl": "reference", "metric": "dag_complex_tflops", "value": v, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": args.workload, "lt": wl.lt, "nvec": wl.nvec,
                   "functions": len(wl.functions), "policy": args.policy,
                   "precision": "fp64", "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: %d of %d correlator trees (random, seeded), "
                                   "their descendant closures evaluated by the complex128 "
                                   "oracle (numpy tensordot per time slice)"
                                   % (samples[0][0], samples[0][1])},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def autotune(nd, stream):
    """Run the library's autotuner on a staged DAG; summary for the line."""
    t0 = time.perf_counter()
    entries = nd.autotune(stream, reps=2)
    return {"best": entries[0], "worst_ms": entries[-1]["ms"], "candidates": len(entries),
            "tune_s": time.perf_counter() - t0}


def shape_breakdown(wl, ids, times, n_exec):
    """Kernel ms per execution grouped by contraction shape (M, N, K per slice;
    K alone for a correlator), largest first."""
    ext = wl.stream_extents()
    shape = {}
    for j, rq in enumerate(wl.requests):
        le = ext[rq.left]
        k = int(np.prod([le[a] for a in rq.la]))
        m = int(np.prod(le)) // k
        n = int(np.prod(ext[rq.right])) // k
        shape[ids[len(wl.leaves) + j]] = "corr K=%d" % k if not ext[len(wl.leaves) + j] \
            else "%dx%dx%d" % (m, n, k)
    agg = {}
    for node, ms in times.items():
        key = shape.get(node, "?")
        c, t = agg.get(key, (0, 0.0))
        agg[key] = (c + 1, t + ms / max(n_exec, 1))
    top = sorted(agg.items(), key=lambda kv: -kv[1][1])[:8]
    return [{"shape": k, "count": c, "ms": round(t, 3)} for k, (c, t) in top]


def main():
    args = parse()
    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import torch.distributed as dist
    import paper_2511_02257_b300 as L
    import synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    from paper_2511_02257_b300 import shard as SH
    sharded = args.shard == "lt" and ws > 1
    shard = (rank, ws) if sharded else None
    wl = synth.make_workload(args.workload, seed=0 if sharded else rank)
    t_lo, t_hi = SH.lt_slices(wl.lt, ws)[rank] if sharded else (0, wl.lt)
    lt_share = (t_hi - t_lo) / wl.lt
    budget = SH.shard_budget(wl.budget_bytes, wl.lt, t_hi - t_lo) if sharded else \
        wl.budget_bytes

    def leaf_fn(li):      # whole leaves; build_dag keeps a shard's own slices
        return synth.leaf_data(wl, li)
    t0 = time.perf_counter()
    nd, ids = L.build_dag(wl, precision=args.precision, leaf_data_fn=leaf_fn, shard=shard)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    planned = nd.schedule(args.policy, args.evict, budget)
    t_sched = time.perf_counter() - t0
    stream = torch.cuda.current_stream().cuda_stream
    dev_stream = torch.cuda.current_stream()

    # ---- device-resident leaves: the kernel-level metric
    nd.stage_leaves(stream)
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
    nd.set_option(L.LQC_OPT_WINDOW, args.window)
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, args.fused_max_n)
    nd.set_option(L.LQC_OPT_SPLIT_POLICY, args.split_policy)
    tuned = None
    if args.precision != "fp64" and args.autotune:
        tuned = autotune(nd, stream)
    nd.set_option(L.LQC_OPT_TIMING, 1)
    for _ in range(args.warmup):
        nd.execute(stream)
    nd.wait()
    info0 = nd.exec_info()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(dev_stream)
        for _ in range(args.steps):
            nd.execute(stream)
        e1.record(dev_stream)
        torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    info1 = nd.exec_info()
    corr = nd.read_all_correlators()
    ms = max_over_ranks(ms, ws)
    flops_step = info1["flops"]
    # work of one step over all ranks: replicas each run a whole DAG; shards
    # together run one
    job_flops = sum_over_ranks(flops_step, ws)
    value = job_flops * args.steps / (ms * 1e-3) / 1e12
    # dominant kernel: the exterior contraction
    n_c = info1["n_contract"] - info0["n_contract"]
    ms_c = info1["ms_contract"] - info0["ms_contract"]
    fl_c = info1["flops_contract"] - info0["flops_contract"]
    ms_a = info1["ms_contract_all"] - info0["ms_contract_all"]
    achieved = fl_c / (ms_c * 1e-3) / 1e12 if ms_c > 0 else None
    breakdown = shape_breakdown(wl, ids, nd.kernel_times(), args.warmup + args.steps)
    probe = L.measure_fp64_peak()
    kernels = info1["n_kernels"]

    # ---- end to end: leaves from pinned host memory, correlators back to the host
    e2e = None
    if not args.no_e2e:
        nd.set_option(L.LQC_OPT_TIMING, 0)
        nd.unstage_leaves()
        nd.execute(stream)
        out = nd.read_all_correlators()
        if sharded:   # each root's full batch extent: the sum of its ranks' slices
            root_lts = [int(v) for v in sum_over_ranks([nd.node_info(r)["lt"]
                                                        for r in nd.roots()], ws)]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            nd.execute(stream)
            nd.read_all_correlators(out)
            if sharded:
                full = SH.gather_correlators(out, root_lts, ws, device="cuda")
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e, ws)
        st = nd.stats()
        e2e = {"value": job_flops * args.steps / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": st["h2d_bytes"],
               "d2h_bytes_per_step": st["d2h_bytes"] + out.nbytes,
               "ms_per_step": 1e3 * t_e2e / args.steps}
        if sharded:
            e2e["gathered_values"] = int(np.asarray(full).size)

    # ---- the precision form on the same workload, against this FP64 run
    pform = None
    if args.precision == "fp64" and args.compare != "none":
        md, _ = L.build_dag(wl, precision=args.compare, leaf_data_fn=leaf_fn, shard=shard)
        mplanned = md.schedule(args.policy, args.evict, budget)
        md.stage_leaves(stream)
        md.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
        md.set_option(L.LQC_OPT_WINDOW, args.window)
        md.set_option(L.LQC_OPT_FUSED_MAX_N, args.fused_max_n)
        md.set_option(L.LQC_OPT_SPLIT_POLICY, args.split_policy)
        mtuned = autotune(md, stream) if args.autotune else None
        for _ in range(args.warmup):
            md.execute(stream)
        torch.cuda.synchronize()
        e0.record(dev_stream)
        for _ in range(args.steps):
            md.execute(stream)
        e1.record(dev_stream)
        torch.cuda.synchronize()
        mms = e0.elapsed_time(e1) / args.steps
        mv = md.read_all_correlators()
        err = np.linalg.norm(mv - corr, axis=-1) / np.linalg.norm(corr, axis=-1)
        mst = md.exec_info()
        pform = {"precision": args.compare, "autotune": mtuned,
                 "time_to_solution_s": mms / 1e3, "tflops": flops_step / (mms * 1e-3) / 1e12,
                 "speedup_vs_fp64": (ms / args.steps) / mms,
                 "err_vs_fp64_max": float(err.max()), "err_vs_fp64_median": float(np.median(err)),
                 "kernels_per_step": mst["n_kernels"],
                 "peak_paper_bytes": mplanned["peak_paper"]}
        md.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        f, t, nr, nt = oracle_sample(wl, 20.0)
        cpu = {"value": f / t / 1e12, "unit": "TFLOP/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": "%d of %d correlator trees (random, seeded) with their descendant "
                         "closures, %.2f GFLOP in %.1f s" % (nr, nt, f / 1e9, t)}

    from paper_2511_02257_b300.roofline import (FP64_NOMINAL_TFLOPS, TENSOR_RATIO,
                                                 dag_roofline_for, measured_peaks)
    droof = dag_roofline_for(wl, ids, args.precision, ms / args.steps / 1e3)
    if sharded:   # this rank's slices: every contraction's work and bytes scale with them
        for k in ("time_s", "compute_bound_s", "memory_bound_s", "flops"):
            droof[k] *= lt_share
        droof["frac"] = droof["time_s"] / (ms / args.steps / 1e3)
    if pform:
        pform["dag_roofline"] = dag_roofline_for(wl, ids, args.compare,
                                                 pform["time_to_solution_s"])
    if args.precision == "fp64":
        roofline = {"kernel": "k_contract_fp64", "bound": "alu", "achieved": achieved,
                    "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_NOMINAL_TFLOPS if achieved else None,
                    "peak_source": "nominal B300 FP64 rate (profiling recipe table)",
                    "fma_probe_tflops": probe,
                    "frac_of_probe": achieved / probe if achieved else None,
                    "traffic": TRAFFIC_PER_LAUNCH, "traffic_note": TRAFFIC_NOTE}
    else:
        # split products: 3 real-embedded GEMMs per complex contraction, each
        # 8 real flops per complex multiply-add (windows time whole levels,
        # so the kernel time is that of the grouped launches)
        peaks, src = measured_peaks()
        peak = peaks["bf16_tflops"] * TENSOR_RATIO[args.precision]
        ach = 3 * achieved if achieved else None
        roofline = {"kernel": "k_gemm_split3", "bound": "tensor", "achieved": ach,
                    "peak": peak, "unit": "TFLOP/s", "frac": ach / peak if ach else None,
                    "peak_source": "%s BF16 GEMM peak x nominal %s/BF16 ratio %.3f"
                                   % (src, args.precision[:4].upper(),
                                      TENSOR_RATIO[args.precision]),
                    "algorithmic_complex_tflops": achieved, "traffic": None}
    roofline.update({"launches": n_c, "kernel_ms_per_step": ms_c / args.steps,
                     "contract_all_ms_per_step": ms_a / args.steps})

    if rank == 0:
        line = {
            "metric": "dag_complex_tflops", "value": value, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None, "dtype": "c128" if args.precision == "fp64" else "c64",
            "data": "synthetic",
            "config": {"workload": args.workload, "lt": wl.lt, "nvec": wl.nvec,
                       "functions": len(wl.functions), "contractions": len(nd.order()),
                       "policy": args.policy, "evict": args.evict, "budget_bytes": budget,
                       "precision": args.precision, "cuda_graph": bool(args.graph),
                       "window": (tuned["best"]["window"] if tuned else args.window)
                                 if args.precision != "fp64" else 0,
                       "autotune": tuned,
                       "fused_max_n": (tuned["best"]["fused_max_n"] if tuned else args.fused_max_n),
                       "split_policy": (tuned["best"]["split_policy"] if tuned
                                        else args.split_policy),
                       "parallelism": ("lt-shard" if sharded else "replicas") if ws > 1
                                      else "single",
                       "l2": "inputs larger than L2 (leaves %.2f GB, arena %.2f GB)"
                             % (sum(nd.node_info(i)["size"] for i in range(len(wl.leaves))) / 1e9,
                                info1["arena_bytes"] / 1e9)},
            "time_to_solution_s": ms / args.steps / 1e3,
            "flops_per_step": flops_step,
            "peak_paper_bytes": planned["peak_paper"], "peak_exec_bytes": planned["peak_exec"],
            "n_evict": planned["n_evict"], "h2d_gb_per_step": planned["h2d_bytes"] / 1e9,
            "d2h_gb_per_step": planned["d2h_bytes"] / 1e9,
            "schedule_ms": 1e3 * t_sched, "dag_build_s": t_build,
            "roofline": roofline,
            "kernel_ms_by_shape": breakdown,
            "dag_roofline": droof,
            "precision_form": pform,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": kernels * args.steps,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
