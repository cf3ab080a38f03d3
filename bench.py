"""Benchmark: execute a correlation-function contraction DAG on B300.

One step = one execution of the whole DAG (every contraction of every
correlation function, in the tree scheduler's order, then the correlators),
i.e. all rows of the hot path over one synthetic workload.  The default is
the batched workload in the mixed precision form: 50 independent
multi-meson DAGs of uneven N (32..256) and Lt (16..128), about 18k
contractions, complex64 storage, split TF32x3 tensor-core products with FP32
accumulation and FP64 correlator sums, grouped windows in a CUDA graph with
the options the library's autotuner picks, under a 48 GiB budget.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched] [--precision tf32x3] [--sub memory_pressure,baryon]

Prints one JSON line (rank 0).  ``value`` = algorithmic complex TFLOP/s
(8 real flops per complex multiply-add) with the leaves already resident in
device memory; ``e2e`` = the same metric through the public C ABI with the
leaves loaded from the library's pinned host store every step and all
correlators read back to the host.  The line also carries:

  fp64_arm      the plain FP64 path (one launch per contraction, CUDA graph)
                on the same DAG and leaves: its time, and the mixed form's
                speedup and per-correlator error against it
  roofline      the dominant kernel (the fused split-3 GEMM) from CUDA events
                recorded between the launches of every window level
  dag_roofline  sum over contractions of max(compute, HBM) bound, and the
                host link bound of the plan's transfers
  sub           the same figures for the memory-pressure workload (Lt 128,
                N 128, 24 GiB budget; with the naive order's evicting run
                against the host link) and the baryon workload

N>1 runs independent replicas (one DAG per rank, weak scaling), or with
``--shard lt`` one DAG split over the ranks along the time-slice axis
(strong scaling); sub-records and the FP64 arm run at N=1 only.
``--impl reference`` times the CPU oracle on this host's cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import contextlib
import hashlib
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

# DRAM bytes per launch of the fused split-3 GEMM from an ncu capture, with
# the hash of the kernel source it was taken on (None until captured: the
# figure is reported only while the source is unchanged).
GEMM_TRAFFIC = {
    "bytes_per_flop": 62.61e9 / 5.099e12, "source_sha16": "ebde4106fbdf049b",
    "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the 39 grouped fused-GEMM "
            "launches (CTA-pair and one-CTA) of one step of the batched workload with 8 parts "
            "(40.09 + 22.52 GB for 5.099e12 algorithmic flops, 71.5 GB of algorithmic operand + "
            "output bytes), scaled by the flops of a launch of this run"}
# DRAM bytes per launch of the dominant FP64 kernel (k_contract_fp64<4,4>),
# same convention.
FP64_TRAFFIC = {
    "bytes_per_launch": 97.88e6, "source_sha16": "fffc41101ef2c194",
    "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of the 239 launches of "
            "k_contract_fp64<4,4> (the instantiation with the largest share of K1 time) in "
            "one step of the multi-meson workload"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=8.0,
                    help="--impl reference: seconds of oracle work per step")
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--workload-kw", default="{}",
                    help="JSON overrides of the workload generator (smaller cases for profiling)")
    ap.add_argument("--policy", default="tree")
    ap.add_argument("--evict", default="lru")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--graph", type=int, default=1,
                    help="1: replay the whole execute as one CUDA graph")
    ap.add_argument("--autotune", type=int, default=1,
                    help="mixed precisions: pick window / fused-form limit / split policy by "
                         "timing every candidate on this DAG before the timed steps")
    ap.add_argument("--window", type=int, default=512,
                    help="with --autotune 0: grouped-window size of the mixed path")
    ap.add_argument("--fused-max-n", type=int, default=1 << 30,
                    help="with --autotune 0: LQC_OPT_FUSED_MAX_N of the mixed path")
    ap.add_argument("--split-policy", type=int, default=1,
                    help="with --autotune 0: LQC_OPT_SPLIT_POLICY of the mixed path")
    ap.add_argument("--fused-kernel", type=int, default=2,
                    help="LQC_OPT_FUSED_KERNEL of the mixed path (0: one CTA per tile, "
                         "1: A in tensor memory, 2: CTA pairs on 256-row tiles)")
    ap.add_argument("--fp64-arm", type=int, default=1,
                    help="executions of the FP64 path on the same DAG (0: skip)")
    ap.add_argument("--sub", default="memory_pressure,baryon",
                    help="comma-separated sub-record workloads ('none' to skip)")
    ap.add_argument("--shard", default="replicas", choices=["replicas", "lt"],
                    help="N>1: independent replicas, or one DAG split over the time slices")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------ ranks
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


# ------------------------------------------------------------------ CPU oracle
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
    rng = np.random.default_rng(rng_seed)
    roots = od.roots()
    perm = rng.permutation(len(roots))
    # calibrate on a few roots, then size the sample; input generation is
    # not part of the timed work
    cal = [roots[i] for i in perm[:12]]
    for u in C.closure(od, cal):
        if od.nodes[u].is_leaf:
            lf(u)
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
    for u in C.closure(od, chosen):
        if od.nodes[u].is_leaf:
            lf(u)
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
                   "precision": "fp64 (complex128 oracle)", "parallelism": "replicas"},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": "each step: %d of %d correlator trees (random, seeded), "
                                   "their descendant closures evaluated by the complex128 "
                                   "oracle (numpy tensordot per time slice)"
                                   % (samples[0][0], samples[0][1])},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ device helpers
def gen_leaves(wl):
    """Every leaf's complex128 data (seeded), generated on all host cores."""
    import synth
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))


def source_sha16(name, start=None, end=None):
    """First 16 hex digits of the SHA-256 of a kernel source, or of its text
    from the first line starting with `start` to the line starting with `end`
    (the code a captured kernel is built from, so that edits elsewhere in the
    file keep its ncu figures)."""
    with open(os.path.join(HERE, "paper_2511_02257_b300", "csrc", name), "rb") as f:
        text = f.read()
    if start is not None:
        text = text[text.index(start.encode()):text.index(end.encode())]
    return hashlib.sha256(text).hexdigest()[:16]


# the fused GEMM's code in kernels_mixed.cu: its helpers and kernels up to the
# A-in-TMEM form (the split-K sums, reorders and correlators come after it)
GEMM_SOURCE = ("kernels_mixed.cu", "#include", "// " + "-" * 60 + " K4t: A in TMEM")


def link_bandwidth(nbytes=1 << 30, reps=3):
    """Pinned host <-> device copy bandwidth (GB/s), one cudaMemcpyAsync per
    copy, best of `reps`, CUDA events on the copying stream."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    out = {}
    for name, fn in (("h2d_gbs", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h_gbs", lambda: h.copy_(d, non_blocking=True))):
        best = 0.0
        fn()
        torch.cuda.synchronize()
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        out[name] = best
    del h, d
    torch.cuda.empty_cache()
    out["bytes_per_copy"] = nbytes
    return out


def set_mixed_options(L, nd, args):
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
    nd.set_option(L.LQC_OPT_WINDOW, args.window)
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, args.fused_max_n)
    nd.set_option(L.LQC_OPT_SPLIT_POLICY, args.split_policy)
    nd.set_option(L.LQC_OPT_FUSED_KERNEL, args.fused_kernel)


def autotune(nd, stream, reps=1):
    """Run the library's autotuner on a scheduled DAG; summary for the line."""
    t0 = time.perf_counter()
    entries = nd.autotune(stream, reps=reps)
    return {"best": entries[0], "worst_ms": entries[-1]["ms"], "candidates": len(entries),
            "tune_s": time.perf_counter() - t0}


def timed_executes(nd, stream, steps, warmup, clocks=None):
    """Device time (ms) of `steps` back-to-back executes after `warmup`,
    CUDA events on the launching stream with a synchronize on both sides."""
    import torch
    dev_stream = torch.cuda.current_stream()   # `stream` is its handle
    for _ in range(warmup):
        nd.execute(stream)
    nd.wait()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ctx = clocks if clocks is not None else contextlib.nullcontext()
    with ctx:
        e0.record(dev_stream)
        for _ in range(steps):
            nd.execute(stream)
        e1.record(dev_stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def per_root_error(v, ref, offs):
    return np.array([np.linalg.norm(v[offs[i]:offs[i + 1]] - ref[offs[i]:offs[i + 1]]) /
                     np.linalg.norm(ref[offs[i]:offs[i + 1]]) for i in range(len(offs) - 1)])


def root_offsets(nd):
    lts = [nd.node_info(r)["lt"] for r in nd.roots()]
    return np.concatenate([[0], np.cumsum(lts)]).astype(np.int64)


def gemm_roofline(L, info, precision, steps_timed):
    """The fused (or plane) split-3 GEMM's achieved tensor rate from the
    per-kind CUDA events of the window levels."""
    from paper_2511_02257_b300.roofline import TENSOR_RATIO, measured_peaks
    kinds = info["ms_kind"]
    ms = kinds["gemm_fused"] + kinds["gemm_planes"]
    n = info["n_kind"]["gemm_fused"] + info["n_kind"]["gemm_planes"]
    fl = info["flops_gemm"]
    peaks, src = measured_peaks()
    ratio = TENSOR_RATIO[precision]
    peak = peaks["bf16_tflops"] * ratio
    peak_s = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * ratio
    ach = 3 * fl / (ms * 1e-3) / 1e12 if ms > 0 else None
    traffic = None
    if GEMM_TRAFFIC and GEMM_TRAFFIC.get("source_sha16") == source_sha16(*GEMM_SOURCE) \
            and n:
        traffic = GEMM_TRAFFIC["bytes_per_flop"] * fl / n
    total = sum(kinds.values())
    return {"kernel": "k_gemm_split3<tf32, fused>" if precision == "tf32x3"
            else "k_gemm_split3<bf16, planes>",
            "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if ach else None,
            "peak_source": "%s BF16 GEMM burst peak x nominal %s/BF16 ratio %.3f (of measured)"
                           % (src, precision[:4].upper(), ratio),
            "peak_sustained": peak_s, "frac_of_sustained": ach / peak_s if ach else None,
            "algorithmic_complex_tflops": ach / 3 if ach else None,
            "work": "3 real-embedded tensor-core products per complex multiply-add, 8 flops each",
            "launches": n, "launches_per_step": n / max(steps_timed, 1),
            "kernel_ms_per_step": ms / max(steps_timed, 1),
            "share_of_timed_kernels": ms / total if total else None,
            "traffic": traffic,
            "traffic_note": GEMM_TRAFFIC.get("note") if traffic else
            "no ncu DRAM capture of this kernel source"}


def kind_breakdown(info, steps):
    return {k: round(v / max(steps, 1), 4) for k, v in info["ms_kind"].items() if v > 0}


def fp64_arm(L, wl, leaves, policy, evict, budget, stream, mixed_vals, offs, executions,
             staged=True):
    """The plain FP64 path on the same DAG: one launch per contraction
    (captured in a CUDA graph), leaves resident unless `staged` is false.
    The program is built before the timed executions."""
    import torch
    nd, _ = L.build_dag(wl, precision="fp64", leaf_data_fn=lambda li: leaves[li])
    nd.schedule(policy, evict, budget)
    if staged:
        nd.stage_leaves(stream)
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    nd.prepare(stream)
    ms = timed_executes(nd, stream, executions, 0)
    vals = nd.read_all_correlators().reshape(-1)
    info = nd.exec_info()
    nd.close()
    del nd
    torch.cuda.empty_cache()
    err = per_root_error(mixed_vals, vals, offs)
    t = ms / executions / 1e3
    return {"executions": executions, "time_to_solution_s": t,
            "tflops": info["flops"] / t / 1e12, "kernels_per_execution": info["n_kernels"],
            "leaves": "device" if staged else "pinned host",
            "err_vs_fp64_max": float(err.max()), "err_vs_fp64_median": float(np.median(err)),
            "correlators": int(len(err))}, vals


def mixed_form(L, wl, leaves, args, precision, policy, budget, stream, steps, warmup,
               clocks=None, staged=True):
    """Build, schedule and (optionally) autotune the mixed form; time
    `steps` executes.  Returns (nd, ids, record)."""
    from paper_2511_02257_b300.roofline import dag_roofline_for
    t0 = time.perf_counter()
    nd, ids = L.build_dag(wl, precision=precision, leaf_data_fn=lambda li: leaves[li])
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    planned = nd.schedule(policy, args.evict, budget)
    t_sched = time.perf_counter() - t0
    if staged:
        nd.stage_leaves(stream)
    set_mixed_options(L, nd, args)
    tuned = autotune(nd, stream) if args.autotune else None
    nd.set_option(L.LQC_OPT_TIMING, 1)
    nd.prepare(stream)
    ms = timed_executes(nd, stream, steps, warmup, clocks)
    info = nd.exec_info()
    t = ms / steps / 1e3
    rec = {"precision": precision, "policy": policy, "budget_bytes": budget,
           "leaves": "device" if staged else "pinned host",
           "contractions": len(nd.order()), "steps": steps, "warmup": warmup,
           "time_to_solution_s": t, "tflops": info["flops"] / t / 1e12,
           "flops_per_step": info["flops"], "kernels_per_step": info["n_kernels"],
           "autotune": tuned,
           "options": {"window": tuned["best"]["window"] if tuned else args.window,
                       "fused_max_n": tuned["best"]["fused_max_n"] if tuned else args.fused_max_n,
                       "split_policy": tuned["best"]["split_policy"] if tuned
                       else args.split_policy, "cuda_graph": bool(args.graph),
                       "fused_kernel": tuned["best"]["fused_kernel"] if tuned
                       else args.fused_kernel},
           "peak_paper_bytes": planned["peak_paper"], "peak_exec_bytes": planned["peak_exec"],
           "n_evict": planned["n_evict"], "h2d_bytes_planned": planned["h2d_bytes"],
           "d2h_bytes_planned": planned["d2h_bytes"],
           "arena_bytes": info["arena_bytes"], "resident_peak_bytes": info["resident_peak_bytes"],
           "schedule_ms": 1e3 * t_sched, "dag_build_s": t_build,
           "roofline": gemm_roofline(L, info, precision, warmup + steps),
           "kernel_ms_per_step_by_kind": kind_breakdown(info, warmup + steps),
           "dag_roofline": dag_roofline_for(wl, ids, precision, t)}
    return nd, ids, rec


def link_record(planned_h2d, planned_d2h, t, link):
    """The host-link bound of a plan's transfers: both directions overlap
    (full duplex), so the bound is the slower direction's copy time."""
    th = planned_h2d / (link["h2d_gbs"] * 1e9)
    td = planned_d2h / (link["d2h_gbs"] * 1e9)
    bound = max(th, td)
    return {"h2d_bytes": planned_h2d, "d2h_bytes": planned_d2h, "bound_s": bound,
            "frac": bound / t if t else None, "h2d_gbs": link["h2d_gbs"],
            "d2h_gbs": link["d2h_gbs"]}


def sub_record(L, name, args, stream, link):
    """Mixed form (tuned, leaves resident), the same from pinned host, and
    the FP64 arm on one workload; memory_pressure adds the naive order's
    evicting run against the host link."""
    import torch
    import synth
    wl = synth.make_workload(name)
    t0 = time.perf_counter()
    leaves = gen_leaves(wl)
    t_gen = time.perf_counter() - t0
    steps, warmup = 3, 2
    nd, ids, rec = mixed_form(L, wl, leaves, args, args.precision, args.policy,
                              wl.budget_bytes, stream, steps, warmup)
    rec["workload"] = name
    rec["leaf_generation_s"] = t_gen
    mixed = nd.read_all_correlators().reshape(-1)
    offs = root_offsets(nd)
    # the same plan with every leaf loaded from pinned host inside the budget
    nd.unstage_leaves()
    nd.set_option(L.LQC_OPT_TIMING, 0)
    nd.prepare(stream)
    ms = timed_executes(nd, stream, 2, 1)
    st = nd.stats()
    th = ms / 2 / 1e3
    rec["host_leaves"] = {"time_to_solution_s": th, "h2d_bytes": st["h2d_bytes"],
                          "link": link_record(st["h2d_bytes"], st["d2h_bytes"], th, link)}
    nd.close()
    del nd
    torch.cuda.empty_cache()
    if args.fp64_arm:
        arm, _ = fp64_arm(L, wl, leaves, args.policy, args.evict, wl.budget_bytes, stream,
                          mixed, offs, 1, staged=False)
        arm["speedup_of_mixed"] = arm["time_to_solution_s"] / rec["time_to_solution_s"]
        rec["fp64_arm"] = arm
    if name == "memory_pressure":
        # the naive topological order under the same budget: evicts, and the
        # host link bounds it
        nn, _ = L.build_dag(wl, precision=args.precision, leaf_data_fn=lambda li: leaves[li])
        pl = nn.schedule("naive", args.evict, wl.budget_bytes)
        set_mixed_options(L, nn, args)
        nn.prepare(stream)
        ms = timed_executes(nn, stream, 1, 0)
        tn = ms / 1e3
        cnt = nn.stats()
        ninfo = nn.exec_info()
        v = nn.read_all_correlators().reshape(-1)
        rec["naive_order"] = {
            "time_to_solution_s": tn, "n_evict": cnt["n_evict"],
            "peak_paper_bytes": pl["peak_paper"], "peak_exec_bytes": pl["peak_exec"],
            "h2d_bytes": cnt["h2d_bytes"], "d2h_bytes": cnt["d2h_bytes"],
            "stats_equal_plan": cnt == pl,
            "arena_bytes": ninfo["arena_bytes"], "budget_bytes": wl.budget_bytes,
            "extra_placement_moves": {k: ninfo[k] for k in ("extra_evictions", "extra_h2d_bytes",
                                                            "extra_d2h_bytes")},
            "correlators_bit_identical_to_tree_order": bool(np.array_equal(
                v.view(np.float64), mixed.view(np.float64))),
            "link": link_record(cnt["h2d_bytes"], cnt["d2h_bytes"], tn, link),
            "tree_order_speedup": tn / rec["host_leaves"]["time_to_solution_s"]}
        nn.close()
        del nn
        torch.cuda.empty_cache()
    del leaves
    return rec


# ------------------------------------------------------------------ main
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
    from paper_2511_02257_b300.roofline import FP64_NOMINAL_TFLOPS, dag_roofline_for
    sharded = args.shard == "lt" and ws > 1
    shard = (rank, ws) if sharded else None
    wl = synth.make_workload(args.workload, seed=0 if sharded else rank,
                             **json.loads(args.workload_kw))
    t_lo, t_hi = SH.lt_slices(wl.lt, ws)[rank] if sharded else (0, wl.lt)
    lt_share = (t_hi - t_lo) / wl.lt
    budget = SH.shard_budget(wl.budget_bytes, wl.lt, t_hi - t_lo) if sharded else \
        wl.budget_bytes
    mixed = args.precision != "fp64"
    t0 = time.perf_counter()
    leaves = gen_leaves(wl)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream().cuda_stream
    dev_stream = torch.cuda.current_stream()

    # ---- device-resident leaves: the kernel-level metric
    t0 = time.perf_counter()
    nd, ids = L.build_dag(wl, precision=args.precision, leaf_data_fn=lambda li: leaves[li],
                          shard=shard)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    planned = nd.schedule(args.policy, args.evict, budget)
    t_sched = time.perf_counter() - t0
    nd.stage_leaves(stream)
    tuned = None
    if mixed:
        set_mixed_options(L, nd, args)
        if args.autotune:
            tuned = autotune(nd, stream)
    else:
        nd.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
    nd.set_option(L.LQC_OPT_TIMING, 1)
    nd.prepare(stream)
    for _ in range(args.warmup):
        nd.execute(stream)
    nd.wait()
    info0 = nd.exec_info()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("timed")
        e0.record(dev_stream)
        for _ in range(args.steps):
            nd.execute(stream)
        e1.record(dev_stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1)
    info1 = nd.exec_info()
    corr = nd.read_all_correlators().reshape(-1)
    offs = root_offsets(nd)
    ms = max_over_ranks(ms, ws)
    flops_step = info1["flops"]
    job_flops = sum_over_ranks(flops_step, ws)
    value = job_flops * args.steps / (ms * 1e-3) / 1e12
    t_step = ms / args.steps / 1e3
    kernels = info1["n_kernels"]
    nsteps = args.warmup + args.steps   # timing covers warm-up and timed steps

    # ---- the dominant kernel's roofline
    if mixed:
        roofline = gemm_roofline(L, info1, args.precision, nsteps)
    else:
        n_c = info1["n_contract"] - info0["n_contract"]
        ms_c = info1["ms_contract"] - info0["ms_contract"]
        fl_c = info1["flops_contract"] - info0["flops_contract"]
        ach = fl_c / (ms_c * 1e-3) / 1e12 if ms_c > 0 else None
        probe = L.measure_fp64_peak()
        traffic = None
        if FP64_TRAFFIC and FP64_TRAFFIC.get("source_sha16") == source_sha16("kernels_fp64.cu"):
            traffic = FP64_TRAFFIC["bytes_per_launch"]
        roofline = {"kernel": "k_contract_fp64", "bound": "alu", "achieved": ach,
                    "peak": probe, "unit": "TFLOP/s", "frac": ach / probe if ach else None,
                    "peak_source": "live FP64 FMA probe on every SM (register-resident FMA "
                                   "chains, this run); nominal %.2f" % FP64_NOMINAL_TFLOPS,
                    "frac_of_nominal": ach / FP64_NOMINAL_TFLOPS if ach else None,
                    "launches": n_c, "kernel_ms_per_step": ms_c / args.steps,
                    "traffic": traffic,
                    "traffic_note": FP64_TRAFFIC["note"] if traffic else
                    "no ncu DRAM capture of this kernel source"}

    # ---- host link
    link = link_bandwidth()

    # ---- end to end: leaves from pinned host memory, correlators back to the host
    e2e = None
    counted_equal = None
    if not args.no_e2e:
        nd.set_option(L.LQC_OPT_TIMING, 0)
        nd.unstage_leaves()
        nd.prepare(stream)
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
        counted_equal = st == planned   # leaves from the host: every plan copy is issued
        e2e = {"value": job_flops * args.steps / t_e2e / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": st["h2d_bytes"],
               "d2h_bytes_per_step": st["d2h_bytes"] + out.nbytes,
               "ms_per_step": 1e3 * t_e2e / args.steps,
               "link": link_record(st["h2d_bytes"], st["d2h_bytes"] + out.nbytes,
                                   t_e2e / args.steps, link)}
        if sharded:
            e2e["gathered_values"] = int(np.asarray(full).size)
    if not args.no_e2e and not sharded:
        # the same with new leaf data every step: each leaf's complex128 values
        # go through the library's host pass (normalisation and conversion into
        # the pinned store) before the execute; the exponents stay, so the
        # program and its graph are reused
        nl = len(wl.leaves)
        used = [i for i in range(nl) if nd.node_info(ids[i])["size"] > 0]
        k_new = min(args.steps, 3)
        p0 = nd.exec_info()["n_programs"]
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_host = 0.0
        for _ in range(k_new):
            th = time.perf_counter()
            for i in used:
                nd.set_leaf_data(ids[i], leaves[i])
            t_host += time.perf_counter() - th
            nd.execute(stream)
            nd.read_all_correlators(out)
        t_new = max_over_ranks(time.perf_counter() - t0, ws)
        e2e["new_leaves_every_step"] = {
            "value": job_flops * k_new / t_new / 1e12, "unit": "TFLOP/s", "steps": k_new,
            "ms_per_step": 1e3 * t_new / k_new, "host_pass_ms_per_step": 1e3 * t_host / k_new,
            "leaf_input_bytes_per_step": int(sum(leaves[i].nbytes for i in used)),
            "programs_built": nd.exec_info()["n_programs"] - p0}
    arena = info1["arena_bytes"]
    resident_peak = info1["resident_peak_bytes"]
    leaf_bytes = sum(nd.node_info(i)["size"] for i in range(len(wl.leaves)))
    ex_info = nd.exec_info()
    n_contr = len(nd.order())
    nd.close()
    del nd
    torch.cuda.empty_cache()

    # ---- the FP64 path on the same DAG (N=1)
    farm = None
    if mixed and args.fp64_arm and ws == 1:
        farm, _ = fp64_arm(L, wl, leaves, args.policy, args.evict, budget, stream, corr, offs,
                           args.fp64_arm)
        farm["speedup_of_mixed"] = farm["time_to_solution_s"] / t_step
    del leaves

    # ---- sub-records (N=1)
    subs = None
    if ws == 1 and args.sub != "none":
        subs = {}
        for name in [s for s in args.sub.split(",") if s and s != args.workload]:
            subs[name] = sub_record(L, name, args, stream, link)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        f, t, nr, nt = oracle_sample(wl, 20.0)
        cpu = {"value": f / t / 1e12, "unit": "TFLOP/s", "cores": blas_threads(),
               "kind": "oracle",
               "sample": "%d of %d correlator trees (random, seeded) of the %s workload with "
                         "their descendant closures, %.2f GFLOP in %.1f s"
                         % (nr, nt, args.workload, f / 1e9, t)}

    droof = dag_roofline_for(wl, ids, args.precision, t_step)
    if sharded:   # this rank's slices: every contraction's work and bytes scale with them
        for k in ("time_s", "compute_bound_s", "memory_bound_s", "flops"):
            droof[k] *= lt_share
        droof["frac"] = droof["time_s"] / t_step
    droof["link_bound_s"] = link_record(planned["h2d_bytes"], planned["d2h_bytes"], t_step,
                                        link)["bound_s"] if planned["n_evict"] else 0.0
    droof["note"] = ("leaves resident: the host link carries only evictions; the bound is "
                     "max(sum of per-contraction max(compute, HBM), link)")

    if rank == 0:
        line = {
            "metric": "dag_complex_tflops", "value": value, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak",
            "vs_baseline": None,
            "dtype": "c64/%s" % args.precision if mixed else "c128/f64",
            "data": "synthetic",
            "config": {"workload": args.workload,
                       "lt": sorted({wl.leaf_lt(i) for i in range(len(wl.leaves))}),
                       "nvec": sorted({wl.leaf_nvec(i) for i in range(len(wl.leaves))}),
                       "functions": len(wl.functions), "contractions": n_contr,
                       "policy": args.policy, "evict": args.evict, "budget_bytes": budget,
                       "precision": args.precision, "cuda_graph": bool(args.graph),
                       "window": (tuned["best"]["window"] if tuned else args.window)
                                 if mixed else 0,
                       "fused_max_n": (tuned["best"]["fused_max_n"] if tuned
                                       else args.fused_max_n) if mixed else None,
                       "split_policy": (tuned["best"]["split_policy"] if tuned
                                        else args.split_policy) if mixed else None,
                       "fused_kernel": (tuned["best"]["fused_kernel"] if tuned
                                        else args.fused_kernel) if mixed else None,
                       "autotune": tuned,
                       "parallelism": ("lt-shard" if sharded else "replicas") if ws > 1
                                      else "single",
                       "l2": "inputs larger than L2 (leaves %.2f GB, arena %.2f GB)"
                             % (leaf_bytes / 1e9, arena / 1e9)},
            "time_to_solution_s": t_step,
            "flops_per_step": flops_step,
            "peak_paper_bytes": planned["peak_paper"], "peak_exec_bytes": planned["peak_exec"],
            "n_evict": planned["n_evict"], "h2d_gb_per_step": planned["h2d_bytes"] / 1e9,
            "d2h_gb_per_step": planned["d2h_bytes"] / 1e9,
            "stats_counted_equal_planned": counted_equal,
            "extra_placement_moves": {k: ex_info[k] for k in ("extra_evictions", "extra_h2d_bytes",
                                                               "extra_d2h_bytes")},
            "arena_bytes": arena, "resident_peak_bytes": resident_peak,
            "schedule_ms": 1e3 * t_sched, "dag_build_s": t_build, "leaf_generation_s": t_gen,
            "roofline": roofline,
            "kernel_ms_per_step_by_kind": kind_breakdown(info1, nsteps) if mixed else None,
            "dag_roofline": droof,
            "fp64_arm": farm,
            "sub": subs,
            "link": link,
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
