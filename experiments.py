"""Scheduler comparisons on the device (the paper's Sec. IV-B and IV-C measurements).

For one synthetic workload and a device budget, every policy (naive
topological order, sibling, tree) is scheduled, planned and executed; the
line per policy reports the paper's figures -- peak memory of the model,
evictions, host<->device transfers (count and bytes, planned and actually
copied) -- and the measured time-to-solution of a full execution with the
leaves starting in pinned host memory.  Correlators of all policies are
compared bit for bit (each node's arithmetic is fixed; an eviction is a
copy), so a schedule can change the time but never a result.

  python experiments.py [--workload memory_pressure]
         [--precision tf32x3] [--evict lru] [--steps 2] [--budget-gib 24[,8]] [--paths]

Prints one JSON line per policy, then a summary line with ratios to the
naive order.

  python experiments.py kernel --shape pxp --n 64 --lt 64
         [--precision tf32x3|bf16x3|fp64] [--reps 20] [--fused-max-n F]

times one contraction shape through the single-contraction C ABI, or, with
--fused-max-n, as a one-contraction DAG (leaves staged on the device, the
executor's options set; F = 0 forces the plane form, a large F the fused
form of TF32X3).

  python experiments.py batched [--workload batched|baryon|...]
         [--steps 2] [--window 64]

runs a workload (default: the batched one, 50 independent DAGs of uneven N
and Lt, ~18k contractions) in the mixed-precision grouped form (windows of independent
contractions per launch, CUDA graphs) and as one launch per contraction in
FP64, with the leaves resident on the device and from pinned host memory;
reports times, speedups and the TF32x3 error of every correlator against
the FP64 path (whose parity with the oracle the test suite establishes).

  python experiments.py paths [--workloads multi_meson,...]
         [--gpu] [--steps 3]

builds each workload's terms twice -- as the generator brackets them and by
contraction-path selection (Sec. II-A) -- and reports distinct
contractions, flops and every scheduler's peak; with --gpu also both DAGs'
tuned TF32x3 time-to-solution and the largest difference of a term's value.

  python experiments.py sched [--dags multi_meson:5000,...] [--reps 5]

times each scheduler's order on the host for synthetic DAGs of the vertex
counts of the paper's Table 2, with their trees, vertices, edges, F_v, F_e.

  python experiments.py optimal [--dags 200] [--max-contr 9]

scores every scheduler's model peak against the optimal peak over all
contraction orders of small synthetic DAGs (exhaustive enumeration).

  python experiments.py model [--workloads ...] [--fractions 1,0.5,0.25]

gives the memory model's peak, evictions and transfer bytes of every
scheduler's plan at budgets relative to the tree order's peak, without
executing.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


SHAPES = {
    # name: (left extents, right extents, la, ra) with N = distillation size
    "pxp": lambda n: ((4, 4, n, n), (4, 4, n, n), (1, 3), (0, 2)),   # over spin + distillation
    "pxm": lambda n: ((4, 4, n, n), (n, n), (3,), (0,)),             # propagator x meson
    "mxm": lambda n: ((n, n), (n, n), (1,), (0,)),                   # meson x meson
    "bxb": lambda n: ((n, n, n), (n, n, n), (1, 2), (0, 1)),         # baryon x baryon, 2 legs
    # meson x propagator over the propagator's first distillation axis, in
    # both operand orders (M = N_dist, N = 16 N_dist and the transpose)
    "mxp": lambda n: ((n, n), (4, 4, n, n), (1,), (2,)),
    "pxm2": lambda n: ((4, 4, n, n), (n, n), (2,), (1,)),
    # meson x baryon over one baryon leg (last, first, middle): M = N_dist rows
    "mxb_t": lambda n: ((n, n), (n, n, n), (1,), (2,)),
    "mxb_h": lambda n: ((n, n), (n, n, n), (1,), (0,)),
    "mxb_m": lambda n: ((n, n), (n, n, n), (1,), (1,)),
    # baryon x meson over one baryon leg (first, middle, last): M = N_dist^2 rows
    "bxm_h": lambda n: ((n, n, n), (n, n), (0,), (0,)),
    "bxm_m": lambda n: ((n, n, n), (n, n), (1,), (0,)),
    "bxm_t": lambda n: ((n, n, n), (n, n), (2,), (0,)),
}


def kernel_bench(argv):
    """One contraction shape through the single-contraction C ABI, timed with
    CUDA events over `--reps` launches after warm-up."""
    import ctypes
    import torch
    import paper_2511_02257_b300 as L
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="pxp", choices=sorted(SHAPES))
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--lt", type=int, default=64)
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--fused-max-n", type=int, default=None)
    ap.add_argument("--fused-kernel", type=int, default=1,
                    help="with --fused-max-n: LQC_OPT_FUSED_KERNEL (0: A in shared memory, "
                         "1: A in tensor memory)")
    args = ap.parse_args(argv)
    sa, sb, la, ra = SHAPES[args.shape](args.n)
    lt = args.lt
    if args.fused_max_n is not None:
        return kernel_bench_dag(args, sa, sb, la, ra)
    P64 = ctypes.POINTER(ctypes.c_int64)
    PI = ctypes.POINTER(ctypes.c_int)
    ea = np.asarray(sa, np.int64)
    eb = np.asarray(sb, np.int64)
    xa = np.asarray(la, np.intc)
    xb = np.asarray(ra, np.intc)
    pa, pb = ea.ctypes.data_as(P64), eb.ctypes.data_as(P64)
    pla, pra = xa.ctypes.data_as(PI), xb.ctypes.data_as(PI)
    K = int(np.prod([sa[i] for i in la]))
    M = int(np.prod(sa)) // K
    N = int(np.prod(sb)) // K
    out_elems = lt * M * N
    g = torch.Generator(device="cuda").manual_seed(1)
    prec = L.PRECISIONS[args.precision]
    vp = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    if prec == L.LQC_PREC_FP64:
        A = torch.randn((lt,) + sa, dtype=torch.complex128, device="cuda", generator=g)
        B = torch.randn((lt,) + sb, dtype=torch.complex128, device="cuda", generator=g)
        C = torch.empty(out_elems, dtype=torch.complex128, device="cuda")

        def run():
            assert L.lqc_contract_fp64(vp(A), len(sa), pa, vp(B), len(sb), pb, len(la), pla, pra,
                                       lt, vp(C), None) == 0
    else:
        A = torch.randn((lt,) + sa, dtype=torch.complex64, device="cuda", generator=g)
        B = torch.randn((lt,) + sb, dtype=torch.complex64, device="cuda", generator=g)
        C = torch.empty(out_elems, dtype=torch.complex64, device="cuda")
        nbytes = L.lqc_contract_mixed_scratch_bytes(len(sa), pa, len(sb), pb, len(la), pla, pra,
                                                    lt, prec)
        S = torch.empty(nbytes, dtype=torch.uint8, device="cuda")

        def run():
            assert L.lqc_contract_mixed(vp(A), len(sa), pa, vp(B), len(sb), pb, len(la), pla, pra,
                                        lt, prec, vp(C), vp(S), None) == 0
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    flops = 8.0 * lt * M * N * K
    elem = 16 if prec == L.LQC_PREC_FP64 else 8
    alg_bytes = lt * (M * K + K * N + M * N) * elem
    print(json.dumps({"shape": args.shape, "n": args.n, "lt": lt, "M": M, "N": N, "K": K,
                      "precision": args.precision, "ms_per_contraction": ms,
                      "complex_tflops": flops / ms / 1e9,
                      "tensor_tflops": (3 if prec != L.LQC_PREC_FP64 else 1) * flops / ms / 1e9,
                      "algorithmic_gbs": alg_bytes / ms / 1e6}), flush=True)


def kernel_bench_dag(args, sa, sb, la, ra):
    """One contraction as a DAG (two staged leaves, one root of rank > 0)."""
    import torch
    import paper_2511_02257_b300 as L
    lt = args.lt
    rng = np.random.default_rng(1)
    d = L.Dag(lt, args.precision)
    a = d.add_leaf(sa, (rng.standard_normal((lt,) + sa) + 1j * rng.standard_normal((lt,) + sa)))
    b = d.add_leaf(sb, (rng.standard_normal((lt,) + sb) + 1j * rng.standard_normal((lt,) + sb)))
    d.add_contraction(a, b, la, ra)
    d.schedule("tree")
    stream = torch.cuda.current_stream().cuda_stream
    d.set_option(L.LQC_OPT_WINDOW, 0)
    d.set_option(L.LQC_OPT_FUSED_MAX_N, args.fused_max_n)
    d.set_option(L.LQC_OPT_FUSED_KERNEL, args.fused_kernel)
    d.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    d.stage_leaves(stream)
    for _ in range(3):
        d.execute(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        d.execute(stream)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    K = int(np.prod([sa[i] for i in la]))
    M = int(np.prod(sa)) // K
    N = int(np.prod(sb)) // K
    flops = 8.0 * lt * M * N * K
    from paper_2511_02257_b300.roofline import measured_peaks, precision_peak
    eb, prod, peak, _, _ = precision_peak(args.precision)
    bound_ms = 1e3 * max(prod * flops / (peak * 1e12),
                         lt * (M * K + K * N + M * N) * eb / (measured_peaks()[0]["hbm_gbs"] * 1e9))
    print(json.dumps({"shape": args.shape, "n": args.n, "lt": lt, "M": M, "N": N, "K": K,
                      "precision": args.precision, "fused_max_n": args.fused_max_n,
                      "fused_kernel": args.fused_kernel,
                      "ms_per_contraction": ms, "complex_tflops": flops / ms / 1e9,
                      "tensor_tflops": prod * flops / ms / 1e9, "roofline_ms": bound_ms,
                      "roofline_frac": bound_ms / ms,
                      "kernels": d.exec_info()["n_kernels"]}), flush=True)


def _gen_leaves(wl):
    import synth
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))


def _time_arm(nd, stream, steps, staged):
    """Best-of-`steps` wall time of execute + read of every correlator."""
    import torch
    if staged:
        nd.stage_leaves(stream)
    nd.execute(stream)                 # warm-up (graph capture, arena allocation)
    vals = nd.read_all_correlators()
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        nd.execute(stream)
        nd.read_all_correlators(vals)
        times.append(time.perf_counter() - t1)
    if staged:
        nd.unstage_leaves()
    return min(times), vals.copy(), nd.exec_info()


def batched_bench(argv):
    """Mixed grouped form vs one FP64 launch per contraction on the batched
    workload; see the module docstring."""
    import torch
    import paper_2511_02257_b300 as L
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--window", type=int, default=64)
    ap.add_argument("--policy", default="tree")
    args = ap.parse_args(argv)
    wl = synth.make_workload(args.workload)
    t0 = time.perf_counter()
    leaves = _gen_leaves(wl)
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream().cuda_stream
    res = {}
    rows = []
    # (precision, window, graph); window "tuned" = the library's autotuner
    arms = [("tf32x3", "tuned", 1), ("tf32x3", args.window, 1), ("tf32x3", 0, 1),
            ("tf32x3", 0, 0), ("fp64", 0, 1)]
    from paper_2511_02257_b300.roofline import dag_roofline_for
    for prec, window, graph in arms:
        nd, ids = L.build_dag(wl, precision=prec, leaf_data_fn=lambda li: leaves[li])
        planned = nd.schedule(args.policy, "lru", wl.budget_bytes)
        nd.set_option(L.LQC_OPT_CUDA_GRAPH, graph)
        tune = None
        if window == "tuned":
            nd.stage_leaves(stream)
            t0 = time.perf_counter()
            entries = nd.autotune(stream, reps=2)
            tune = {"best": entries[0], "worst_ms": entries[-1]["ms"],
                    "tune_s": time.perf_counter() - t0}
            nd.unstage_leaves()
        else:
            nd.set_option(L.LQC_OPT_WINDOW, window)
        for staged in (True, False):
            t, vals, info = _time_arm(nd, stream, args.steps, staged)
            row = {"workload": args.workload, "precision": prec, "window": window,
                   "cuda_graph": bool(graph), "leaves": "device" if staged else "pinned host",
                   "contractions": len(nd.order()), "time_to_solution_s": t,
                   "tflops": info["flops"] / t / 1e12, "kernels": info["n_kernels"],
                   "peak_paper_gib": planned["peak_paper"] / 2 ** 30,
                   "peak_exec_gib": planned["peak_exec"] / 2 ** 30,
                   "budget_gib": wl.budget_bytes / 2 ** 30, "n_evict": planned["n_evict"],
                   "h2d_gib": 0.0 if staged else planned["h2d_bytes"] / 2 ** 30,
                   "dag_roofline": dag_roofline_for(wl, ids, prec, t) if staged else None,
                   "autotune": tune}
            rows.append(row)
            res[(prec, window, graph, staged)] = (t, vals.reshape(-1))
            print(json.dumps(row), flush=True)
        nd.close()
        del nd
        torch.cuda.empty_cache()
    nd, _ = L.build_dag(wl, with_data=False)
    roots = nd.roots()
    lts = [nd.node_info(r)["lt"] for r in roots]
    offs = np.concatenate([[0], np.cumsum(lts)])
    ref64 = res[("fp64", 0, 1, True)][1]
    mixed = res[("tf32x3", "tuned", 1, True)][1]

    def per_root(v, ref):
        return np.array([np.linalg.norm(v[offs[i]:offs[i + 1]] - ref[offs[i]:offs[i + 1]]) /
                         np.linalg.norm(ref[offs[i]:offs[i + 1]]) for i in range(len(roots))])
    e_mixed = per_root(mixed, ref64)
    # fixed-option forms: same per-tile arithmetic, so the same bits
    same = all(np.array_equal(res[("tf32x3", args.window, 1, True)][1].view(np.float64),
                              res[("tf32x3", w, g, s2)][1].view(np.float64))
               for (w, g, s2) in ((0, 1, True), (0, 0, True), (args.window, 1, False)))
    t64 = res[("fp64", 0, 1, True)][0]
    summary = {
        "summary": args.workload, "roots": len(roots), "leaf_generation_s": t_gen,
        "speedup_tuned_tf32x3_vs_fp64": t64 / res[("tf32x3", "tuned", 1, True)][0],
        "speedup_tuned_tf32x3_vs_fp64_host_leaves":
            res[("fp64", 0, 1, False)][0] / res[("tf32x3", "tuned", 1, False)][0],
        "speedup_grouped_tf32x3_vs_fp64": t64 / res[("tf32x3", args.window, 1, True)][0],
        "speedup_grouping_vs_single_launches_tf32x3":
            res[("tf32x3", 0, 1, True)][0] / res[("tf32x3", args.window, 1, True)][0],
        "speedup_grouping_graph_vs_single_launches_no_graph_tf32x3":
            res[("tf32x3", 0, 0, True)][0] / res[("tf32x3", args.window, 1, True)][0],
        "tf32x3_err_vs_fp64_max": float(e_mixed.max()),
        "tf32x3_err_vs_fp64_median": float(np.median(e_mixed)),
        "tf32x3_forms_bit_identical": bool(same),
    }
    print(json.dumps(summary), flush=True)


def dag_contraction_flops(nd, elem_bytes: int = 16) -> int:
    """Real flops (8 per complex multiply-add) of every distinct contraction
    of a Dag stored with `elem_bytes` per element, from its node sizes: M*K,
    K*N and M*N are the per-slice element counts of the two operands and the
    output, so K^2 = MK * KN / MN."""
    import math
    total = 0
    for u in range(nd.num_nodes()):
        left, right, _, _ = nd.node_operands(u)
        if left < 0:
            continue
        lt = nd.node_info(u)["lt"]

        def elems(x):
            return nd.node_info(x)["size"] // (elem_bytes * lt)
        mk, kn, mn = elems(left), elems(right), elems(u)
        k = math.isqrt(mk * kn // mn)
        assert k * k * mn == mk * kn
        total += 8 * lt * (mk // k) * (kn // k) * k
    return total


def term_values(nd, flat, term_roots):
    """Correlator of each listed root from read_all_correlators' output
    (roots in ascending id, each with its own batch extent)."""
    roots = nd.roots()
    lts = [nd.node_info(r)["lt"] for r in roots]
    offs = np.concatenate([[0], np.cumsum(lts)]).astype(np.int64)
    flat = np.asarray(flat).reshape(-1)
    if flat.size != offs[-1]:
        raise ValueError("%d correlator values for %d slices" % (flat.size, offs[-1]))
    pos = {r: i for i, r in enumerate(roots)}
    return [flat[offs[pos[r]]:offs[pos[r] + 1]] for r in term_roots]


def paths_bench(argv):
    """Contraction-path selection (Sec. II-A) against the generator's own
    bracketing of the same terms: distinct contractions, flops, peak memory
    of each scheduler (at the storage size of --precision) and the host
    build time; with --gpu also the time-to-solution of both DAGs (leaves
    on the device; mixed precisions autotuned) and the largest relative
    difference of any term's correlator between them."""
    import paper_2511_02257_b300 as L
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="multi_meson,baryon,memory_pressure")
    ap.add_argument("--policies", default="naive,sibling,tree,rsgs,node")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--gpu", action="store_true")
    ap.add_argument("--steps", type=int, default=3)
    args = ap.parse_args(argv)
    eb = 16 if args.precision == "fp64" else 8
    for name in args.workloads.split(","):
        wl = synth.make_workload(name)
        nl = len(wl.leaves)
        gen_roots = [r for f in wl.functions for r in f]      # stream index of each term
        rows = {}
        for arm in ("generator", "paths"):
            t0 = time.perf_counter()
            nd, ids = L.build_dag(wl, precision=args.precision, with_data=False,
                                  paths=(arm == "paths"))
            t_build = time.perf_counter() - t0
            row = {"workload": name, "arm": arm, "precision": args.precision,
                   "terms": len(wl.graphs), "contractions": nd.num_nodes() - nl,
                   "build_s": t_build, "tflop": dag_contraction_flops(nd, eb) / 1e12}
            for pol in args.policies.split(","):
                st = nd.schedule(pol, "lru", 0)
                row["peak_exec_gib_" + pol] = st["peak_exec"] / 2 ** 30
            rows[arm] = (row, ids)
            nd.close()
        if args.gpu:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
            leaves = _gen_leaves(wl)
            vals = {}
            for arm in ("generator", "paths"):
                row, _ = rows[arm]
                nd, ids = L.build_dag(wl, precision=args.precision,
                                      leaf_data_fn=lambda li: leaves[li], paths=(arm == "paths"))
                nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
                nd.schedule("tree", "lru", wl.budget_bytes)
                best = None
                if args.precision != "fp64":
                    nd.stage_leaves(stream)
                    best = nd.autotune(stream, reps=2)[0]
                    nd.unstage_leaves()
                t, flat, info = _time_arm(nd, stream, args.steps, True)
                term_roots = [ids[r] for r in gen_roots] if arm == "generator" else ids[nl:]
                vals[arm] = term_values(nd, flat, term_roots)
                row.update({"time_to_solution_s": t, "tflops": info["flops"] / t / 1e12,
                            "autotune_best": best})
                nd.close()
                del nd
                torch.cuda.empty_cache()
            rel = [np.linalg.norm(a - b) / np.linalg.norm(a)
                   for a, b in zip(vals["generator"], vals["paths"])]
            rows["paths"][0]["max_rel_diff_vs_generator"] = float(max(rel))
        for arm in ("generator", "paths"):
            print(json.dumps(rows[arm][0]), flush=True)
        g, p = rows["generator"][0], rows["paths"][0]
        summ = {"summary": name, "contraction_ratio": p["contractions"] / g["contractions"],
                "flop_ratio": p["tflop"] / g["tflop"]}
        if args.gpu:
            summ["speedup_paths_vs_generator"] = g["time_to_solution_s"] / p["time_to_solution_s"]
        print(json.dumps(summ), flush=True)


def dag_properties(nd) -> dict:
    """The DAG columns of the paper's Table 2: trees (roots), vertices,
    edges (operand -> consumer, distinct), F_v = average number of trees a
    vertex belongs to, F_e = the same for edges (an edge belongs to the trees
    holding its consumer)."""
    n = nd.num_nodes()
    kids = []
    for u in range(n):
        left, right, _, _ = nd.node_operands(u)
        kids.append(() if left < 0 else ((left,) if left == right else (left, right)))
    roots = nd.roots()
    stamp = [-1] * n
    ntrees = [0] * n
    for i, r in enumerate(roots):
        stack = [r]
        while stack:
            u = stack.pop()
            if stamp[u] == i:
                continue
            stamp[u] = i
            ntrees[u] += 1
            stack.extend(kids[u])
    edges = sum(len(k) for k in kids)
    return {"trees": len(roots), "vertices": n, "edges": edges,
            "F_v": sum(ntrees) / n,
            "F_e": sum(ntrees[u] * len(kids[u]) for u in range(n)) / max(edges, 1)}


def sched_bench(argv):
    """Host time of each scheduler's order (the paper's Table 4) on synthetic
    DAGs scaled to the vertex counts of the paper's Table 2: the median of
    `--reps` calls of lqc_dag_schedule minus the plan replay of the same
    order (lqc_dag_set_order), so that only the order is timed."""
    import paper_2511_02257_b300 as L
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--dags", default="multi_meson:1000,multi_meson:5000,multi_meson:20000,"
                                      "baryon:3000,baryon:20000")
    ap.add_argument("--policies", default="naive,rsgs,sibling,tree,node")
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args(argv)
    for spec in args.dags.split(","):
        name, nf = spec.split(":")
        wl = synth.make_workload(name, n_functions=int(nf))
        nd, _ = L.build_dag(wl, with_data=False)
        row = {"workload": name, "functions": int(nf)}
        row.update(dag_properties(nd))
        for pol in args.policies.split(","):
            ts = []
            for _ in range(args.reps):
                t0 = time.perf_counter()
                nd.schedule(pol, "lru", 0)
                t1 = time.perf_counter()
                nd.set_order(nd.order(), "lru", 0)
                t2 = time.perf_counter()
                ts.append((t1 - t0) - (t2 - t1))
            row["order_ms_" + pol] = 1e3 * max(float(np.median(ts)), 0.0)
        print(json.dumps(row), flush=True)
        nd.close()


def contraction_orders(nd):
    """Every topological order of a Dag's contractions (operands first), by
    depth-first enumeration over the contractions whose operands are done."""
    n = nd.num_nodes()
    deps = {}
    for u in range(n):
        left, right, _, _ = nd.node_operands(u)
        if left >= 0:
            deps[u] = [c for c in {left, right} if nd.node_operands(c)[0] >= 0]
    todo = sorted(deps)
    done, cur = set(), []

    def rec():
        if len(cur) == len(todo):
            yield list(cur)
            return
        for u in todo:
            if u not in done and all(c in done for c in deps[u]):
                done.add(u)
                cur.append(u)
                yield from rec()
                cur.pop()
                done.discard(u)
    yield from rec()


def optimal_peak(nd):
    """(smallest model peak over every contraction order, number of orders):
    each order's peak from the native plan replay (no budget)."""
    best, count = None, 0
    for order in contraction_orders(nd):
        p = nd.set_order(order, "lru", 0)["peak_paper"]
        best = p if best is None else min(best, p)
        count += 1
    return best, count


def optimal_bench(argv):
    """Each scheduler's model peak against the optimal peak over all
    contraction orders, on small synthetic DAGs (at most --max-contr
    contractions) built by the meson and baryon generators."""
    import paper_2511_02257_b300 as L
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--dags", type=int, default=200)
    ap.add_argument("--max-contr", type=int, default=9)
    ap.add_argument("--policies", default="naive,rsgs,sibling,tree,node")
    args = ap.parse_args(argv)
    pols = args.policies.split(",")
    ratios = {p: [] for p in pols}
    n_dags = n_orders = seed = 0
    while n_dags < args.dags and seed < 100 * args.dags:
        name = "baryon" if seed % 3 == 2 else "multi_meson"
        kw = dict(n_functions=1 + seed % 3, nvec=4, lt=2, prefix_pool=2)
        if name == "baryon":
            kw = dict(n_functions=1 + seed % 2, nvec=3, lt=2)
        seed += 1
        wl = synth.make_workload(name, seed=seed, **kw)
        nd, _ = L.build_dag(wl, with_data=False)
        nc = nd.num_nodes() - len(wl.leaves)
        if nc < 3 or nc > args.max_contr:
            nd.close()
            continue
        opt, count = optimal_peak(nd)
        n_dags += 1
        n_orders += count
        for p in pols:
            ratios[p].append(nd.schedule(p, "lru", 0)["peak_paper"] / opt)
        nd.close()
    out = {"dags": n_dags, "orders_enumerated": n_orders}
    for p in pols:
        r = np.asarray(ratios[p])
        out[p] = {"optimal_fraction": float(np.mean(r <= 1.0)), "mean_ratio": float(r.mean()),
                  "max_ratio": float(r.max())}
    print(json.dumps(out), flush=True)


def model_bench(argv):
    """The memory model's figures (Sec. II-C) for every scheduler without
    executing: model peak, evictions and host<->device bytes of the plan at
    budgets given as fractions of the tree order's peak (1 = no eviction for
    the tree order).  Storage at the size of --precision."""
    import paper_2511_02257_b300 as L
    import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--workloads", default="multi_meson,baryon,memory_pressure,batched")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--fractions", default="1,0.5,0.25")
    ap.add_argument("--policies", default="naive,rsgs,sibling,tree,node")
    ap.add_argument("--evict", default="lru")
    args = ap.parse_args(argv)
    for spec in args.workloads.split(","):
        name, _, nf = spec.partition(":")
        wl = synth.make_workload(name, **({"n_functions": int(nf)} if nf else {}))
        nd, _ = L.build_dag(wl, precision=args.precision, with_data=False)
        tree_peak = nd.schedule("tree", args.evict, 0)["peak_exec"]
        for frac in (float(f) for f in args.fractions.split(",")):
            budget = int(tree_peak * frac)
            row = {"workload": spec, "precision": args.precision, "budget_fraction": frac,
                   "budget_bytes": budget}
            for pol in args.policies.split(","):
                try:
                    st = nd.schedule(pol, args.evict, budget)
                    row[pol] = {"peak_paper": st["peak_paper"], "n_evict": st["n_evict"],
                                "h2d_bytes": st["h2d_bytes"], "d2h_bytes": st["d2h_bytes"]}
                except L.LqcError as e:
                    row[pol] = {"error": str(e)}
            print(json.dumps(row), flush=True)
        nd.close()


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "kernel":
        return kernel_bench(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "batched":
        return batched_bench(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "paths":
        return paths_bench(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "sched":
        return sched_bench(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "optimal":
        return optimal_bench(sys.argv[2:])
    if len(sys.argv) > 1 and sys.argv[1] == "model":
        return model_bench(sys.argv[2:])
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="memory_pressure")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--evict", default="lru")
    ap.add_argument("--policies", default="naive,sibling,tree")
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--budget-gib", default=None,
                    help="device budget(s) in GiB, comma-separated (default: the workload's)")
    ap.add_argument("--graph", type=int, default=1)
    ap.add_argument("--paths", action="store_true",
                    help="build the DAG by contraction-path selection over the workload's terms")
    args = ap.parse_args()

    import torch
    import paper_2511_02257_b300 as L
    import synth

    wl = synth.make_workload(args.workload)
    budgets = [int(float(b) * 2 ** 30) for b in args.budget_gib.split(",")] \
        if args.budget_gib is not None else [wl.budget_bytes]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        leaves = list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))
    t_gen = time.perf_counter() - t0
    nd, _ = L.build_dag(wl, precision=args.precision, leaf_data_fn=lambda li: leaves[li],
                        paths=args.paths)
    del leaves
    stream = torch.cuda.current_stream().cuda_stream
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, args.graph)
    from bench import link_bandwidth
    args.link = link_bandwidth()
    print(json.dumps({"host_link": args.link}), flush=True)
    for budget in budgets:
        _compare_policies(args, wl, nd, budget, stream, t_gen)


def _compare_policies(args, wl, nd, budget, stream, t_gen):
    import torch
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
            "workload": args.workload, "paths": bool(args.paths),
            "precision": args.precision, "policy": pol,
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
            "arena_within_budget": info["arena_bytes"] <= budget,
            "extra_placement_moves": {k: info[k] for k in ("extra_evictions", "extra_h2d_bytes",
                                                            "extra_d2h_bytes")},
            # host link: copies of both directions overlap (full duplex), so the
            # bound is the slower direction's copy time at the measured bandwidth
            "link_bound_s": max(info["copied_h2d"] / (args.link["h2d_gbs"] * 1e9),
                                info["copied_d2h"] / (args.link["d2h_gbs"] * 1e9)),
            "link_frac": max(info["copied_h2d"] / (args.link["h2d_gbs"] * 1e9),
                             info["copied_d2h"] / (args.link["d2h_gbs"] * 1e9)) / min(times),
            "leaf_generation_s": t_gen,
        }
        rows.append(row)
        print(json.dumps(row), flush=True)
    base = rows[0]
    summary = {"summary": "ratios to %s" % base["policy"], "budget_bytes": budget}
    for r in rows[1:]:
        summary[r["policy"]] = {
            k: (base[k] / r[k] if r[k] else None)
            for k in ("peak_paper_gib", "n_evict", "h2d_gib", "time_to_solution_s")}
    print(json.dumps(summary), flush=True)


if __name__ == "__main__":
    main()
