"""Roofline of a whole contraction DAG.

Each distinct contraction i is bounded below by the larger of its compute
time F_i / P and its memory time B_i / BW, where F_i = 8 Lt M N K real flops
(complex multiply-adds) times the number of real products per complex one
in the precision form (3 for the split products, 1 in FP64), and B_i = the
bytes of both operands and the output at the storage element size (a
correlator's output is a few bytes and is left out).  The DAG bound is the
sum over contractions (each runs once), the host link left out for resident
leaves.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Sequence

import numpy as np

FP64_NOMINAL_TFLOPS = 1.25   # B300 FP64 rate, nominal
# dense tensor rates relative to BF16 (nominal B300 figures: TF32 1.1 and
# BF16 2.25 PFLOP/s), applied to the measured BF16 GEMM peak
TENSOR_RATIO = {"tf32x3": 1.1 / 2.25, "bf16x3": 1.0}


def measured_peaks():
    """(peaks, source): the copy bandwidth and BF16 GEMM rate measured on
    this machine's GPUs (MEASURED_PEAKS.json at the repository root), else
    fallback figures of an earlier B300 measurement."""
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, \
            "fallback"


def precision_peak(precision: str):
    """(elem_bytes, products, peak TFLOP/s, bound, source) of a precision."""
    peaks, src = measured_peaks()
    if precision == "fp64":
        return 16, 1, FP64_NOMINAL_TFLOPS, "alu", "nominal FP64"
    return 8, 3, peaks["bf16_tflops"] * TENSOR_RATIO[precision], "tensor", \
        "%s BF16 GEMM x nominal %s/BF16 %.3f" % (src, precision[:4].upper(),
                                                 TENSOR_RATIO[precision])


def contraction_shapes(wl, ids: Sequence[int]) -> Dict[int, tuple]:
    """{node id: (lt, M, N, K, out_elems_per_slice)} of the distinct
    contractions of a synth.Workload, from its request stream."""
    ext = wl.stream_extents()
    nl = len(wl.leaves)
    lt_of: List[int] = [wl.leaf_lt(i) for i in range(nl)]
    out = {}
    for j, rq in enumerate(wl.requests):
        lt = lt_of[rq.left]
        lt_of.append(lt)
        node = ids[nl + j]
        if node in out:
            continue
        le, re_ = ext[rq.left], ext[rq.right]
        k = int(np.prod([le[a] for a in rq.la], dtype=np.int64))
        m = int(np.prod(le, dtype=np.int64)) // k
        n = int(np.prod(re_, dtype=np.int64)) // k
        out[node] = (lt, m, n, k, int(np.prod(ext[nl + j], dtype=np.int64)) if ext[nl + j] else 0)
    return out


def dag_roofline_for(wl, ids, precision: str, measured_s: float = None) -> dict:
    """dag_roofline with the peaks of `precision`; frac = bound / measured."""
    eb, prod, peak, _, src = precision_peak(precision)
    r = dag_roofline(wl, ids, eb, prod, peak, measured_peaks()[0]["hbm_gbs"])
    r["peak_source"] = src
    if measured_s:
        r["frac"] = r["time_s"] / measured_s
    return r


def dag_roofline(wl, ids, elem_bytes: int, products: int, peak_tflops: float,
                 hbm_gbs: float) -> dict:
    """Lower bound on the device time of one execution, with its compute-
    and memory-bound parts."""
    t_c = t_m = 0.0
    flops = 0
    for (lt, m, n, k, o) in contraction_shapes(wl, ids).values():
        f = 8 * lt * m * n * k
        flops += f
        b = lt * (m * k + k * n + o) * elem_bytes
        tc = products * f / (peak_tflops * 1e12)
        tm = b / (hbm_gbs * 1e9)
        if tc >= tm:
            t_c += tc
        else:
            t_m += tm
    return {"time_s": t_c + t_m, "compute_bound_s": t_c, "memory_bound_s": t_m,
            "flops": flops, "peak_tflops": peak_tflops, "hbm_gbs": hbm_gbs}
