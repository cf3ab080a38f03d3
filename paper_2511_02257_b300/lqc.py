"""ctypes binding of the C ABI in ``include/lqc.h`` (argument marshalling only).

Every function of the header is exposed under the same name; ``Dag`` is a
small convenience wrapper that owns a handle.  Streams are passed as raw
``cudaStream_t`` integers (e.g. ``torch.cuda.current_stream().cuda_stream``).
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "_lib", "liblqc.so")
if not os.path.exists(library_path):
    raise ImportError("native library %s is missing: build it with "
                      "`python paper_2511_02257_b300/build.py`" % library_path)
_lib = ctypes.CDLL(library_path)

c_i64 = ctypes.c_int64
c_i32 = ctypes.c_int32
P_i64 = ctypes.POINTER(ctypes.c_int64)
P_i32 = ctypes.POINTER(ctypes.c_int32)
P_int = ctypes.POINTER(ctypes.c_int)
P_dbl = ctypes.POINTER(ctypes.c_double)
c_vp = ctypes.c_void_p

LQC_OK, LQC_ERR_ARG, LQC_ERR_BUDGET, LQC_ERR_CUDA = 0, -1, -2, -3
LQC_ERR_HOST_MEM, LQC_ERR_STATE, LQC_ERR_TIMEOUT = -4, -5, -6
LQC_SCHED_NAIVE_TOPO, LQC_SCHED_TREE, LQC_SCHED_SIBLING = 0, 1, 2
LQC_SCHED_NODE, LQC_SCHED_RSGS = 3, 4
LQC_EVICT_LRU, LQC_EVICT_NEXT_USE = 0, 1
LQC_PREC_FP64, LQC_PREC_TF32X3, LQC_PREC_BF16X3 = 0, 1, 2
LQC_OPT_CUDA_GRAPH, LQC_OPT_POISON, LQC_OPT_TIMING, LQC_OPT_WINDOW = 1, 2, 3, 4
LQC_OPT_FUSED_MAX_N, LQC_OPT_SPLIT_POLICY, LQC_OPT_FUSED_KERNEL = 5, 6, 7
OP_NAMES = {0: "LOAD", 1: "EVICT", 2: "CONTRACT", 3: "FREE"}
LQC_NUM_KINDS = 8
KIND_NAMES = {0: "reorder", 1: "pack", 2: "gemm_planes", 3: "gemm_fused", 4: "reduce",
              5: "correlator", 6: "correlator_sum"}
POLICIES = {"naive": LQC_SCHED_NAIVE_TOPO, "tree": LQC_SCHED_TREE, "sibling": LQC_SCHED_SIBLING,
            "node": LQC_SCHED_NODE, "rsgs": LQC_SCHED_RSGS}
EVICTS = {"lru": LQC_EVICT_LRU, "next_use": LQC_EVICT_NEXT_USE}
PRECISIONS = {"fp64": LQC_PREC_FP64, "tf32x3": LQC_PREC_TF32X3, "bf16x3": LQC_PREC_BF16X3}


class lqc_stats(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in ("peak_paper", "peak_exec", "n_evict", "n_h2d", "n_d2h",
                                     "h2d_bytes", "d2h_bytes")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}

    def as_tuple(self):
        return tuple(int(getattr(self, n)) for n, _ in self._fields_)


class lqc_exec_info(ctypes.Structure):
    _fields_ = [(n, c_i64) for n in ("n_kernels", "flops", "arena_bytes", "copied_h2d",
                                     "copied_d2h", "n_ops", "n_contract", "n_contract_all")] + \
        [("ms_contract", ctypes.c_double), ("ms_contract_all", ctypes.c_double),
         ("flops_contract", c_i64), ("flops_contract_all", c_i64), ("host_arena_bytes", c_i64),
         ("n_kind", c_i64 * LQC_NUM_KINDS), ("ms_kind", ctypes.c_double * LQC_NUM_KINDS),
         ("flops_gemm", c_i64), ("resident_peak_bytes", c_i64),
         ("extra_evictions", c_i64), ("extra_h2d_bytes", c_i64), ("extra_d2h_bytes", c_i64),
         ("n_programs", c_i64)]

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        d["n_kind"] = {KIND_NAMES[k]: int(self.n_kind[k]) for k in KIND_NAMES}
        d["ms_kind"] = {KIND_NAMES[k]: float(self.ms_kind[k]) for k in KIND_NAMES}
        return d


class lqc_tune_entry(ctypes.Structure):
    _fields_ = [("window", c_i64), ("fused_max_n", c_i64), ("split_policy", c_i64),
                ("fused_kernel", c_i64), ("ms", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("lqc_dag_create", ctypes.c_int, [ctypes.POINTER(c_vp), c_i64, ctypes.c_int])
_sig("lqc_dag_destroy", ctypes.c_int, [c_vp])
_sig("lqc_dag_set_batch", ctypes.c_int, [c_vp, c_i64])
_sig("lqc_dag_add_leaf_tensor", ctypes.c_int, [c_vp, ctypes.c_int, P_i64, P_dbl, P_i64])
_sig("lqc_dag_set_leaf_data", ctypes.c_int, [c_vp, c_i64, P_dbl])
_sig("lqc_dag_add_contraction", ctypes.c_int, [c_vp, c_i64, c_i64, ctypes.c_int, P_int, P_int, P_i64])
_sig("lqc_dag_add_graphs", ctypes.c_int, [c_vp, c_i64, P_i64, P_i64, P_i64, P_i32, P_i64])
_sig("lqc_dag_add_contractions", ctypes.c_int, [c_vp, c_i64, P_i64, P_i64, P_int, P_int, P_int,
                                                P_i64])
_sig("lqc_dag_schedule", ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                        ctypes.POINTER(lqc_stats)])
_sig("lqc_dag_set_order", ctypes.c_int, [c_vp, P_i64, c_i64, ctypes.c_int, ctypes.c_uint64,
                                         ctypes.POINTER(lqc_stats)])
_sig("lqc_dag_get_order", ctypes.c_int, [c_vp, P_i64, c_i64, P_i64])
_sig("lqc_dag_get_plan", ctypes.c_int, [c_vp, P_i32, P_i64, P_i32, c_i64, P_i64])
_sig("lqc_dag_set_option", ctypes.c_int, [c_vp, ctypes.c_int, c_i64])
_sig("lqc_dag_stage_leaves", ctypes.c_int, [c_vp, c_vp])
_sig("lqc_dag_unstage_leaves", ctypes.c_int, [c_vp])
_sig("lqc_dag_execute", ctypes.c_int, [c_vp, c_vp])
_sig("lqc_dag_prepare", ctypes.c_int, [c_vp, c_vp])
_sig("lqc_test_inject_failure", ctypes.c_int, [ctypes.c_int, c_i64])
_sig("lqc_test_expire_wait", ctypes.c_int, [c_i64, c_vp])
_sig("lqc_test_tamper_plan", ctypes.c_int, [c_vp, ctypes.c_int])
_sig("lqc_test_tf32_rounding", ctypes.c_int, [c_i64, ctypes.c_uint32, P_i64])
_sig("lqc_test_read_leaf_store", ctypes.c_int, [c_vp, c_i64, c_vp, c_i64, P_int])
_sig("lqc_dag_wait", ctypes.c_int, [c_vp, c_i64])
_sig("lqc_dag_autotune", ctypes.c_int, [c_vp, c_vp, ctypes.c_int, ctypes.POINTER(lqc_tune_entry),
                                        c_i64, P_i64])
_sig("lqc_dag_read_correlator", ctypes.c_int, [c_vp, c_i64, P_dbl])
_sig("lqc_dag_read_all_correlators", ctypes.c_int, [c_vp, P_dbl, c_i64])
_sig("lqc_dag_get_roots", ctypes.c_int, [c_vp, P_i64, c_i64, P_i64])
_sig("lqc_dag_num_nodes", ctypes.c_int, [c_vp, P_i64])
_sig("lqc_dag_node_info", ctypes.c_int, [c_vp, c_i64, P_i64, P_int, P_int, P_i64])
_sig("lqc_dag_node_operands", ctypes.c_int, [c_vp, c_i64, P_i64, P_i64, P_int, P_int, P_int])
_sig("lqc_dag_get_stats", ctypes.c_int, [c_vp, ctypes.POINTER(lqc_stats)])
_sig("lqc_dag_get_exec_info", ctypes.c_int, [c_vp, ctypes.POINTER(lqc_exec_info)])
_sig("lqc_last_error", ctypes.c_char_p, [c_vp])
_sig("lqc_dag_get_kernel_times", ctypes.c_int, [c_vp, P_i64, P_dbl, c_i64, P_i64])
_sig("lqc_contract_fp64", ctypes.c_int, [c_vp, ctypes.c_int, P_i64, c_vp, ctypes.c_int, P_i64,
                                         ctypes.c_int, P_int, P_int, c_i64, c_vp, c_vp])
_sig("lqc_contract_all_fp64", ctypes.c_int, [c_vp, ctypes.c_int, P_i64, c_vp, ctypes.c_int, P_i64,
                                             ctypes.c_int, P_int, P_int, c_i64, c_vp, c_vp, c_vp])
_sig("lqc_contract_all_scratch_bytes", c_i64, [c_i64, c_i64])
_sig("lqc_measure_fp64_peak", ctypes.c_int, [P_dbl])
_sig("lqc_contract_mixed", ctypes.c_int, [c_vp, ctypes.c_int, P_i64, c_vp, ctypes.c_int, P_i64,
                                          ctypes.c_int, P_int, P_int, c_i64, ctypes.c_int, c_vp,
                                          c_vp, c_vp])
_sig("lqc_contract_mixed_scratch_bytes", c_i64, [ctypes.c_int, P_i64, ctypes.c_int, P_i64,
                                                 ctypes.c_int, P_int, P_int, c_i64, ctypes.c_int])
_sig("lqc_contract_all_c64", ctypes.c_int, [c_vp, ctypes.c_int, P_i64, c_vp, ctypes.c_int, P_i64,
                                            ctypes.c_int, P_int, P_int, c_i64, ctypes.c_double,
                                            c_vp, c_vp, c_vp])
_sig("lqc_mixed_error", ctypes.c_int, [ctypes.c_int])
_sig("lqc_contract_all_c64_scratch_bytes", c_i64, [ctypes.c_int, P_i64, ctypes.c_int, P_i64,
                                                   ctypes.c_int, P_int, P_int, c_i64])

# re-export the raw entry points under their C names
for _n in ("lqc_dag_create", "lqc_dag_destroy", "lqc_dag_set_batch", "lqc_dag_add_leaf_tensor", "lqc_dag_set_leaf_data",
           "lqc_dag_add_contraction", "lqc_dag_add_contractions", "lqc_dag_add_graphs",
           "lqc_dag_schedule", "lqc_dag_set_order", "lqc_dag_get_order",
           "lqc_dag_get_plan", "lqc_dag_set_option", "lqc_dag_stage_leaves",
           "lqc_dag_unstage_leaves", "lqc_dag_execute", "lqc_dag_wait", "lqc_dag_autotune",
           "lqc_dag_read_correlator",
           "lqc_dag_read_all_correlators", "lqc_dag_get_roots", "lqc_dag_num_nodes",
           "lqc_dag_node_info", "lqc_dag_node_operands", "lqc_dag_get_stats", "lqc_dag_get_exec_info", "lqc_last_error",
           "lqc_dag_get_kernel_times",
           "lqc_contract_fp64", "lqc_contract_all_fp64", "lqc_contract_all_scratch_bytes",
           "lqc_measure_fp64_peak", "lqc_contract_mixed", "lqc_contract_mixed_scratch_bytes",
           "lqc_contract_all_c64", "lqc_mixed_error", "lqc_contract_all_c64_scratch_bytes",
           "lqc_dag_prepare", "lqc_test_inject_failure", "lqc_test_expire_wait",
           "lqc_test_tamper_plan", "lqc_test_tf32_rounding", "lqc_test_read_leaf_store"):
    globals()[_n] = getattr(_lib, _n)


def measure_fp64_peak() -> float:
    """FP64 FMA throughput of the current device in TFLOP/s (diagnostic)."""
    v = ctypes.c_double()
    rc = _lib.lqc_measure_fp64_peak(ctypes.byref(v))
    if rc != LQC_OK:
        raise LqcError(rc, "lqc_measure_fp64_peak")
    return v.value


class LqcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lqc error %d: %s" % (code, msg))
        self.code = code


def _i64arr(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.int64))
    return a, a.ctypes.data_as(P_i64)


def _intarr(xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.intc))
    return a, a.ctypes.data_as(P_int)


class Dag:
    """Owns one ``lqc_dag`` handle."""

    def __init__(self, lt: int, precision: str = "fp64"):
        h = c_vp()
        rc = _lib.lqc_dag_create(ctypes.byref(h), int(lt), PRECISIONS[precision])
        if rc != LQC_OK:
            raise LqcError(rc, "lqc_dag_create")
        self.h = h
        self.lt = int(lt)          # batch extent of the leaves registered next
        self.precision = precision
        self._root_lts = None      # (num_nodes, roots, their batch extents)

    def close(self):
        if getattr(self, "h", None):
            _lib.lqc_dag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != LQC_OK:
            msg = _lib.lqc_last_error(self.h)
            raise LqcError(rc, "%s: %s" % (what, msg.decode() if msg else ""))

    # -- building
    def set_batch(self, lt: int):
        """Batch extent of the leaves registered next (independent problems
        with different time extents in one DAG)."""
        self._check(_lib.lqc_dag_set_batch(self.h, int(lt)), "set_batch")
        self.lt = int(lt)

    def add_leaf(self, extents: Sequence[int], data: Optional[np.ndarray] = None,
                 lt: Optional[int] = None) -> int:
        if lt is not None and int(lt) != self.lt:
            self.set_batch(lt)
        ext, pe = _i64arr(list(extents) or [0])
        nid = c_i64()
        pd = None
        if data is not None:
            arr = np.ascontiguousarray(data, dtype=np.complex128)
            expect = self.lt * int(np.prod(extents, dtype=np.int64))
            if arr.size != expect:
                raise ValueError("leaf data has %d values, expected %d" % (arr.size, expect))
            pd = arr.view(np.float64).ctypes.data_as(P_dbl)
        self._check(_lib.lqc_dag_add_leaf_tensor(self.h, len(extents), pe, pd, ctypes.byref(nid)),
                    "add_leaf_tensor")
        return nid.value

    def set_leaf_data(self, leaf: int, data: np.ndarray):
        arr = np.ascontiguousarray(data, dtype=np.complex128)
        self._check(_lib.lqc_dag_set_leaf_data(self.h, int(leaf),
                                               arr.view(np.float64).ctypes.data_as(P_dbl)),
                    "set_leaf_data")

    def leaf_store(self, leaf: int):
        """(values, exponent) of a leaf's host store as the library keeps it:
        complex128 values (FP64), or complex64 values x * 2^-exponent (mixed
        precisions); shape (Lt, elements).  A test hook."""
        info = self.node_info(leaf)
        dt = np.complex128 if self.precision == "fp64" else np.complex64
        out = np.zeros(info["size"] // np.dtype(dt).itemsize, dtype=dt)
        e = ctypes.c_int()
        self._check(_lib.lqc_test_read_leaf_store(self.h, int(leaf), out.ctypes.data_as(c_vp),
                                                  out.nbytes, ctypes.byref(e)),
                    "test_read_leaf_store")
        return out.reshape(info["lt"], -1), e.value

    def add_contraction(self, left: int, right: int, la: Sequence[int], ra: Sequence[int]) -> int:
        a, pa = _intarr(la)
        b, pb = _intarr(ra)
        nid = c_i64()
        self._check(_lib.lqc_dag_add_contraction(self.h, int(left), int(right), len(la), pa, pb,
                                                 ctypes.byref(nid)), "add_contraction")
        return nid.value

    def add_contractions(self, requests) -> List[int]:
        """Many contractions in one call: requests = [(left, right, la, ra)];
        an operand is an existing id, or -(k + 1) for the node request k < i
        of this call receives.  Returns the node ids; on error nothing is
        added."""
        n = len(requests)
        if n == 0:
            return []
        ids = np.zeros(n, dtype=np.int64)
        left = np.fromiter((q[0] for q in requests), dtype=np.int64, count=n)
        right = np.fromiter((q[1] for q in requests), dtype=np.int64, count=n)
        npairs = np.fromiter((len(q[2]) for q in requests), dtype=np.intc, count=n)
        la_a, pla = _intarr([a for q in requests for a in q[2]] or [0])
        ra_a, pra = _intarr([b for q in requests for b in q[3]] or [0])
        self._check(_lib.lqc_dag_add_contractions(self.h, n, left.ctypes.data_as(P_i64),
                                                  right.ctypes.data_as(P_i64),
                                                  npairs.ctypes.data_as(P_int), pla, pra,
                                                  ids.ctypes.data_as(P_i64)), "add_contractions")
        return ids.tolist()

    def add_graphs(self, graphs) -> List[int]:
        """Contraction-path selection (Sec. II-A): reduce every graph
        (vertex node ids, edges (vertex a, axis a, vertex b, axis b) with
        graph-local vertices) to one node; returns each graph's root id."""
        vo, vn, eo, ed = [0], [], [0], []
        for nodes, edges in graphs:
            vn.extend(int(u) for u in nodes)
            vo.append(len(vn))
            for e in edges:
                ed.extend(int(x) for x in e)
            eo.append(len(ed) // 4)
        a, pa = _i64arr(vo)
        b, pb = _i64arr(vn)
        c, pc = _i64arr(eo)
        e = np.ascontiguousarray(np.asarray(ed if ed else [0], dtype=np.int32))
        roots = np.zeros(max(len(graphs), 1), dtype=np.int64)
        self._check(_lib.lqc_dag_add_graphs(self.h, len(graphs), pa, pb, pc,
                                            e.ctypes.data_as(P_i32), roots.ctypes.data_as(P_i64)),
                    "add_graphs")
        return roots[:len(graphs)].tolist()

    # -- scheduling
    def schedule(self, policy="tree", evict="lru", budget_bytes: int = 0) -> dict:
        st = lqc_stats()
        self._check(_lib.lqc_dag_schedule(self.h, POLICIES.get(policy, policy),
                                          EVICTS.get(evict, evict), int(budget_bytes),
                                          ctypes.byref(st)), "schedule")
        return st.as_dict()

    def set_order(self, order, evict="lru", budget_bytes: int = 0) -> dict:
        o, po = _i64arr(order)
        st = lqc_stats()
        self._check(_lib.lqc_dag_set_order(self.h, po, len(o), EVICTS.get(evict, evict),
                                           int(budget_bytes), ctypes.byref(st)), "set_order")
        return st.as_dict()

    def order(self):
        n = c_i64()
        _lib.lqc_dag_get_order(self.h, None, 0, ctypes.byref(n))
        out = np.zeros(max(n.value, 1), dtype=np.int64)
        self._check(_lib.lqc_dag_get_order(self.h, out.ctypes.data_as(P_i64), len(out),
                                           ctypes.byref(n)), "get_order")
        return out[:n.value].tolist()

    def plan(self):
        n = c_i64()
        _lib.lqc_dag_get_plan(self.h, None, None, None, 0, ctypes.byref(n))
        m = max(n.value, 1)
        k = np.zeros(m, dtype=np.int32)
        nd = np.zeros(m, dtype=np.int64)
        fl = np.zeros(m, dtype=np.int32)
        self._check(_lib.lqc_dag_get_plan(self.h, k.ctypes.data_as(P_i32), nd.ctypes.data_as(P_i64),
                                          fl.ctypes.data_as(P_i32), m, ctypes.byref(n)), "get_plan")
        return [(OP_NAMES[int(k[i])], int(nd[i]), int(fl[i])) for i in range(n.value)]

    def set_option(self, option: int, value: int):
        self._check(_lib.lqc_dag_set_option(self.h, int(option), int(value)), "set_option")

    # -- execution
    def stage_leaves(self, stream: int = 0):
        self._check(_lib.lqc_dag_stage_leaves(self.h, c_vp(stream)), "stage_leaves")

    def unstage_leaves(self):
        self._check(_lib.lqc_dag_unstage_leaves(self.h), "unstage_leaves")

    def execute(self, stream: int = 0):
        self._check(_lib.lqc_dag_execute(self.h, c_vp(stream)), "execute")

    def prepare(self, stream: int = 0):
        self._check(_lib.lqc_dag_prepare(self.h, c_vp(stream)), "prepare")

    def autotune(self, stream: int = 0, reps: int = 3):
        """Time every candidate of (window, fused-form limit, split policy,
        fused GEMM tile) on this DAG and keep the fastest; returns the
        candidates with their ms per execute, fastest first."""
        entries = (lqc_tune_entry * 64)()
        n = c_i64()
        self._check(_lib.lqc_dag_autotune(self.h, c_vp(stream), int(reps), entries, 64,
                                          ctypes.byref(n)), "autotune")
        return sorted((entries[i].as_dict() for i in range(n.value)), key=lambda e: e["ms"])

    def wait(self, timeout_ms: int = 60000):
        self._check(_lib.lqc_dag_wait(self.h, int(timeout_ms)), "wait")

    def roots(self):
        n = c_i64()
        _lib.lqc_dag_get_roots(self.h, None, 0, ctypes.byref(n))
        out = np.zeros(max(n.value, 1), dtype=np.int64)
        self._check(_lib.lqc_dag_get_roots(self.h, out.ctypes.data_as(P_i64), len(out),
                                           ctypes.byref(n)), "get_roots")
        return out[:n.value].tolist()

    def _roots_and_lts(self):
        nn = self.num_nodes()
        if self._root_lts is None or self._root_lts[0] != nn:
            roots = self.roots()
            self._root_lts = (nn, roots, [self.node_info(r)["lt"] for r in roots])
        return self._root_lts[1], self._root_lts[2]

    def read_correlator(self, root: int) -> np.ndarray:
        out = np.zeros(2 * self.node_info(root)["lt"], dtype=np.float64)
        self._check(_lib.lqc_dag_read_correlator(self.h, int(root), out.ctypes.data_as(P_dbl)),
                    "read_correlator")
        return out.view(np.complex128)

    def read_all_correlators(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """[n_roots][lt] when all roots share one batch extent, else the
        roots' correlators concatenated in ascending root id (1-D)."""
        roots, lts = self._roots_and_lts()
        if out is None:
            if len(set(lts)) <= 1:
                out = np.zeros((len(roots), lts[0] if lts else self.lt), dtype=np.complex128)
            else:
                out = np.zeros(int(sum(lts)), dtype=np.complex128)
        self._check(_lib.lqc_dag_read_all_correlators(self.h, out.view(np.float64).ctypes.data_as(P_dbl),
                                                      out.size * 2), "read_all_correlators")
        return out

    def num_nodes(self) -> int:
        n = c_i64()
        self._check(_lib.lqc_dag_num_nodes(self.h, ctypes.byref(n)), "num_nodes")
        return n.value

    def node_info(self, nid: int):
        sz, rk, lf, lt = c_i64(), ctypes.c_int(), ctypes.c_int(), c_i64()
        self._check(_lib.lqc_dag_node_info(self.h, int(nid), ctypes.byref(sz), ctypes.byref(rk),
                                           ctypes.byref(lf), ctypes.byref(lt)), "node_info")
        return {"size": sz.value, "rank": rk.value, "is_leaf": bool(lf.value), "lt": lt.value}

    def node_operands(self, nid: int):
        """(left, right, la, ra) of a node; (-1, -1, (), ()) for a leaf."""
        l, r, n = c_i64(), c_i64(), ctypes.c_int()
        la = (ctypes.c_int * 8)()
        ra = (ctypes.c_int * 8)()
        self._check(_lib.lqc_dag_node_operands(self.h, int(nid), ctypes.byref(l), ctypes.byref(r),
                                               ctypes.byref(n), la, ra), "node_operands")
        return l.value, r.value, tuple(la[:n.value]), tuple(ra[:n.value])

    def stats(self) -> dict:
        st = lqc_stats()
        self._check(_lib.lqc_dag_get_stats(self.h, ctypes.byref(st)), "get_stats")
        return st.as_dict()

    def kernel_times(self):
        """{node id: summed kernel ms} of the timed contractions."""
        n = c_i64()
        _lib.lqc_dag_get_kernel_times(self.h, None, None, 0, ctypes.byref(n))  # size query
        m = max(n.value, 1)
        nodes = np.zeros(m, dtype=np.int64)
        ms = np.zeros(m, dtype=np.float64)
        self._check(_lib.lqc_dag_get_kernel_times(self.h, nodes.ctypes.data_as(P_i64),
                                                  ms.ctypes.data_as(P_dbl), m, ctypes.byref(n)),
                    "get_kernel_times")
        return {int(nodes[i]): float(ms[i]) for i in range(n.value)}

    def exec_info(self) -> dict:
        info = lqc_exec_info()
        self._check(_lib.lqc_dag_get_exec_info(self.h, ctypes.byref(info)), "get_exec_info")
        return info.as_dict()


def build_dag(wl, precision: str = "fp64", with_data: bool = True, leaf_data_fn=None,
              paths: bool = False, shard=None):
    """Feed a ``synth.Workload`` request stream into a new Dag.

    Returns (dag, ids) where ids maps stream index -> node id.  With
    ``paths`` the contractions come from path selection over the workload's
    graphs instead (Sec. II-A) and ids lists the leaf ids then the roots.
    With ``shard=(rank, world)`` the Dag holds only this rank's time slices
    of every tensor (``shard.lt_slices`` of each leaf's batch extent; leaf
    data sliced accordingly)."""
    from .shard import lt_slices
    rank, world = shard if shard is not None else (0, 1)
    t0, t1 = lt_slices(wl.lt, world)[rank]
    d = Dag(t1 - t0, precision)
    ids = []
    for li, lf in enumerate(wl.leaves):
        a, b = lt_slices(wl.leaf_lt(li), world)[rank]
        data = None
        if with_data and leaf_data_fn:
            data = leaf_data_fn(li)
            if world > 1:
                data = data[a:b]
        ids.append(d.add_leaf(lf.extents, data, lt=b - a))
    if paths:
        return d, ids + d.add_graphs([([ids[v] for v in items], edges)
                                      for items, edges in wl.graphs])
    # the request stream in one call: stream index k >= n_leaves refers to
    # request k - n_leaves of this same call
    nl = len(ids)

    def ref(k):
        return ids[k] if k < nl else -(k - nl + 1)
    ids.extend(d.add_contractions([(ref(rq.left), ref(rq.right), rq.la, rq.ra)
                                   for rq in wl.requests]))
    return d, ids
