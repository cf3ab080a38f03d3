"""Batched workloads: independent correlation-function DAGs of uneven shape
(own distillation size N and own batch extent Lt) held in one DAG.

* Oracle pins: a node's size carries its own batch extent.  The naive order
  of a batched DAG runs the parts one after the other and the memory of
  each part falls back to zero at its end (M_n = 0, Sec. II-C), so the
  batched peak equals the largest peak of the parts, each computed as a
  standalone single-Lt DAG (sizes from the DAG-wide Lt there).
* Operands with different batch extents are rejected on both sides.
* Native orders, plans and figures bit-exact with the oracle's simulator.
* GPU: every correlator of a reduced batched DAG against the oracle, FP64
  (<= 1e-12) and TF32x3 in grouped windows with CUDA graphs (<= 1e-6), and
  the ragged layout of read_all_correlators.
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D
from oracle import memory as M
from oracle import schedule as S

L = pytest.importorskip("paper_2511_02257_b300")

SMALL = dict(n_dags=6, nvecs=(16, 24, 32, 48), lts=(4, 8, 12), n_functions=8)


def _parts(wl):
    """Split the stream into its independent parts (connected components of
    leaves and requests), each as (leaf indices, request indices)."""
    parent = list(range(len(wl.leaves) + len(wl.requests)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x
    nl = len(wl.leaves)
    for k, rq in enumerate(wl.requests):
        for o in (rq.left, rq.right):
            parent[find(o)] = find(nl + k)
    comps = {}
    for i in range(len(parent)):
        comps.setdefault(find(i), []).append(i)
    out = []
    for members in comps.values():
        lv = [i for i in members if i < nl]
        rq = [i - nl for i in members if i >= nl]
        if rq:
            out.append((lv, rq))
    return out


def test_batched_workload_shape():
    wl = synth.make_workload("batched")
    od, _ = D.build_from_workload(wl)
    n_contr = len(od.non_leaf())
    assert 15000 <= n_contr <= 25000
    assert {lf.nvec for lf in wl.leaves} <= set(synth.BATCHED["batched"].nvecs)
    assert len({(lf.nvec, lf.lt) for lf in wl.leaves}) >= 10
    for n in od.nodes:                       # contractions never mix parts
        if not n.is_leaf:
            assert od.nodes[n.left].lt == od.nodes[n.right].lt == n.lt


@pytest.mark.parametrize("seed", [0, 1])
def test_batched_peak_is_max_of_standalone_parts(seed):
    wl = synth.make_workload("batched", seed=seed, **SMALL)
    od, ids = D.build_from_workload(wl)
    parts = _parts(wl)
    assert len(parts) >= SMALL["n_dags"]
    peaks, leaf_bytes = [], 0
    for lv, rq in parts:
        lts = {wl.leaf_lt(i) for i in lv}
        assert len(lts) == 1
        # standalone DAG of this part: sizes from the DAG-wide batch extent
        pd = D.Dag(lts.pop())
        pid = {}
        for i in sorted(lv):
            pid[i] = pd.add_leaf(wl.leaves[i].extents)
        nl = len(wl.leaves)
        for k in sorted(rq):
            r = wl.requests[k]
            pid[nl + k] = pd.add_contraction(pid[r.left], pid[r.right], r.la, r.ra)
        order = S.naive(pd)
        peaks.append(M.peak_paper(pd, order))
        leaf_bytes += sum(pd.size(u) for u in pd.used_leaves())
    order = S.naive(od)
    assert M.peak_paper(od, order) == max(peaks)
    plan = M.replay(od, order)
    assert plan.stats.h2d_bytes == leaf_bytes          # every used leaf loaded once


def test_mismatched_batch_extents_rejected():
    od = D.Dag(4)
    a = od.add_leaf((3, 3))
    b = od.add_leaf((3, 3), lt=5)
    with pytest.raises(ValueError):
        od.add_contraction(a, b, (1,), (0,))
    nd = L.Dag(4)
    a = nd.add_leaf((3, 3))
    b = nd.add_leaf((3, 3), lt=5)
    with pytest.raises(L.LqcError) as ei:
        nd.add_contraction(a, b, [1], [0])
    assert ei.value.code == L.LQC_ERR_ARG
    c = nd.add_contraction(b, b, [1], [0])
    assert nd.node_info(c)["lt"] == 5 and nd.node_info(c)["size"] == 5 * 9 * 16
    with pytest.raises(L.LqcError):
        nd.set_batch(0)


@pytest.mark.parametrize("evict", [M.LRU, M.NEXT_USE])
def test_batched_orders_and_plans_bit_exact(evict):
    wl = synth.make_workload("batched", seed=2, **SMALL)
    od, _ = D.build_from_workload(wl)
    nd, _ = L.build_dag(wl, with_data=False)
    assert nd.num_nodes() == len(od.nodes)
    for u in range(len(od.nodes)):
        info = nd.node_info(u)
        assert (info["size"], info["lt"]) == (od.size(u), od.nodes[u].lt)
    budget = M.replay(od, S.naive(od)).stats.peak_exec // 3
    for sched in ("naive", "sibling", "tree"):
        order = S.SCHEDULERS[sched](od)
        st = nd.schedule(sched, {M.LRU: "lru", M.NEXT_USE: "next_use"}[evict], budget)
        assert nd.order() == order
        plan = M.replay(od, order, budget=budget, policy=evict)
        assert tuple(st[k] for k in st) == plan.stats.as_tuple()
        assert nd.plan() == [(k, u, f) for (k, u, f) in plan.ops]


# ---------------------------------------------------------------- GPU
@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("tf32x3", 1e-6)])
def test_batched_dag_vs_oracle(precision, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("batched", seed=3, **SMALL)
    od, _ = D.build_from_workload(wl)
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
    nd, _ = L.build_dag(wl, precision=precision, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    planned = nd.schedule("tree", "lru", 0)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                       # capture, then replay
        nd.execute(stream)
        flat = nd.read_all_correlators()
    assert nd.stats() == planned
    roots = nd.roots()
    assert sorted(roots) == sorted(ref)
    assert flat.ndim == 1 and flat.size == sum(od.nodes[r].lt for r in roots)
    off = 0
    errs = []
    for r in roots:
        v = nd.read_correlator(r)
        assert v.shape == (od.nodes[r].lt,)
        assert np.array_equal(v, flat[off:off + v.size])
        off += v.size
        errs.append(np.linalg.norm(v - ref[r]) / np.linalg.norm(ref[r]))
    assert max(errs) < tol, max(errs)


@pytest.mark.gpu
def test_batched_full_size_sampled_roots_tf32x3():
    """The full batched workload (50 parts, ~18k contractions, N 32..256,
    Lt 16..128) in grouped windows with CUDA graphs: 64 seeded correlators,
    at least two of every (N, Lt) class of the parts, against the oracle
    (<= 1e-6), and every correlator against the FP64 GPU path (whose parity
    with the oracle the other tests pin) within the same bar."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("batched")
    cache = {}

    def leaf(li):
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    stream = torch.cuda.current_stream().cuda_stream
    vals = {}
    for precision in ("tf32x3", "fp64"):
        nd, _ = L.build_dag(wl, precision=precision, leaf_data_fn=leaf)
        nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
        if precision != "fp64":
            nd.set_option(L.LQC_OPT_WINDOW, 512)
            nd.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
        planned = nd.schedule("tree", "lru", wl.budget_bytes)
        nd.execute(stream)
        assert nd.stats() == planned
        vals[precision] = {r: nd.read_correlator(r) for r in nd.roots()}
        nd.close()
    od, _ = D.build_from_workload(wl)
    roots = od.roots()
    assert sorted(roots) == sorted(vals["tf32x3"])
    # every correlator against the FP64 path
    e64 = [np.linalg.norm(vals["tf32x3"][r] - vals["fp64"][r]) / np.linalg.norm(vals["fp64"][r])
           for r in roots]
    assert max(e64) < 1e-6, max(e64)
    # 64 seeded roots against the oracle, two or more from every class
    rng = np.random.default_rng(9)
    by_class = {}
    for r in rng.permutation(roots).tolist():
        leafnode = next(u for u in od.tree(r) if od.nodes[u].is_leaf)
        li = od.nodes[leafnode].leaf_index
        by_class.setdefault((wl.leaf_nvec(li), wl.leaf_lt(li)), []).append(r)
    assert len(by_class) >= 10
    pick = [r for rs in by_class.values() for r in rs[:2]]
    rest = [r for r in rng.permutation(roots).tolist() if r not in set(pick)]
    pick += rest[:max(0, 64 - len(pick))]
    assert len(pick) >= 64
    ref = C.evaluate(od, lambda u: leaf(od.nodes[u].leaf_index), pick)
    errs = {r: float(np.linalg.norm(vals["tf32x3"][r] - ref[r]) / np.linalg.norm(ref[r]))
            for r in pick}
    assert max(errs.values()) < 1e-6, max(errs.values())
    e64o = [np.linalg.norm(vals["fp64"][r] - ref[r]) / np.linalg.norm(ref[r]) for r in pick]
    assert max(e64o) < 1e-12, max(e64o)
