"""The native schedulers and planner (C ABI) against the oracle, bit-exact.

* orders of naive / sibling / tree identical to the oracle's on random DAGs
  and on every synthetic workload;
* planned op lists and every figure (peak_paper, peak_exec, evictions,
  H2D/D2H counts and bytes) identical to the oracle's replay, for every
  topological order of tiny DAGs (exhaustive enumeration) under several
  budgets and both eviction policies;
* DAG build: merging of identical requests gives the oracle's node ids.
No GPU is needed: leaves are registered without data.
"""
import pytest

import synth
from oracle import dag as D
from oracle import memory as M
from oracle import schedule as S
from oracle.enumerate import topological_orders
from tests.dagutil import random_spec

L = pytest.importorskip("paper_2511_02257_b300")

POL = {"naive": "naive", "sibling": "sibling", "tree": "tree", "node": "node", "rsgs": "rsgs"}
EV = {M.LRU: "lru", M.NEXT_USE: "next_use"}
STAT_KEYS = ("peak_paper", "peak_exec", "n_evict", "n_h2d", "n_d2h", "h2d_bytes", "d2h_bytes")


def native_from_spec(lt, leaves, contr):
    d = L.Dag(lt)
    for ext in leaves:
        d.add_leaf(ext)
    for (l, r, la, ra) in contr:
        d.add_contraction(l, r, la, ra)
    return d


def stats_tuple(st):
    return tuple(st[k] for k in STAT_KEYS)


def test_library_exports_every_header_symbol():
    import ctypes
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "lqc.h")).read()
    names = set(re.findall(r"^\s*(?:int|int64_t|const char\*)\s+(lqc_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 25
    lib = ctypes.CDLL(L.library_path)
    for n in sorted(names):
        assert hasattr(lib, n), n


@pytest.mark.parametrize("seed", range(30))
def test_dedup_ids_match_oracle(seed):
    lt, leaves, contr = random_spec(seed, n_leaves=5, n_contr=12)
    contr = contr + contr[: len(contr) // 2]   # repeated requests merge
    od = D.from_spec(lt, leaves, contr)
    nd = native_from_spec(lt, leaves, contr)
    assert nd.num_nodes() == len(od.nodes)
    for u in range(len(od.nodes)):
        info = nd.node_info(u)
        assert info["size"] == od.size(u)
        assert info["is_leaf"] == od.nodes[u].is_leaf
        assert info["rank"] == len(od.nodes[u].extents)


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("sched", ["naive", "sibling", "tree", "node", "rsgs"])
def test_orders_bit_exact_random(seed, sched):
    lt, leaves, contr = random_spec(500 + seed, n_leaves=6, n_contr=16, share=0.7)
    od = D.from_spec(lt, leaves, contr)
    nd = native_from_spec(lt, leaves, contr)
    nd.schedule(POL[sched])
    assert nd.order() == S.SCHEDULERS[sched](od)


@pytest.mark.parametrize("name", ["tiny", "multi_meson", "memory_pressure", "baryon"])
def test_orders_and_plans_bit_exact_workloads(name):
    wl = synth.make_workload(name)
    od, _ = D.build_from_workload(wl)
    nd, ids = L.build_dag(wl, with_data=False)
    assert nd.num_nodes() == len(od.nodes)
    budget = wl.budget_bytes or None
    for sched in ("naive", "sibling", "tree", "node", "rsgs"):
        order = S.SCHEDULERS[sched](od)
        for pol in (M.LRU, M.NEXT_USE):
            st = nd.schedule(POL[sched], EV[pol], budget or 0)
            assert nd.order() == order, (name, sched)
            plan = M.replay(od, order, budget=budget, policy=pol)
            assert stats_tuple(st) == plan.stats.as_tuple(), (name, sched, pol)
            got = nd.plan()
            assert len(got) == len(plan.ops)
            assert got == [(k, u, f) for (k, u, f) in plan.ops]


@pytest.mark.parametrize("seed", range(40))
def test_plans_bit_exact_exhaustive(seed):
    # 10 nodes: every topological order of the contractions, no cap
    lt, leaves, contr = random_spec(2000 + seed, n_leaves=4, n_contr=6, share=0.6)
    od = D.from_spec(lt, leaves, contr)
    nd = native_from_spec(lt, leaves, contr)
    n_orders = 0
    for order in topological_orders(od):
        n_orders += 1
        free = M.replay(od, order)
        need = max(sum(od.size(x) for x in od.nodes[c].children) + od.size(c) for c in order)
        for budget in sorted({None, need, (need + free.stats.peak_exec) // 2}, key=lambda b: b or 0):
            for pol in (M.LRU, M.NEXT_USE):
                plan = M.replay(od, order, budget=budget, policy=pol)
                st = nd.set_order(order, EV[pol], budget or 0)
                assert stats_tuple(st) == plan.stats.as_tuple()
                assert nd.plan() == [(k, u, f) for (k, u, f) in plan.ops]
        # one byte below the largest single-step need: budget error on both sides
        with pytest.raises(M.BudgetError):
            M.replay(od, order, budget=need - 1)
        with pytest.raises(L.LqcError) as ei:
            nd.set_order(order, "lru", need - 1)
        assert ei.value.code == L.LQC_ERR_BUDGET
    assert n_orders == sum(1 for _ in topological_orders(od))


def test_table1_schedules_native():
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))
    from tests.test_oracle_memory import _named_dag, UNIT
    od, idx, names = _named_dag(g)
    lt = 1
    nd = native_from_spec(lt, [od.nodes[u].extents for u in range(4)],
                          [(od.nodes[u].left, od.nodes[u].right, od.nodes[u].la, od.nodes[u].ra)
                           for u in range(4, len(od.nodes))])
    for sname in ("S1", "S2"):
        st = nd.set_order([idx[n] for n in g[sname]["order"]])
        assert st["peak_paper"] // UNIT == g["peak"][sname]
    h = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_traces.json")))
    nd.schedule("sibling")
    assert [names[u] for u in nd.order()] == h["sibling"]["order"]
    nd.schedule("tree")
    assert [names[u] for u in nd.order()] == h["tree"]["order"]
    for sched in ("node", "rsgs"):
        nd.schedule(sched)
        assert [names[u] for u in nd.order()] == h[sched]["order"]


def test_argument_errors():
    d = L.Dag(2)
    a = d.add_leaf((3, 4))
    b = d.add_leaf((4, 5))
    with pytest.raises(L.LqcError) as ei:
        d.add_contraction(a, b, [0], [0])      # extents 3 vs 4
    assert ei.value.code == L.LQC_ERR_ARG
    with pytest.raises(L.LqcError):
        d.add_contraction(a, 7, [1], [0])      # no such node
    with pytest.raises(L.LqcError):
        d.add_contraction(a, b, [1, 1], [0, 0])  # axis paired twice
    c = d.add_contraction(a, b, [1], [0])
    assert d.add_contraction(a, b, [1], [0]) == c   # identical request merged
    with pytest.raises(L.LqcError) as ei:
        d.execute()
    assert ei.value.code == L.LQC_ERR_STATE
    with pytest.raises(L.LqcError) as ei:
        d.order()
    assert ei.value.code == L.LQC_ERR_STATE
    d.schedule("tree")
    with pytest.raises(L.LqcError) as ei:
        d.add_leaf((2,))                        # frozen after scheduling
    assert ei.value.code == L.LQC_ERR_STATE
    with pytest.raises(L.LqcError):
        d.set_order([c, c])


def test_size_limits_without_overflow():
    """Sizes are checked before they are multiplied: a slice holds at most
    2^40 elements, a tensor at most 2^58, the batch extent is below 2^31;
    rank-8 extents near 2^31 are rejected instead of wrapping around."""
    with pytest.raises(L.LqcError):
        L.Dag(1 << 31)
    d = L.Dag(1)
    with pytest.raises(L.LqcError) as ei:
        d.set_batch(1 << 31)
    assert ei.value.code == L.LQC_ERR_ARG
    big = [(1 << 31)] * 8                      # product 2^248 per slice
    with pytest.raises(L.LqcError) as ei:
        d.add_leaf(big)
    assert ei.value.code == L.LQC_ERR_ARG
    a = d.add_leaf([1 << 20, 1 << 19, 2])      # 2^40 elements: at the limit
    b = d.add_leaf([2, 1 << 20, 1 << 19])
    ok = d.add_contraction(a, b, [0, 1], [1, 2])  # valid pairing, 2 x 2 output
    assert d.node_info(ok)["rank"] == 2
    with pytest.raises(L.LqcError) as ei:      # paired over the 2s only: 2^78 elements
        d.add_contraction(a, b, [2], [0])
    assert ei.value.code == L.LQC_ERR_ARG
    assert "output too large" in str(ei.value)
    d.set_batch(1 << 20)
    with pytest.raises(L.LqcError) as ei:      # 2^20 slices x 2^40 elements
        d.add_leaf([1 << 20, 1 << 20])
    assert ei.value.code == L.LQC_ERR_ARG
    d.add_leaf([1 << 19, 1 << 19])             # 2^20 x 2^38 = 2^58: at the limit


@pytest.mark.parametrize("sched", ["tree", "rsgs", "sibling", "node"])
def test_orders_bit_exact_large_dag(sched):
    """A 9.5k-vertex DAG (3,580 trees, a leaf with 487 consumers):
    the native schedulers' incremental bookkeeping (threshold buckets,
    indexed heap, touched-tree scans) gives the oracle's orders."""
    wl = synth.make_workload("multi_meson", n_functions=1000)
    od, _ = D.build_from_workload(wl)
    nd, _ = L.build_dag(wl, with_data=False)
    nd.schedule(sched, "lru", 0)
    assert nd.order() == S.SCHEDULERS[sched](od)


@pytest.mark.parametrize("name", ["tiny", "multi_meson", "baryon", "batched"])
def test_bulk_contractions_equal_single_calls(name):
    """lqc_dag_add_contractions (one call for the request stream, operands
    of earlier requests given as back-references) builds the DAG that one
    lqc_dag_add_contraction per request builds: same ids, operands, sizes."""
    kw = {} if name == "tiny" else dict(n_functions=20) if name != "batched" else \
        dict(n_dags=3, nvecs=(8, 12), lts=(2, 3), n_functions=6)
    wl = synth.make_workload(name, **kw)
    bulk, ids_b = L.build_dag(wl, with_data=False)
    one = L.Dag(wl.lt)
    ids = [one.add_leaf(lf.extents, lt=wl.leaf_lt(i)) for i, lf in enumerate(wl.leaves)]
    for rq in wl.requests:
        ids.append(one.add_contraction(ids[rq.left], ids[rq.right], rq.la, rq.ra))
    assert ids_b == ids and bulk.num_nodes() == one.num_nodes()
    for u in range(one.num_nodes()):
        assert bulk.node_operands(u) == one.node_operands(u)
        assert bulk.node_info(u) == one.node_info(u)


def test_bulk_contractions_errors_leave_dag_unchanged():
    """A failing request anywhere in a bulk call (here the second, whose
    paired extents differ) or a reference to a later request leaves the DAG
    as it was; identical requests within one call merge."""
    d = L.Dag(2)
    a = d.add_leaf((3, 4))
    b = d.add_leaf((4, 5))
    n0 = d.num_nodes()
    with pytest.raises(L.LqcError) as ei:
        # request 0: A.B -> (3, 5); request 1 pairs its axis 0 (3) with A's axis 1 (4)
        d.add_contractions([(a, b, [1], [0]), (-1, a, [0], [1])])
    assert ei.value.code == L.LQC_ERR_ARG and d.num_nodes() == n0
    with pytest.raises(L.LqcError) as ei:
        d.add_contractions([(-2, b, [1], [0]), (a, b, [1], [0])])
    assert ei.value.code == L.LQC_ERR_ARG and d.num_nodes() == n0
    ids = d.add_contractions([(a, b, [1], [0]), (a, b, [1], [0]), (-2, -1, [0], [0])])
    assert ids[0] == ids[1] == n0 and ids[2] == n0 + 1
    assert d.node_operands(ids[2]) == (n0, n0, (0,), (0,))


def test_add_contractions_rejects_extreme_back_references():
    """Operand ids below -(i) (no earlier request of the call), down to
    INT64_MIN, are argument errors and leave the DAG unchanged."""
    d = L.Dag(2)
    a = d.add_leaf((3, 3))
    n0 = d.num_nodes()
    for bad in (-(2 ** 63), -(2 ** 63) + 1, -2, -1):
        with pytest.raises(L.LqcError) as ei:
            d.add_contractions([(a, bad, [1], [0])])
        assert ei.value.code == L.LQC_ERR_ARG
        assert d.num_nodes() == n0
    ab = d.add_contractions([(a, a, [1], [0]), (-1, a, [1], [0])])
    assert ab == [n0, n0 + 1]
