"""Pins of the oracle's memory model and budgeted replay (oracle.memory).

* Table 1 of the paper (Sec. II-C) -- the only worked example it prints.
* M_n = 0 (Sec. II-C) and the closed-form interval profile, which computes
  every M_i from tensor lifetimes instead of replaying events.
* A hand-worked eviction example (every op derived below by hand).
* Invariants of budgeted replays on exhaustively enumerated orders, checked
  by an independent op-list validator.
"""
import json
import os

import pytest

from oracle import dag as D
from oracle import memory as M
from oracle.enumerate import topological_orders
from tests.dagutil import random_spec, unit_spec

GOLD = os.path.join(os.path.dirname(__file__), "golden")
UNIT = 16  # bytes of a unit tensor (lt=1, extents of 1, complex128)


def _named_dag(spec):
    names = list(spec["leaves"])
    idx = {n: i for i, n in enumerate(names)}
    contr = []
    for (name, l, r, root) in spec["contractions"]:
        contr.append((idx[l], idx[r], root))
        idx[name] = len(names)
        names.append(name)
    lt, leaves, cs = unit_spec(len(spec["leaves"]), contr)
    return D.from_spec(lt, leaves, cs), idx, names


def test_table1_memory_contents():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    dag, idx, names = _named_dag(g)
    for sname in ("S1", "S2"):
        s = g[sname]
        order = [idx[n] for n in s["order"]]
        assert D.validate_order(dag, order) is None
        sizes, sets = M.model_trace(dag, order)
        assert [x // UNIT for x in sizes] == s["size"]
        rows = s.get("after") or s["after_printed"]
        checked = s.get("rows_checked_as_sets", range(len(rows)))
        for i in checked:
            assert sorted(names[u] for u in sets[i]) == sorted(rows[i]), (sname, i)
        assert M.peak_paper(dag, order) // UNIT == g["peak"][sname]
        # S2 row g: the model's set is {e}, the printed {a} is the typo
    _, sets2 = M.model_trace(dag, [idx[n] for n in g["S2"]["order"]])
    assert sorted(names[u] for u in sets2[2]) == ["e"]


def test_table1_interval_form_agrees():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    dag, idx, _ = _named_dag(g)
    for sname in ("S1", "S2"):
        order = [idx[n] for n in g[sname]["order"]]
        after, during = M.interval_profile(dag, order)
        sizes, _ = M.model_trace(dag, order)
        assert after == sizes
        assert M.replay(dag, order).trace == sizes


@pytest.mark.parametrize("seed", range(40))
def test_closed_form_and_mn_zero_exhaustive(seed):
    lt, leaves, contr = random_spec(seed, n_leaves=4, n_contr=6)
    dag = D.from_spec(lt, leaves, contr)
    count = 0
    for order in topological_orders(dag):
        count += 1
        after, during = M.interval_profile(dag, order)
        sizes, _ = M.model_trace(dag, order)
        assert sizes == after
        assert sizes[-1] == 0                      # M_n = 0
        plan = M.replay(dag, order)               # unlimited budget
        assert plan.trace == after
        assert plan.stats.peak_exec == max(during)
        assert plan.stats.peak_paper == max(after)
        assert plan.stats.n_evict == 0 and plan.stats.d2h_bytes == 0
        assert plan.stats.h2d_bytes == sum(dag.size(u) for u in dag.used_leaves())
    assert count >= 1      # every order of the 10-node DAG (at most 6! of them)


@pytest.mark.parametrize("seed", range(25))
@pytest.mark.parametrize("policy", [M.LRU, M.NEXT_USE])
def test_budgeted_replays_valid(seed, policy):
    lt, leaves, contr = random_spec(100 + seed, n_leaves=4, n_contr=6)
    dag = D.from_spec(lt, leaves, contr)       # 10 nodes: every order
    for order in topological_orders(dag):
        free = M.replay(dag, order)
        need_max = max(sum(dag.size(x) for x in dag.nodes[c].children) + dag.size(c)
                       for c in order)
        # budget at or above the unbudgeted execution peak: identical to the free run
        same = M.replay(dag, order, budget=free.stats.peak_exec, policy=policy)
        assert same.stats.as_tuple() == free.stats.as_tuple()
        assert same.ops == free.ops
        for B in sorted({need_max, (need_max + free.stats.peak_exec) // 2}):
            plan = M.replay(dag, order, budget=B, policy=policy)
            M.check_plan(dag, order, plan, B)
            assert plan.stats.peak_exec <= B
            assert plan.stats.peak_paper == free.stats.peak_paper
            # every byte written back is read back at most as often as it is reloaded
            assert plan.stats.h2d_bytes >= free.stats.h2d_bytes
        with pytest.raises(M.BudgetError):
            M.replay(dag, order, budget=need_max - 1, policy=policy)


def test_eviction_hand_example():
    """Unit tensors a,b,c,d; n4=a.b n5=c.d n6=n4.c n7=n5.a n8=n6.n7 (root)
    n9=n4.d (root); order n4..n9.

    Budget 5, LRU: step n6 needs 1 unit with {a,n4,c,d,n5} resident (5):
    victim among non-operands {a,d,n5}, oldest touch a (step 0).  Step n7
    needs a back (1) + output (1) with {n4,d,n5,n6}: victim among {n4,d,n6},
    oldest d (step 1); a is reloaded.  n9 reloads d.  2 evictions, 6 loads.
    Budget 5, NEXT_USE: at n6 the farthest next use among a (n7, pos 3),
    d (n9, pos 5), n5 (n7, pos 3) is d; afterwards everything fits: 1
    eviction, 5 loads.  Budget 4, LRU: n5 already needs room: a and n4 tie
    at touch 0 -> a (smaller id); n6: d and n5 tie at 1 -> d; n7: n4 and n6
    tie at 2 -> n4, an intermediate with no host copy: written back (D2H)
    and reloaded for n9.  Budget 2: n4 alone needs 3 -> budget error."""
    g = json.load(open(os.path.join(GOLD, "eviction_example.json")))
    dag, idx, names = _named_dag(g)
    order = [idx[n] for n in g["order"]]
    code = {M.LOAD: "L", M.CONTRACT: "C", M.FREE: "F"}
    for case in g["cases"]:
        if case.get("error"):
            with pytest.raises(M.BudgetError):
                M.replay(dag, order, budget=case["budget"] * UNIT, policy=case["policy"])
            continue
        plan = M.replay(dag, order, budget=case["budget"] * UNIT, policy=case["policy"])
        got = []
        for kind, u, flag in plan.ops:
            c = ("W" if flag else "E") if kind == M.EVICT else code[kind]
            got.append("%s %s" % (c, names[u]))
        assert got == case["ops"], case
        st = case["stats"]
        assert plan.stats.peak_paper == st["peak_paper"] * UNIT
        assert plan.stats.peak_exec == st["peak_exec"] * UNIT
        assert plan.stats.n_evict == st["n_evict"]
        assert plan.stats.n_h2d == st["n_h2d"]
        assert plan.stats.n_d2h == st["n_d2h"]
        M.check_plan(dag, order, plan, case["budget"] * UNIT)


def test_planted_mistake_caught():
    """Plant a plausible bug in the oracle (forget to release a root's
    output) and check that the Table 1 pin fails."""
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    dag, idx, names = _named_dag(g)
    order = [idx[n] for n in g["S1"]["order"]]
    saved = [list(nd.parents) for nd in dag.nodes]
    # a root that looks like it has a consumer is never released
    dag.nodes[idx["g"]].parents.append(idx["h"])
    sizes, _ = M.model_trace(dag, order)
    for nd, p in zip(dag.nodes, saved):
        nd.parents = p
    assert [x // UNIT for x in sizes] != g["S1"]["size"]
