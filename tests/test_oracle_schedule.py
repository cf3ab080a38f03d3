"""Pins of the oracle schedulers (oracle.schedule).

* Hand traces of Alg. 1-3 (sibling) and Alg. 4-8 (tree) on the Table 1 DAG.
* The tree scheduler's incrementally maintained gains equal the gains
  recomputed from scratch (the definition M - M' of Sec. III-B) before every
  selection.
* Every order is a valid topological order covering each contraction once;
  the sibling scheduler processes every node exactly once (Sec. III-A).
* Peaks are never below the exhaustive optimum; on tiny DAGs the tree
  scheduler's peak is compared with that optimum.
"""
import json
import os

import pytest

import synth
from oracle import dag as D
from oracle import memory as M
from oracle import schedule as S
from oracle.enumerate import topological_orders
from tests.dagutil import random_spec
from tests.test_oracle_memory import GOLD, UNIT, _named_dag


def test_hand_traces_table1_dag():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    h = json.load(open(os.path.join(GOLD, "hand_traces.json")))
    dag, idx, names = _named_dag(g)
    sib = S.sibling(dag)
    assert [names[u] for u in sib] == h["sibling"]["order"]
    seen = []

    def check(st, remaining):
        seen.append({names[st.roots[i]]: st.tgain[i] // UNIT for i in remaining})

    tr = S.tree(dag, check=check)
    assert [names[u] for u in tr] == h["tree"]["order"]
    assert seen[0] == h["tree"]["initial_tgain"]
    assert seen[1] == h["tree"]["tgain_after_first_tree"]
    assert seen[2] == h["tree"]["tgain_after_second_tree"]
    assert M.peak_paper(dag, sib) // UNIT == h["peaks"]["sibling"]
    assert M.peak_paper(dag, tr) // UNIT == h["peaks"]["tree"]


def _gain_check(st, remaining):
    for i in remaining:
        assert st.tgain[i] == st.gain_from_scratch(i), (i, st.tgain[i], st.gain_from_scratch(i))
        assert st.tgain[i] == st.cgain[i] + sum(
            st.igain[(u, i)] for u in st.trees[i] if st.state[u] == S.AVAIL)
    # tau + delta = |outAv| for every INMEM node and tree it precedes
    # (the paper maintains tau/delta only while u is in T_i.pred)
    for (u, i), t in st.tau.items():
        if st.state[u] == S.INMEM and u in st.pred[i]:
            assert t + st.delta[(u, i)] == len(st.outAv[u])


@pytest.mark.parametrize("seed", range(60))
def test_tree_gains_match_from_scratch_random(seed):
    lt, leaves, contr = random_spec(seed, n_leaves=6, n_contr=14, share=0.7)
    dag = D.from_spec(lt, leaves, contr)
    order = S.tree(dag, check=_gain_check)
    assert D.validate_order(dag, order) is None


@pytest.mark.parametrize("name", ["tiny", "multi_meson"])
def test_tree_gains_match_from_scratch_workloads(name):
    wl = synth.make_workload(name, n_functions=40) if name != "tiny" else synth.make_workload(name)
    dag, _ = D.build_from_workload(wl)
    order = S.tree(dag, check=_gain_check)
    assert D.validate_order(dag, order) is None


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("sched", ["naive", "sibling", "tree"])
def test_orders_valid_and_not_below_optimum(seed, sched):
    lt, leaves, contr = random_spec(1000 + seed, n_leaves=4, n_contr=7)
    dag = D.from_spec(lt, leaves, contr)
    order = S.SCHEDULERS[sched](dag)
    assert D.validate_order(dag, order) is None
    best = min(M.peak_paper(dag, o) for o in topological_orders(dag))
    assert M.peak_paper(dag, order) >= best


def test_sibling_processes_each_node_once():
    wl = synth.make_workload("multi_meson", n_functions=30)
    dag, _ = D.build_from_workload(wl)
    order = S.sibling(dag)
    assert len(order) == len(set(order)) == len(dag.non_leaf())


@pytest.mark.parametrize("name", ["multi_meson", "memory_pressure", "baryon"])
def test_workload_orders_valid(name):
    wl = synth.make_workload(name)
    dag, _ = D.build_from_workload(wl)
    for s in ("naive", "sibling", "tree"):
        assert D.validate_order(dag, S.SCHEDULERS[s](dag)) is None


def test_tree_beats_naive_on_level_emitted_workloads():
    """The paper's claim (Sec. IV-B): the tree scheduler lowers the peak of
    the model relative to a structure-blind order."""
    for name in ("multi_meson", "memory_pressure"):
        wl = synth.make_workload(name)
        dag, _ = D.build_from_workload(wl)
        assert M.peak_paper(dag, S.tree(dag)) < M.peak_paper(dag, S.naive(dag))


def test_planted_gain_mistake_caught():
    """Plant a plausible bug (case 2a of PROCESS-CHILD adds nothing) and
    check that the from-scratch gain pin catches it."""
    orig = S.TreeState.process_child

    def buggy(self, u, x):
        size = self.dag.size(x)
        for i in self.succ_trees[x]:
            if x not in self.pred[i]:
                continue
            if i in self.ctree_set[u]:
                if self.tau[(x, i)] == 1 and self.delta[(x, i)] == 0:
                    self.cgain[i] -= size
                    self.tgain[i] -= size
                self.tau[(x, i)] -= 1
                if self.tau[(x, i)] == 0:
                    self.pred[i].discard(x)
            else:
                self.delta[(x, i)] -= 1
        self.outAv[x].discard(u)
        if not self.outAv[x]:
            self.state[x] = S.RELEASED

    S.TreeState.process_child = buggy
    try:
        caught = False
        for seed in range(30):
            lt, leaves, contr = random_spec(seed, n_leaves=6, n_contr=14, share=0.7)
            dag = D.from_spec(lt, leaves, contr)
            try:
                S.tree(dag, check=_gain_check)
            except AssertionError:
                caught = True
                break
        assert caught
    finally:
        S.TreeState.process_child = orig
