"""Pins of the oracle schedulers (oracle.schedule).

* Hand traces of Alg. 1-3 (sibling) and Alg. 4-8 (tree) on the Table 1 DAG.
* The tree scheduler's incrementally maintained gains equal the gains
  recomputed from scratch (the definition M - M' of Sec. III-B) before every
  selection.
* Every order is a valid topological order covering each contraction once;
  the sibling scheduler processes every node exactly once (Sec. III-A).
* Peaks are never below the exhaustive optimum; on tiny DAGs the tree
  scheduler's peak is compared with that optimum.
* Node-based gain scheduler: hand trace on the Table 1 DAG; before every
  selection, the chosen node is the available one whose step lowers the
  memory model's M the most, with M recomputed by the model itself
  (oracle.memory.model_trace on the prefix plus the candidate); a planted
  sign mistake in the gain is caught.
* Similarity order of trees (RS-GS): hand trace on the Table 1 DAG and a
  constructed DAG whose tree sequence is fixed by inspection.
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
@pytest.mark.parametrize("sched", ["naive", "sibling", "tree", "node", "rsgs"])
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
    for s in ("naive", "sibling", "tree", "node", "rsgs"):
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


def test_node_and_rsgs_hand_traces():
    g = json.load(open(os.path.join(GOLD, "table1.json")))
    h = json.load(open(os.path.join(GOLD, "hand_traces.json")))
    dag, idx, names = _named_dag(g)
    order = S.node(dag)
    assert [names[u] for u in order] == h["node"]["order"]
    sizes, _ = M.model_trace(dag, order)
    assert [x // UNIT for x in sizes] == h["node"]["sizes"]
    assert [names[u] for u in S.rsgs(dag)] == h["rsgs"]["order"]
    ex = json.load(open(os.path.join(GOLD, "rsgs_example.json")))
    dag2 = D.from_spec(1, [(1, 1)] * ex["leaves"],
                       [(l, r, tuple(la), tuple(ra)) for (l, r, la, ra) in ex["contractions"]])
    assert S.rsgs(dag2) == ex["rsgs_order"]


def _node_check_via_model(dag, expected):
    """Independent of node_gain: the step that lowers M the most, M taken
    from the memory model's own trace."""
    def check(prefix, avail):
        base = M.model_trace(dag, prefix)[0][-1] if prefix else 0
        delta = {v: M.model_trace(dag, prefix + [v])[0][-1] - base for v in avail}
        expected.append(min(avail, key=lambda v: (delta[v], v)))
    return check


@pytest.mark.parametrize("seed", range(30))
def test_node_choice_lowers_model_memory_most(seed):
    lt, leaves, contr = random_spec(3000 + seed, n_leaves=6, n_contr=14, share=0.6)
    dag = D.from_spec(lt, leaves, contr)
    expected = []
    order = S.node(dag, check=_node_check_via_model(dag, expected))
    assert order == expected
    assert D.validate_order(dag, order) is None


def test_node_choice_on_workload_prefix():
    wl = synth.make_workload("tiny", seed=1)
    dag, _ = D.build_from_workload(wl)
    expected = []
    assert S.node(dag, check=_node_check_via_model(dag, expected)) == expected


def test_planted_node_gain_mistake_caught(monkeypatch):
    """Plant a plausible bug (the output size counted with the wrong sign)
    and check that the model-based pin catches it."""
    orig = S.node_gain

    def buggy(dag, u, resident, pending):
        g = orig(dag, u, resident, pending)
        return g + 2 * dag.size(u) if dag.nodes[u].parents else g
    monkeypatch.setattr(S, "node_gain", buggy)
    caught = 0
    for seed in range(10):
        lt, leaves, contr = random_spec(3000 + seed, n_leaves=6, n_contr=14, share=0.6)
        dag = D.from_spec(lt, leaves, contr)
        expected = []
        if S.node(dag, check=_node_check_via_model(dag, expected)) != expected:
            caught += 1
    assert caught > 0
