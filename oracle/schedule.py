"""Contraction orders: a naive topological baseline, the sibling scheduler
(Sec. III-A, Alg. 1-3), the tree scheduler (Sec. III-B, Alg. 4-8), and two
schedulers the paper only names: a node-based gain scheduler (its stated
future work, Sec. VI) and the similarity ordering of trees it attributes to
Redstar (RS-GS, Sec. II-A).

Each scheduler returns the order of the non-leaf nodes (the contractions).
Leaves "brought to memory" inside a scheduler have no effect on the order;
in the memory model leaves are loaded on first use (Sec. II-C).

Readings where the paper leaves a choice open (all deterministic):
* naive: non-leaf nodes in ascending id (ids are topological by build).
* sibling: the "random" WAITING leaf of Alg. 1 is the smallest-id WAITING
  leaf that has a consumer; queues are FIFO; a node's parents are visited in
  ascending id; children/parents are distinct sets (a contraction of a
  tensor with itself has one distinct child, so rp starts at 1).
* tree: trees T_i are the descendant closures of the roots, indexed by
  ascending root id; ties of max tgain go to the smallest index; the
  initial tgain is the sum of the individual gains (Alg. 5's last loop
  accumulates g(u,T_i), but the text defines tgain as cgain + sum of igain;
  the text is followed); PROCESS-CHILD's "x.outAv = v.outAv - u" is read as
  x.outAv - u; "INMMEM" is INMEM; PROCESS-CTREE visits the nodes of T by a
  post-order walk from the root (left operand first, each node once) and
  skips nodes an earlier tree already processed (their sub-trees too).
* node (one sentence in Sec. VI: a node-based scheduler using the tree
  scheduler's gain concept): at every step, among the contractions whose
  non-leaf inputs are computed, take the one whose processing lowers the
  resident memory of the model (Sec. II-C) the most -- gain = bytes of the
  inputs it releases (it is their last pending consumer) - bytes of the
  leaves it loads - its output bytes (none for a root, released at once);
  ties to the smallest id.
* rsgs (Sec. II-A: trees sorted by similarity, trees sharing contractions
  processed one after the other): start with the first tree (smallest root
  id); next, the unprocessed tree sharing the most contractions (non-leaf
  nodes) with the tree processed last, ties to the smallest index; each
  tree's not yet processed nodes are emitted by the same post-order walk as
  the tree scheduler's.
"""
from __future__ import annotations

import collections
import sys
from typing import Callable, Dict, List, Optional, Tuple

from .dag import Dag

WAITING, QUEUED, INMEM, RELEASED, AVAIL = "WAITING", "QUEUED", "INMEM", "RELEASED", "AVAIL"


def naive(dag: Dag) -> List[int]:
    return dag.non_leaf()


# --------------------------------------------------------------------------
# Sibling scheduler (Alg. 1 SB-SCHEDULER, Alg. 2 SB-PROCESS, Alg. 3 SB-PROP-DOWN)
# --------------------------------------------------------------------------
def ranks(dag: Dag) -> List[int]:
    """Eq. (1): 0 for a leaf, else 1 + the largest child rank."""
    r = [0] * len(dag.nodes)
    for nd in dag.nodes:            # ids are topological
        if not nd.is_leaf:
            r[nd.id] = 1 + max(r[c] for c in nd.children)
    return r


def sibling(dag: Dag) -> List[int]:
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 1_000_000))
    nodes = dag.nodes
    rank = ranks(dag)
    rs = [len(nd.parents) for nd in nodes]
    rp = [len(nd.children) for nd in nodes]
    state = [WAITING] * len(nodes)
    q = max(rank) if rank else 0
    queues: Dict[int, collections.deque] = {i: collections.deque() for i in range(1, q + 1)}
    order: List[int] = []

    def process(u: int):                                    # Alg. 2
        nd = nodes[u]
        if not nd.is_leaf:
            order.append(u)                                 # perform the contraction
        state[u] = INMEM
        if not nd.is_leaf:
            for v in nd.children:
                rs[v] -= 1
                if rs[v] == 0:
                    state[v] = RELEASED
            if not nd.parents:                              # ROOT
                state[u] = RELEASED
        for v in nd.parents:
            rp[v] -= 1
            if rp[v] == 1:
                w = [c for c in nodes[v].children if c != u][0]
                if state[w] == WAITING:
                    prop_down(w)
            elif rp[v] == 0:
                queues[rank[v]].append(v)
                state[v] = QUEUED

    def prop_down(u: int):                                  # Alg. 3
        if state[u] != WAITING:
            return
        nd = nodes[u]
        if nd.is_leaf:
            process(u)
            return
        prop_down(nd.left)
        prop_down(nd.right)

    n_contr = len(dag.non_leaf())
    leaves = [nd.id for nd in nodes if nd.is_leaf and nd.parents]
    leaf_ptr = 0
    while len(order) < n_contr:                             # Alg. 1
        top = next((i for i in range(q, 0, -1) if queues[i]), None)
        if top is None:
            while state[leaves[leaf_ptr]] != WAITING:
                leaf_ptr += 1
            u = leaves[leaf_ptr]
        else:
            u = queues[top].popleft()
        process(u)
    return order


# --------------------------------------------------------------------------
# Tree scheduler (Alg. 4 TR-SCHEDULER .. Alg. 8 PROCESS-NODE)
# --------------------------------------------------------------------------
class TreeState:
    """All fields of Sec. III-B: per node ctree/state/outAv and tau/delta per
    (node, tree); per tree pred, igain, cgain, tgain."""

    def __init__(self, dag: Dag):
        self.dag = dag
        self.roots = dag.roots()
        self.trees: List[List[int]] = [dag.tree(r) for r in self.roots]
        n = len(dag.nodes)
        # TR-INIT (Alg. 5)
        self.outAv: List[set] = [set(nd.parents) for nd in dag.nodes]
        self.ctree: List[List[int]] = [[] for _ in range(n)]
        self.state: List[str] = [AVAIL] * n
        k = len(self.trees)
        self.pred: List[set] = [set() for _ in range(k)]
        self.cgain: List[int] = [0] * k
        self.tgain: List[int] = [0] * k
        for i, T in enumerate(self.trees):
            for u in T:
                self.ctree[u].append(i)
        self.ctree_set = [set(c) for c in self.ctree]
        self.igain: Dict[Tuple[int, int], int] = {}
        g: Dict[Tuple[int, int], int] = {}
        for i, T in enumerate(self.trees):
            for u in T:
                g[(u, i)] = len(self.outAv[u])
        for v, nd in enumerate(dag.nodes):          # edges (u, v)
            for u in nd.children:
                for i in self.ctree[u]:
                    if i in self.ctree_set[v]:
                        g[(u, i)] -= 1
        for (u, i), gv in g.items():
            ig = 0 if gv == 0 else -dag.size(u)
            self.igain[(u, i)] = ig
            self.tgain[i] += ig
        self.tau: Dict[Tuple[int, int], int] = {}
        self.delta: Dict[Tuple[int, int], int] = {}
        self.succ_trees: List[List[int]] = [[] for _ in range(n)]  # trees with x in pred (candidates)

    def process_child(self, u: int, x: int):                   # Alg. 7
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
                if self.delta[(x, i)] == 1:
                    self.cgain[i] += size
                    self.tgain[i] += size
                self.delta[(x, i)] -= 1
        self.outAv[x].discard(u)
        if not self.outAv[x]:
            self.state[x] = RELEASED

    def process_node(self, u: int):                            # Alg. 8
        size = self.dag.size(u)
        for i in self.ctree[u]:
            self.tgain[i] -= self.igain[(u, i)]
        S: List[int] = []
        seen = set()
        n_out = len(self.outAv[u])
        for v in sorted(self.outAv[u]):
            for i in self.ctree[v]:
                if i not in seen:
                    self.tau[(u, i)] = 0
                    self.delta[(u, i)] = n_out
                    seen.add(i)
                    S.append(i)
                    self.pred[i].add(u)
                self.delta[(u, i)] -= 1
                self.tau[(u, i)] += 1
        self.succ_trees[u] = S
        for i in S:
            if self.delta[(u, i)] == 0:
                self.cgain[i] += size
                self.tgain[i] += size
        self.state[u] = RELEASED if not self.outAv[u] else INMEM

    def topo(self, i: int) -> List[int]:
        """Nodes of T_i still AVAIL, children before parents, left first."""
        out: List[int] = []
        seen = set()

        def rec(u):
            if u in seen or self.state[u] != AVAIL:
                return
            seen.add(u)
            nd = self.dag.nodes[u]
            if not nd.is_leaf:
                rec(nd.left)
                rec(nd.right)
            out.append(u)

        rec(self.roots[i])
        return out

    def process_ctree(self, i: int, order: List[int]):          # Alg. 6
        for u in self.topo(i):
            nd = self.dag.nodes[u]
            if not nd.is_leaf:
                for v in nd.children:
                    self.process_child(u, v)
            self.process_node(u)
            if not nd.is_leaf:
                order.append(u)

    def gain_from_scratch(self, i: int) -> int:
        """M - M' of contracting T_i now, recomputed from the node states
        alone (the definition of a tree's gain, Sec. III-B)."""
        dag = self.dag
        Ti = set(self.trees[i])
        avail = [u for u in Ti if self.state[u] == AVAIL]
        stays = sum(dag.size(u) for u in avail
                    if any(p not in Ti for p in dag.nodes[u].parents))
        released = 0
        for x in range(len(dag.nodes)):
            if self.state[x] != INMEM:
                continue
            av = [p for p in dag.nodes[x].parents if self.state[p] == AVAIL]
            if av and all(p in Ti for p in av):
                released += dag.size(x)
        return released - stays


def tree(dag: Dag, check: Optional[Callable[[TreeState, List[int]], None]] = None) -> List[int]:
    """Alg. 4.  ``check(state, remaining)`` is called before every selection
    (test hook for the from-scratch gain invariant)."""
    sys.setrecursionlimit(max(sys.getrecursionlimit(), 1_000_000))
    st = TreeState(dag)
    remaining = list(range(len(st.trees)))
    alive = [True] * len(st.trees)
    order: List[int] = []
    for _ in range(len(st.trees)):
        if check is not None:
            check(st, [i for i in remaining if alive[i]])
        best = -1
        for i in remaining:
            if alive[i] and (best < 0 or st.tgain[i] > st.tgain[best]):
                best = i
        st.process_ctree(best, order)
        alive[best] = False
    return order


# --------------------------------------------------------------------------
# Node-based gain scheduler (Sec. VI, future work; reading in the header)
# --------------------------------------------------------------------------
def node_gain(dag: Dag, u: int, resident, pending) -> int:
    """Bytes by which processing u lowers the resident memory of the model:
    released inputs - loaded leaves - the output (kept unless u is a root)."""
    nd = dag.nodes[u]
    g = 0
    for x in nd.children:
        if dag.nodes[x].is_leaf and x not in resident:
            g -= dag.size(x)
        if pending[x] == 1:          # u is x's last pending consumer
            g += dag.size(x)
    if nd.parents:
        g -= dag.size(u)
    return g


def node(dag: Dag, check: Optional[Callable[[List[int], List[int]], None]] = None) -> List[int]:
    """Greedy by gain over the available contractions, recomputed from the
    definition at every step.  ``check(order_so_far, available)`` runs before
    every selection (test hook)."""
    nodes = dag.nodes
    pending = [len(nd.parents) for nd in nodes]
    resident = set()
    done = [False] * len(nodes)

    def ready(u):
        return all(nodes[c].is_leaf or done[c] for c in nodes[u].children)
    avail = {u for u in dag.non_leaf() if ready(u)}
    order: List[int] = []
    while avail:
        if check is not None:
            check(list(order), sorted(avail))
        best = min(avail, key=lambda u: (-node_gain(dag, u, resident, pending), u))
        avail.discard(best)
        order.append(best)
        done[best] = True
        for x in nodes[best].children:
            if nodes[x].is_leaf:
                resident.add(x)
            pending[x] -= 1
            if pending[x] == 0:
                resident.discard(x)
        if nodes[best].parents:
            resident.add(best)
        for p in nodes[best].parents:
            if not done[p] and ready(p):
                avail.add(p)
    return order


# --------------------------------------------------------------------------
# RS-GS: trees ordered by similarity (Sec. II-A; reading in the header)
# --------------------------------------------------------------------------
def _post_order(dag: Dag, root: int, done, out: List[int]) -> None:
    stack = [(root, False)]
    while stack:
        u, expanded = stack.pop()
        nd = dag.nodes[u]
        if nd.is_leaf or done[u]:
            continue
        if expanded:
            done[u] = True
            out.append(u)
            continue
        stack.append((u, True))
        for c in reversed(nd.children):   # left operand first
            stack.append((c, False))


def rsgs(dag: Dag) -> List[int]:
    roots = dag.roots()
    contr = [set(u for u in dag.tree(r) if not dag.nodes[u].is_leaf) for r in roots]
    done = [False] * len(dag.nodes)
    used = [False] * len(roots)
    order: List[int] = []
    cur = 0 if roots else -1
    while cur >= 0:
        used[cur] = True
        _post_order(dag, roots[cur], done, order)
        best, best_shared = -1, -1
        for j in range(len(roots)):
            if not used[j]:
                shared = len(contr[cur] & contr[j])
                if shared > best_shared:
                    best, best_shared = j, shared
        cur = best
    return order


SCHEDULERS = {"naive": naive, "sibling": sibling, "tree": tree, "node": node, "rsgs": rsgs}
