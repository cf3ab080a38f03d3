"""Contraction-path selection (Sec. II-A, the step Redstar runs before the
scheduler): the terms of the correlation functions are graphs -- vertices
are tensors, edges are index pairs -- and each is reduced to one vertex by
binary contractions.  Redstar counts how often each edge occurs across all
contraction trees and weighs it with the cost of its contraction,
preferring edges that recur and contractions that are expensive, so that a
costly contraction is done once and reused.

Test infrastructure only: never imported by the library.

Reading used (the paper gives the idea in prose only):
* a candidate of a graph is a pair of its current vertices joined by at
  least one edge; contracting it pairs every edge between the two.  Its key
  is the DAG's merge key: (left node, right node, left axes, right axes),
  left = the vertex whose tensor has more elements (the paper leaves the
  orientation open; this one puts the larger free extent on the output's
  rows, M >= N), ties to the smaller node id, then to the vertex whose axis
  labels come first; pairs sorted by the left axis;
* value of a key = (number of graphs holding a candidate with that key) x
  (complex multiply-adds of the contraction, Lt * M * N * K); outputs with
  more elements than the graph's largest input tensor are not candidates
  unless the graph has no other;
* each step takes the key of largest value (ties: the smallest key) and
  contracts it in every graph that holds it (repeatedly, first pair first,
  while the graph still does); identical contractions of different graphs
  thus become one DAG node;
* a graph is done when one vertex is left: its root.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from .dag import Dag

Edge = Tuple[int, int, int, int]


class _Vertex:
    def __init__(self, node: int, labels):
        self.node = node
        self.labels = list(labels)      # (item, axis) of every axis, in axis order


def _candidate(dag: Dag, p: _Vertex, q: _Vertex, partner):
    """(key, cost, out_elems, left, right) of contracting p with q, or None."""
    qpos = {lab: j for j, lab in enumerate(q.labels)}
    pairs = [(i, qpos[partner[lab]]) for i, lab in enumerate(p.labels)
             if partner.get(lab) in qpos]
    if not pairs:
        return None
    pe = int(np.prod(dag.nodes[p.node].extents, dtype=np.int64))
    qe = int(np.prod(dag.nodes[q.node].extents, dtype=np.int64))
    if (-pe, p.node, min(p.labels)) <= (-qe, q.node, min(q.labels)):
        left, right, lr = p, q, pairs
    else:
        left, right, lr = q, p, [(j, i) for (i, j) in pairs]
    lr = sorted(lr)
    la = tuple(i for i, _ in lr)
    ra = tuple(j for _, j in lr)
    le, re_ = dag.nodes[left.node].extents, dag.nodes[right.node].extents
    k = int(np.prod([le[i] for i in la], dtype=np.int64))
    m = int(np.prod(le, dtype=np.int64)) // k
    n = int(np.prod(re_, dtype=np.int64)) // k
    cost = dag.nodes[left.node].lt * m * n * k
    return (left.node, right.node, la, ra), cost, m * n, left, right


def select_paths(dag: Dag, graphs: Sequence[Tuple[Sequence[int], Sequence[Edge]]]) -> List[int]:
    """Add the contractions of every graph to ``dag``; graph g's vertices are
    existing node ids, its edges (vertex a, axis a, vertex b, axis b) local
    indices.  Returns each graph's root node id."""
    state = []
    for nodes, edges in graphs:
        verts = [_Vertex(u, [(i, a) for a in range(len(dag.nodes[u].extents))])
                 for i, u in enumerate(nodes)]
        partner = {}
        for (va, aa, vb, ab) in edges:
            partner[(va, aa)] = (vb, ab)
            partner[(vb, ab)] = (va, aa)
        cap = max(int(np.prod(dag.nodes[u].extents, dtype=np.int64)) for u in nodes)
        state.append((verts, partner, cap))

    def candidates(g):
        verts, partner, cap = state[g]
        out = []
        for x in range(len(verts)):
            for y in range(x + 1, len(verts)):
                c = _candidate(dag, verts[x], verts[y], partner)
                if c is not None:
                    out.append((x, y) + c)
        ok = [c for c in out if c[4] <= cap]
        return ok if ok else out

    while True:
        count, cost = {}, {}
        for g in range(len(state)):
            if len(state[g][0]) < 2:
                continue
            cands = candidates(g)
            for key in {c[2] for c in cands}:
                count[key] = count.get(key, 0) + 1
            for c in cands:
                cost[c[2]] = c[3]
        if not count:
            break
        best = min(count, key=lambda kk: (-count[kk] * cost[kk], kk))
        for g in range(len(state)):
            verts, partner, cap = state[g]
            while True:
                hit = [c for c in candidates(g) if c[2] == best]
                if not hit:
                    break
                x, y, key, _, _, left, right = hit[0]
                node = dag.add_contraction(key[0], key[1], key[2], key[3])
                labels = [lab for i, lab in enumerate(left.labels) if i not in key[2]] + \
                    [lab for j, lab in enumerate(right.labels) if j not in key[3]]
                verts[x] = _Vertex(node, labels)
                del verts[y]
    roots = []
    for verts, _, _ in state:
        if len(verts) != 1:
            raise ValueError("a graph is not connected")
        roots.append(verts[0].node)
    return roots


def build_with_paths(wl, elem_bytes: int = 16):
    """Oracle DAG of a synth.Workload built from its graphs by path selection
    (leaves first, as registered by the workload).  Returns (dag, roots)."""
    dag = Dag(wl.lt, elem_bytes)
    for li, lf in enumerate(wl.leaves):
        dag.add_leaf(lf.extents, leaf_index=li, lt=wl.leaf_lt(li))
    roots = select_paths(dag, [([items[v] for v in range(len(items))], edges)
                               for items, edges in wl.graphs])
    return dag, roots
