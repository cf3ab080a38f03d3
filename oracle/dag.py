"""Contraction DAG as defined in Sec. II-B ("Notation") of the paper.

Nodes are leaves (a tensor only) or binary contractions (a contraction and its
output tensor).  Node types follow the paper: LEAF (no inputs), ROOT (no
consumers; one per contraction tree) and INTERIOR (the rest).  Trees are the
descendant closures of the roots.  Identical requests -- same operand nodes,
same contracted axis pairs -- are merged into one node, which is how the
contraction trees of many correlation functions share nodes and edges.

Edge weights w(u, v) = u.size are not stored separately: a consumer reads the
operand's size.  Children and parents are *sets* of distinct nodes (a request
that contracts a tensor with itself has one distinct child).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Tuple

LEAF, INTERIOR, ROOT = "LEAF", "INTERIOR", "ROOT"


@dataclasses.dataclass
class Node:
    id: int
    extents: Tuple[int, ...]
    left: int = -1
    right: int = -1
    la: Tuple[int, ...] = ()
    ra: Tuple[int, ...] = ()
    parents: List[int] = dataclasses.field(default_factory=list)  # distinct, ascending
    leaf_index: int = -1    # index into the workload's leaf list
    lt: int = 1             # batch (time-slice) extent, never contracted

    @property
    def is_leaf(self) -> bool:
        return self.left < 0

    @property
    def children(self) -> List[int]:
        if self.is_leaf:
            return []
        return [self.left] if self.left == self.right else [self.left, self.right]


class Dag:
    def __init__(self, lt: int, elem_bytes: int = 16):
        self.lt = lt
        self.elem_bytes = elem_bytes
        self.nodes: List[Node] = []
        self._index: Dict[Tuple, int] = {}

    # -- building ---------------------------------------------------------
    def add_leaf(self, extents, leaf_index: int = -1, lt: Optional[int] = None) -> int:
        """A leaf with batch extent ``lt`` (default: the DAG's)."""
        nid = len(self.nodes)
        self.nodes.append(Node(nid, tuple(int(e) for e in extents), leaf_index=leaf_index,
                               lt=int(lt if lt is not None else self.lt)))
        return nid

    def add_contraction(self, left: int, right: int, la, ra) -> int:
        la, ra = tuple(int(a) for a in la), tuple(int(a) for a in ra)
        key = (left, right, la, ra)
        if key in self._index:
            return self._index[key]
        L, R = self.nodes[left], self.nodes[right]
        if len(la) != len(ra) or len(set(la)) != len(la) or len(set(ra)) != len(ra):
            raise ValueError("bad axis pairs")
        for a, b in zip(la, ra):
            if L.extents[a] != R.extents[b]:
                raise ValueError("paired axes differ in extent")
        if L.lt != R.lt:
            raise ValueError("operands differ in the batch extent")
        ext = tuple(e for i, e in enumerate(L.extents) if i not in la) + \
            tuple(e for j, e in enumerate(R.extents) if j not in ra)
        nid = len(self.nodes)
        self.nodes.append(Node(nid, ext, left, right, la, ra, lt=L.lt))
        for c in sorted({left, right}):
            self.nodes[c].parents.append(nid)
        self._index[key] = nid
        return nid

    # -- queries ----------------------------------------------------------
    def size(self, u: int) -> int:
        """u.size: bytes of the tensor, its own batch axis included."""
        n = self.nodes[u].lt * self.elem_bytes
        for e in self.nodes[u].extents:
            n *= e
        return n

    def type(self, u: int) -> str:
        nd = self.nodes[u]
        if nd.is_leaf:
            return LEAF
        return ROOT if not nd.parents else INTERIOR

    def non_leaf(self) -> List[int]:
        return [n.id for n in self.nodes if not n.is_leaf]

    def roots(self) -> List[int]:
        return [n.id for n in self.nodes if not n.is_leaf and not n.parents]

    def used_leaves(self) -> List[int]:
        return [n.id for n in self.nodes if n.is_leaf and n.parents]

    def tree(self, root: int) -> List[int]:
        """Descendant closure of a root (nodes of contraction tree T_root)."""
        seen, stack = set(), [root]
        while stack:
            u = stack.pop()
            if u in seen:
                continue
            seen.add(u)
            stack.extend(self.nodes[u].children)
        return sorted(seen)


def build_from_workload(wl, elem_bytes: int = 16) -> Tuple[Dag, List[int]]:
    """Build the DAG from a synth.Workload request stream.

    Returns the DAG and the map from stream index to node id.
    """
    dag = Dag(wl.lt, elem_bytes)
    ids: List[int] = []
    for li, lf in enumerate(wl.leaves):
        ids.append(dag.add_leaf(lf.extents, leaf_index=li, lt=wl.leaf_lt(li)))
    for rq in wl.requests:
        ids.append(dag.add_contraction(ids[rq.left], ids[rq.right], rq.la, rq.ra))
    return dag, ids


def from_spec(lt: int, leaves, contractions, elem_bytes: int = 16) -> Dag:
    """Small hand-written DAGs: ``leaves`` = list of extents tuples,
    ``contractions`` = list of (left, right, la, ra) over node ids."""
    dag = Dag(lt, elem_bytes)
    for i, ext in enumerate(leaves):
        dag.add_leaf(ext, leaf_index=i)
    for (l, r, la, ra) in contractions:
        dag.add_contraction(l, r, la, ra)
    return dag


def validate_order(dag: Dag, order) -> Optional[str]:
    """None if ``order`` lists every non-leaf node once, children first."""
    pos = {}
    for i, u in enumerate(order):
        if dag.nodes[u].is_leaf:
            return "leaf %d in order" % u
        if u in pos:
            return "node %d twice" % u
        pos[u] = i
    if set(pos) != set(dag.non_leaf()):
        return "order does not cover the non-leaf nodes"
    for u in order:
        for c in dag.nodes[u].children:
            if not dag.nodes[c].is_leaf and pos[c] > pos[u]:
                return "node %d before its child %d" % (u, c)
    return None
