"""Correlator values, computed two independent ways on the CPU in complex128.

1. ``evaluate``: node by node in id order.  Each binary contraction is, for
   every time slice t separately, ``numpy.tensordot`` of the two operands over
   the paired axes -- the textbook definition of a tensor contraction, whose
   output axes are the left operand's free axes followed by the right
   operand's, exactly the node convention.  The batch axis t is never
   contracted and slices never mix (a correlation function is computed per
   time slice).  A rank-0 output is the contract-all of a root: one complex
   number per time slice.

2. ``brute_force``: the whole tree of a root expanded into one sum over every
   index label at once (``numpy.einsum`` without path optimisation), with no
   intermediates.  Only feasible on tiny inputs; it pins ``evaluate``.

The paper itself leaves the contraction arithmetic to Redstar's Hadron
library (Sec. II-A); the definition used here is the generic index-pair
contraction of a binary tensor contraction (Sec. II-B: each non-leaf node is
a binary contraction producing an output tensor).
"""
from __future__ import annotations

from typing import Callable, Dict, Iterable, List, Optional

import numpy as np

from .dag import Dag


def contract_pair(A: np.ndarray, B: np.ndarray, la, ra) -> np.ndarray:
    """out[t, free(A)..., free(B)...] = sum over pairs of A[t,..] * B[t,..].

    ``A``/``B`` carry the batch axis first; ``la``/``ra`` index the per-slice
    axes (batch excluded)."""
    lt = A.shape[0]
    out = None
    for t in range(lt):
        r = np.tensordot(A[t], B[t], axes=(list(la), list(ra)))
        if out is None:
            out = np.empty((lt,) + np.shape(r), dtype=np.complex128)
        out[t] = r
    return out


def closure(dag: Dag, roots: Iterable[int]) -> List[int]:
    seen = set()
    for r in roots:
        seen.update(dag.tree(r))
    return sorted(seen)


def evaluate(dag: Dag, leaf_fn: Callable[[int], np.ndarray],
             roots: Optional[Iterable[int]] = None) -> Dict[int, np.ndarray]:
    """Correlator C_r(t) of each requested root (default: all roots).

    ``leaf_fn(node_id)`` returns the leaf's complex128 data ``[Lt][...]``.
    Intermediates are dropped after their last consumer in id order."""
    roots = dag.roots() if roots is None else list(roots)
    nodes = closure(dag, roots)
    inset = set(nodes)
    users = {u: sum(1 for p in dag.nodes[u].parents if p in inset) for u in nodes}
    vals: Dict[int, np.ndarray] = {}
    out: Dict[int, np.ndarray] = {}
    want = set(roots)
    for u in nodes:
        nd = dag.nodes[u]
        if nd.is_leaf:
            vals[u] = np.asarray(leaf_fn(u), dtype=np.complex128)
            continue
        r = contract_pair(vals[nd.left], vals[nd.right], nd.la, nd.ra)
        for c in nd.children:
            users[c] -= 1
            if users[c] == 0:
                del vals[c]
        if u in want:
            out[u] = r
        if users[u] > 0:
            vals[u] = r
    return out


def expand_tree(dag: Dag, root: int):
    """Expand the tree of ``root`` into (operands, output labels).

    operands: list of (leaf node id, label list) -- one entry per *occurrence*
    of a leaf in the fully expanded expression.  Contracted axis pairs share a
    label.  Labels are small integers."""
    counter = [0]

    def fresh(k):
        out = list(range(counter[0], counter[0] + k))
        counter[0] += k
        return out

    def rec(u):
        nd = dag.nodes[u]
        if nd.is_leaf:
            lab = fresh(len(nd.extents))
            return [(u, lab)], lab
        opsL, labL = rec(nd.left)
        opsR, labR = rec(nd.right)
        ren = {labR[b]: labL[a] for a, b in zip(nd.la, nd.ra)}
        opsR = [(leaf, [ren.get(x, x) for x in lab]) for leaf, lab in opsR]
        labR = [ren.get(x, x) for x in labR]
        free = [x for i, x in enumerate(labL) if i not in nd.la] + \
            [x for j, x in enumerate(labR) if j not in nd.ra]
        return opsL + opsR, free

    return rec(root)


def brute_force(dag: Dag, root: int, leaf_fn: Callable[[int], np.ndarray]) -> np.ndarray:
    """C_root(t) as a single direct summation over all index labels."""
    ops, out_labels = expand_tree(dag, root)
    tlab = 1 + max(max(lab) for _, lab in ops if lab) if any(lab for _, lab in ops) else 0
    args = []
    for leaf, lab in ops:
        args.append(np.asarray(leaf_fn(leaf), dtype=np.complex128))
        args.append([tlab] + list(lab))
    args.append([tlab] + list(out_labels))
    return np.einsum(*args, optimize=False)
