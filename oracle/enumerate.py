"""Exhaustive enumeration of the contraction orders of tiny DAGs.

Every topological order of the non-leaf nodes (every linear extension of the
dependency relation among contractions) is generated.  With at most ~10
contractions this is feasible and gives, for every order, the memory-model
figures of Sec. II-C, hence the optimal peak the schedulers of Sec. III aim
for.
"""
from __future__ import annotations

from typing import Iterator, List

from .dag import Dag


def topological_orders(dag: Dag) -> Iterator[List[int]]:
    nl = dag.non_leaf()
    deps = {u: [c for c in dag.nodes[u].children if not dag.nodes[c].is_leaf] for u in nl}
    placed = set()
    cur: List[int] = []

    def rec():
        if len(cur) == len(nl):
            yield list(cur)
            return
        for u in nl:
            if u not in placed and all(c in placed for c in deps[u]):
                placed.add(u)
                cur.append(u)
                yield from rec()
                cur.pop()
                placed.discard(u)

    yield from rec()
