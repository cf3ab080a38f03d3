"""Memory model of Sec. II-C ("Problem definition", Table 1) and a budgeted
replay with eviction to host memory.

Memory model (Sec. II-C): contractions c_1..c_n run in order, M_0 = 0.  Step
i (1) brings in any leaf tensor c_i needs that is not in device memory --
leaves start on the host and count only from their first use, (2) performs
c_i, producing its output, (3) releases every tensor no remaining contraction
depends on, the output included (a root's output is released at once).
M_i is the memory in use after step i; the peak is max_i M_i and M_n = 0.
Temporary memory of a contraction is not counted.

Budgeted replay (the paper relies on MemHC, Sec. II-A: when a contraction
does not fit, blocks are evicted to the host under a "pre-protected LRU"
policy; this is the stand-in whose rules are fixed here):
  * before c_i: need = bytes of inputs not on the device + bytes of the output.
    If inputs + output alone exceed the budget B -> BudgetError.
  * while resident + need > B: evict one resident tensor that is not an input
    of c_i (the operands are protected).  LRU: least recent touch (load,
    production or use as input), ties to the smaller id.  NEXT_USE: the
    farthest next use in the order, ties to the larger size, then the
    smaller id.  A tensor whose only copy is on the device (an intermediate
    never written out) is copied to the host (one D2H); leaves and tensors
    reloaded from a host copy are dropped without a copy.
  * missing inputs are loaded (one H2D each: a leaf from the host store or an
    evicted intermediate from its host copy), left operand first.
  * c_i runs; the device then holds resident + output bytes (peak_exec is
    the maximum of this), then step (3) releases as in the model.

All figures are Python ints (exact).  An eviction is one tensor dropped
from the device to make room.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence, Tuple

from .dag import Dag

LRU, NEXT_USE = "lru", "next_use"
LOAD, EVICT, CONTRACT, FREE = "LOAD", "EVICT", "CONTRACT", "FREE"


class BudgetError(Exception):
    pass


@dataclasses.dataclass
class Stats:
    peak_paper: int = 0
    peak_exec: int = 0
    n_evict: int = 0
    n_h2d: int = 0
    n_d2h: int = 0
    h2d_bytes: int = 0
    d2h_bytes: int = 0

    def as_tuple(self) -> Tuple[int, ...]:
        return (self.peak_paper, self.peak_exec, self.n_evict, self.n_h2d,
                self.n_d2h, self.h2d_bytes, self.d2h_bytes)


def model_trace(dag: Dag, order: Sequence[int]) -> Tuple[List[int], List[frozenset]]:
    """M_1..M_n and the resident sets after each step (Sec. II-C, Table 1)."""
    remaining = {u: len(dag.nodes[u].parents) for u in range(len(dag.nodes))}
    mem: set = set()
    sizes, sets = [], []
    for c in order:
        nd = dag.nodes[c]
        for x in nd.children:                      # (i) bring leaves in
            if dag.nodes[x].is_leaf:
                mem.add(x)
        mem.add(c)                                 # (ii) contract
        for x in nd.children:                      # (iii) release
            remaining[x] -= 1
            if remaining[x] == 0:
                mem.discard(x)
        if not nd.parents:
            mem.discard(c)
        sizes.append(sum(dag.size(u) for u in mem))
        sets.append(frozenset(mem))
    return sizes, sets


def peak_paper(dag: Dag, order: Sequence[int]) -> int:
    sizes, _ = model_trace(dag, order)
    return max(sizes) if sizes else 0


@dataclasses.dataclass
class Plan:
    ops: List[Tuple[str, int, int]]   # (kind, node, flag); flag = 1 for a D2H write-back
    stats: Stats
    trace: List[int]                  # device bytes after each step's releases


def replay(dag: Dag, order: Sequence[int], budget: Optional[int] = None,
           policy: str = LRU) -> Plan:
    """Budgeted replay of ``order`` (budget None = unlimited)."""
    pos = {c: i for i, c in enumerate(order)}
    remaining = {u: len(dag.nodes[u].parents) for u in range(len(dag.nodes))}
    # future uses of every tensor: positions of its consumers in the order
    uses: Dict[int, List[int]] = {}
    for c in order:
        for x in dag.nodes[c].children:
            uses.setdefault(x, []).append(pos[c])
    for x in uses:
        uses[x].sort()
    resident: Dict[int, int] = {}     # node -> last touch (step index)
    host_copy = set(u for u in range(len(dag.nodes)) if dag.nodes[u].is_leaf)
    st = Stats()
    ops: List[Tuple[str, int, int]] = []
    trace: List[int] = []
    res_bytes = 0

    def next_use(x: int, i: int) -> int:
        for p in uses.get(x, []):
            if p > i:
                return p
        return len(order)  # unreachable for resident tensors

    for i, c in enumerate(order):
        nd = dag.nodes[c]
        inputs = nd.children
        out_b = dag.size(c)
        if budget is not None and sum(dag.size(x) for x in inputs) + out_b > budget:
            raise BudgetError("contraction %d needs more than the budget" % c)
        missing = [x for x in inputs if x not in resident]
        need = sum(dag.size(x) for x in missing) + out_b
        if budget is not None:
            while res_bytes + need > budget:
                cands = [x for x in resident if x not in inputs]
                if policy == LRU:
                    victim = min(cands, key=lambda x: (resident[x], x))
                elif policy == NEXT_USE:
                    victim = min(cands, key=lambda x: (-next_use(x, i), -dag.size(x), x))
                else:
                    raise ValueError(policy)
                wb = 0
                if victim not in host_copy:
                    wb = 1
                    host_copy.add(victim)
                    st.n_d2h += 1
                    st.d2h_bytes += dag.size(victim)
                ops.append((EVICT, victim, wb))
                st.n_evict += 1
                del resident[victim]
                res_bytes -= dag.size(victim)
        for x in missing:
            ops.append((LOAD, x, 0))
            st.n_h2d += 1
            st.h2d_bytes += dag.size(x)
            resident[x] = i
            res_bytes += dag.size(x)
        ops.append((CONTRACT, c, 0))
        st.peak_exec = max(st.peak_exec, res_bytes + out_b)
        for x in inputs:
            resident[x] = i
        resident[c] = i
        res_bytes += out_b
        for x in inputs:
            remaining[x] -= 1
            if remaining[x] == 0:
                ops.append((FREE, x, 0))
                del resident[x]
                res_bytes -= dag.size(x)
        if not nd.parents:
            ops.append((FREE, c, 0))
            del resident[c]
            res_bytes -= out_b
        trace.append(res_bytes)
    st.peak_paper = peak_paper(dag, order)
    return Plan(ops, st, trace)


def interval_profile(dag: Dag, order: Sequence[int]) -> Tuple[List[int], List[int]]:
    """Closed form of the unbudgeted model, independent of ``replay``.

    Every tensor x lives on [start, end]: start = its own step (non-leaf) or
    its first consumer's step (leaf); end = its last consumer's step (a root
    ends where it starts).  After step i it is held iff start <= i < end;
    during step i it is held iff start <= i <= end.  Returns (M_i, exec_i)."""
    pos = {c: i for i, c in enumerate(order)}
    n = len(order)
    after = [0] * n
    during = [0] * n
    for u, nd in enumerate(dag.nodes):
        cons = [pos[p] for p in nd.parents]
        if nd.is_leaf:
            if not cons:
                continue
            s, e = min(cons), max(cons)
        else:
            s = pos[u]
            e = max(cons) if cons else s
        for i in range(s, e + 1):
            during[i] += dag.size(u)
            if i < e:
                after[i] += dag.size(u)
    return after, during


def check_plan(dag: Dag, order: Sequence[int], plan: Plan, budget: Optional[int]) -> None:
    """Independent validity check of an op list: every operand is on the
    device when used, the budget is never exceeded, every figure of the
    stats is recounted from the ops.  Raises AssertionError."""
    res: Dict[int, bool] = {}
    on_host = set(u for u in range(len(dag.nodes)) if dag.nodes[u].is_leaf)
    cnt = Stats()
    k = 0
    bytes_now = 0
    for (kind, u, flag) in plan.ops:
        sz = dag.size(u)
        if kind == LOAD:
            assert u not in res and u in on_host
            res[u] = True
            bytes_now += sz
            cnt.n_h2d += 1
            cnt.h2d_bytes += sz
        elif kind == EVICT:
            assert u in res
            if flag:
                assert u not in on_host
                on_host.add(u)
                cnt.n_d2h += 1
                cnt.d2h_bytes += sz
            else:
                assert u in on_host
            del res[u]
            bytes_now -= sz
            cnt.n_evict += 1
        elif kind == CONTRACT:
            assert order[k] == u
            k += 1
            for x in dag.nodes[u].children:
                assert x in res, "operand %d not on device for %d" % (x, u)
            res[u] = True
            bytes_now += sz
            cnt.peak_exec = max(cnt.peak_exec, bytes_now)
        elif kind == FREE:
            assert u in res
            del res[u]
            bytes_now -= sz
        if budget is not None:
            assert bytes_now <= budget
    assert k == len(order) and not res
    assert (cnt.peak_exec, cnt.n_evict, cnt.n_h2d, cnt.n_d2h, cnt.h2d_bytes, cnt.d2h_bytes) == \
        (plan.stats.peak_exec, plan.stats.n_evict, plan.stats.n_h2d, plan.stats.n_d2h,
         plan.stats.h2d_bytes, plan.stats.d2h_bytes)
