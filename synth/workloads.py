"""Seeded synthetic stand-ins for the paper's correlation-function workloads.

The paper evaluates six Redstar correlation functions (Table 2) that are not
available here.  These generators produce contraction DAG inputs with the
same structure: many small binary contraction trees (a few to ~10 nodes
each), leaves shared between trees, identical sub-contractions recurring
across trees (so a DAG builder that merges identical requests sees reuse),
and tensor shapes taken from the workload table of this project:

* ``M`` meson elemental, per time slice ``[N][N]`` (distillation in, out)
* ``P`` spin-diluted propagator, per slice ``[4][4][N][N]`` (spin in, spin
  out, distillation in, distillation out)
* ``B`` baryon elemental, per slice ``[N][N][N]`` (three distillation legs)

Every tensor carries a leading batch axis ``Lt`` (time slice) that is never
contracted.  Entries are i.i.d. complex normal with E|z|^2 = 1/N (real and
imaginary parts each of variance 1/(2N)), so chained products stay O(1).

A workload is a *request stream*: stream indices ``0..L-1`` are the leaves,
``L..`` are binary contraction requests in emission order, each naming its
operands by earlier stream index.  Identical sub-trees are emitted again
every time they occur; merging them is the DAG builder's job, not this
module's.  Contraction semantics (shared by both consumers, stated here only
as the input convention): a request contracts left axis ``la[i]`` with right
axis ``ra[i]`` (equal extents) and its output axes are the left operand's
free axes in order followed by the right operand's free axes in order; an
output of rank 0 is a correlator (one complex number per time slice).
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import Dict, List, Sequence, Tuple

import numpy as np

SPIN = 4


@dataclasses.dataclass(frozen=True)
class Leaf:
    kind: str                 # 'M', 'P' or 'B'
    extents: Tuple[int, ...]  # per-time-slice extents (Lt excluded)
    seed: int                 # data seed (see leaf_data)
    lt: int = 0               # batch extent; 0 = the workload's Lt
    nvec: int = 0             # distillation size; 0 = the workload's N


@dataclasses.dataclass(frozen=True)
class Request:
    left: int                 # stream index of the left operand
    right: int                # stream index of the right operand
    la: Tuple[int, ...]       # contracted axes of the left operand
    ra: Tuple[int, ...]       # paired contracted axes of the right operand


@dataclasses.dataclass
class Workload:
    name: str
    lt: int
    nvec: int
    leaves: List[Leaf]
    requests: List[Request]
    # one entry per correlation function: stream indices of its term roots
    functions: List[List[int]]
    budget_bytes: int = 0     # 0 = unlimited device budget
    seed: int = 0
    # every term as a graph before any bracketing: (leaf indices of its
    # items, edges (item a, axis of a, item b, axis of b), one per index
    # pair), in the order of the diagrams; graph_functions[f] lists the
    # graphs of function f (a batched workload concatenates its parts')
    graphs: List[Tuple[List[int], List[Tuple[int, int, int, int]]]] = \
        dataclasses.field(default_factory=list)
    graph_functions: List[List[int]] = dataclasses.field(default_factory=list)

    @property
    def n_leaves(self) -> int:
        return len(self.leaves)

    def stream_extents(self) -> List[Tuple[int, ...]]:
        """Per-slice extents of every stream entry (leaves, then requests)."""
        ext: List[Tuple[int, ...]] = [lf.extents for lf in self.leaves]
        for rq in self.requests:
            le, re_ = ext[rq.left], ext[rq.right]
            lf = tuple(e for i, e in enumerate(le) if i not in rq.la)
            rf = tuple(e for i, e in enumerate(re_) if i not in rq.ra)
            ext.append(lf + rf)
        return ext

    def roots(self) -> List[int]:
        return [r for f in self.functions for r in f]

    def leaf_lt(self, li: int) -> int:
        """Batch extent of leaf ``li`` (independent problems of a batched
        workload have their own)."""
        return self.leaves[li].lt or self.lt

    def leaf_nvec(self, li: int) -> int:
        return self.leaves[li].nvec or self.nvec


def leaf_data(wl: Workload, leaf_index: int, dtype=np.complex128) -> np.ndarray:
    """Dense leaf tensor ``[Lt][extents...]`` drawn from its own PCG64 stream."""
    lf = wl.leaves[leaf_index]
    rng = np.random.Generator(np.random.PCG64([wl.seed, 7919, lf.seed]))
    shape = (wl.leaf_lt(leaf_index),) + tuple(lf.extents)
    sd = np.sqrt(1.0 / (2.0 * wl.leaf_nvec(leaf_index)))
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    out = np.empty(shape, dtype=np.complex128)
    out.real = re * sd
    out.imag = im * sd
    return out.astype(dtype, copy=False)


# --------------------------------------------------------------------------
# axis-label bookkeeping for ring / baryon diagrams
# --------------------------------------------------------------------------
# An axis label is (item_position, role).  Roles: 'din','dout' (distillation
# in/out), 'sin','sout' (spin in/out), 'l0','l1','l2' (baryon legs).
Label = Tuple[int, str]


def _leaf_axes(kind: str, pos: int) -> List[Label]:
    if kind == "M":
        return [(pos, "din"), (pos, "dout")]
    if kind == "P":
        return [(pos, "sin"), (pos, "sout"), (pos, "din"), (pos, "dout")]
    if kind == "B":
        return [(pos, "l0"), (pos, "l1"), (pos, "l2")]
    raise ValueError(kind)


def _ring_links(kinds: Sequence[str]) -> Dict[Label, Label]:
    """Links of a closed quark ring: distillation chain over all items,
    spin chain over the propagators (a ring with exactly one propagator has
    no binary spin closure and is not allowed)."""
    h = len(kinds)
    link: Dict[Label, Label] = {}

    def tie(a: Label, b: Label):
        link[a] = b
        link[b] = a

    for j in range(h):
        tie((j, "dout"), ((j + 1) % h, "din"))
    ps = [j for j, k in enumerate(kinds) if k == "P"]
    if len(ps) == 1:
        raise ValueError("a ring needs zero or at least two propagators")
    for i, j in enumerate(ps):
        tie((j, "sout"), (ps[(i + 1) % len(ps)], "sin"))
    return link


def ring_edges(kinds: Sequence[str], link: Dict[Label, Label]) -> List[Tuple[int, int, int, int]]:
    """The index pairs of a diagram as edges (item a, axis a, item b, axis b),
    a < b by (item, axis), sorted."""
    out = set()
    for la, lb in link.items():
        a = (la[0], _leaf_axes(kinds[la[0]], la[0]).index(la))
        b = (lb[0], _leaf_axes(kinds[lb[0]], lb[0]).index(lb))
        if a > b:
            a, b = b, a
        out.add((a[0], a[1], b[0], b[1]))
    return sorted(out)


def _all_brackets(lo: int, hi: int):
    if lo == hi:
        yield lo
        return
    for k in range(lo, hi):
        for a in _all_brackets(lo, k):
            for b in _all_brackets(k + 1, hi):
                yield (a, b)


def _bracket(rng: np.random.Generator, lo: int, hi: int, style: str):
    if lo == hi:
        return lo
    if style == "left":
        k = hi - 1
    elif style == "balanced":
        k = (lo + hi - 1) // 2
    else:
        k = int(rng.integers(lo, hi))
    return (_bracket(rng, lo, k, style), _bracket(rng, k + 1, hi, style))


def ring_requests(kinds: Sequence[str], link: Dict[Label, Label], bracket,
                  extents: Sequence[Tuple[int, ...]], max_elems: int):
    """Requests of one diagram for a given bracketing of its item positions.

    Returns a list of ``(lref, rref, la, ra)`` where a ref is ``("leaf", pos)``
    (item position) or ``("req", k)`` (k-th request of this list); the last
    request is the diagram's root.  Returns None if the bracketing contains an
    outer product (no contracted pair), an output larger than ``max_elems``
    or leaves an index open at the root.
    """
    pending: List[tuple] = []

    def rec(node):
        if isinstance(node, int):
            return ("leaf", node), _leaf_axes(kinds[node], node), list(extents[node])
        (lref, lax, lext), (rref, rax, rext) = rec(node[0]), rec(node[1])
        if lref is None or rref is None:
            return None, None, None
        rpos = {lab: j for j, lab in enumerate(rax)}
        pairs = []
        for i, lab in enumerate(lax):
            other = link.get(lab)
            if other is not None and other in rpos:
                pairs.append((i, rpos[other]))
        if not pairs:
            return None, None, None
        la = tuple(p[0] for p in pairs)
        ra = tuple(p[1] for p in pairs)
        oax = [lab for i, lab in enumerate(lax) if i not in la] + \
              [lab for j, lab in enumerate(rax) if j not in ra]
        oext = [e for i, e in enumerate(lext) if i not in la] + \
               [e for j, e in enumerate(rext) if j not in ra]
        if int(np.prod(oext, dtype=np.int64)) > max_elems:
            return None, None, None
        pending.append((lref, rref, la, ra))
        return ("req", len(pending) - 1), oax, oext

    ref, ax, _ = rec(bracket)
    if ref is None or ax:
        return None
    return pending


# --------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------
@dataclasses.dataclass(frozen=True)
class Recipe:
    name: str
    lt: int
    nvec: int
    n_functions: int
    hadrons: Tuple[int, int]          # min/max hadrons per meson function
    terms: Tuple[int, int]            # min/max terms (trees) per function
    pool_m: int
    pool_p: int
    pool_b: int = 0
    p_spin: float = 0.0               # probability a meson hadron is a propagator
    p_baryon_fn: float = 0.0          # probability a function is a two-baryon one
    bracket: str = "mixed"            # 'balanced' | 'left' | 'random' | 'mixed'
    p_canonical: float = 0.5          # for 'mixed': probability of left-deep
    prefix_pool: int = 0              # >0: functions start from a shared prefix
    budget_bytes: int = 0
    # 'tree': each diagram's requests together; 'level': all diagrams'
    # first-level contractions, then second-level, ... (stage-by-stage
    # construction, one eliminated edge at a time across all graphs)
    emission: str = "tree"


GIB = 1 << 30

CONFIGS: Dict[str, Recipe] = {
    # 3 functions, 3-4 hadrons, Lt=8, N=16, balanced trees, ~20 nodes
    "tiny": Recipe("tiny", lt=8, nvec=16, n_functions=3, hadrons=(3, 4), terms=(2, 3),
                   pool_m=4, pool_p=3, p_spin=0.45, bracket="balanced"),
    # 200 meson functions, 2-6 hadrons, Lt=64, N=64, ~2,100 contractions, ~28% shared
    "multi_meson": Recipe("multi_meson", lt=64, nvec=64, n_functions=200, hadrons=(2, 6),
                          terms=(3, 7), pool_m=32, pool_p=10, p_spin=0.25,
                          bracket="mixed", p_canonical=0.7, prefix_pool=60,
                          emission="level"),
    # Lt=128, N=128, ~4,800 contractions, ~38% shared, 24 GiB device budget
    "memory_pressure": Recipe("memory_pressure", lt=128, nvec=128, n_functions=440,
                              hadrons=(2, 6), terms=(3, 9), pool_m=32, pool_p=20,
                              p_spin=0.3, bracket="mixed", p_canonical=0.85,
                              prefix_pool=40, budget_bytes=24 * GIB,
                              emission="level"),
    # baryon-like: B_64 + P_64 leaves, 1-2 index contractions, ~3,000 nodes
    "baryon": Recipe("baryon", lt=64, nvec=64, n_functions=530, hadrons=(2, 4),
                     terms=(2, 6), pool_m=24, pool_p=8, pool_b=12, p_spin=0.35,
                     p_baryon_fn=0.7, bracket="random", prefix_pool=0,
                     emission="level"),
}


def _meson_function(rng, rc: Recipe, pools, prefixes):
    """Hadron kinds and leaf choices of one meson function; with a prefix pool,
    most functions start from a shared all-meson prefix (shared sub-trees)."""
    h = int(rng.integers(rc.hadrons[0], rc.hadrons[1] + 1))
    kinds = ["P" if rng.random() < rc.p_spin else "M" for _ in range(h)]
    seq = [int(pools[k][rng.integers(len(pools[k]))]) for k in kinds]
    if prefixes and h >= 3 and rng.random() < 0.7:
        pseq = prefixes[int(rng.integers(len(prefixes)))]
        pl = min(len(pseq), h - 1)
        kinds[:pl] = ["M"] * pl
        seq[:pl] = list(pseq[:pl])
    if kinds.count("P") == 1:
        j = kinds.index("P")
        kinds[j] = "M"
        seq[j] = int(pools["M"][rng.integers(len(pools["M"]))])
    return kinds, seq


@dataclasses.dataclass(frozen=True)
class BatchedRecipe:
    """Many independent correlation-function DAGs of uneven shape in one
    request stream: each part draws its distillation size N and its batch
    extent Lt, then follows the multi-meson recipe at that size (propagator
    leaves only where N <= max_n_spin, which keeps the largest products
    P x P at N = 64 instead of 4N = 1024 rows per slice)."""
    name: str = "batched"
    n_dags: int = 50
    nvecs: Tuple[int, ...] = (32, 48, 64, 96, 128, 192, 256)
    lts: Tuple[int, ...] = (16, 32, 64, 128)
    n_functions: int = 40          # per part: ~400 contractions
    pool_m: int = 8
    pool_p: int = 3
    p_spin: float = 0.25
    max_n_spin: int = 64
    budget_bytes: int = 48 * GIB


BATCHED = {"batched": BatchedRecipe()}


def _make_batched(rc: BatchedRecipe, seed: int) -> Workload:
    rng = np.random.Generator(np.random.PCG64([seed, 130363]))
    leaves: List[Leaf] = []
    parts = []
    for d in range(rc.n_dags):
        n = int(rc.nvecs[int(rng.integers(len(rc.nvecs)))])
        lt = int(rc.lts[int(rng.integers(len(rc.lts)))])
        spin = n <= rc.max_n_spin
        sub = make_workload("multi_meson", seed=int(rng.integers(1 << 31)), lt=lt, nvec=n,
                            n_functions=rc.n_functions, pool_m=rc.pool_m,
                            pool_p=rc.pool_p if spin else 0, p_spin=rc.p_spin if spin else 0.0,
                            prefix_pool=rc.n_functions // 3)
        parts.append((len(leaves), sub))
        for lf in sub.leaves:
            leaves.append(Leaf(lf.kind, lf.extents, len(leaves), lt, n))
    requests: List[Request] = []
    functions: List[List[int]] = []
    graphs: List[Tuple[List[int], List[Tuple[int, int, int, int]]]] = []
    graph_functions: List[List[int]] = []
    n_leaves = len(leaves)
    for loff, sub in parts:
        roff = n_leaves + len(requests)

        def remap(i, loff=loff, roff=roff, sl=sub.n_leaves):
            return loff + i if i < sl else roff + (i - sl)
        for rq in sub.requests:
            requests.append(Request(remap(rq.left), remap(rq.right), rq.la, rq.ra))
        functions.extend([[remap(r) for r in f] for f in sub.functions])
        goff = len(graphs)
        graphs.extend([([loff + i for i in items], list(edges)) for items, edges in sub.graphs])
        graph_functions.extend([[goff + g for g in fn] for fn in sub.graph_functions])
    return Workload(name=rc.name, lt=leaves[0].lt, nvec=max(lf.nvec for lf in leaves),
                    leaves=leaves, requests=requests, functions=functions,
                    budget_bytes=rc.budget_bytes, seed=seed, graphs=graphs,
                    graph_functions=graph_functions)


def make_workload(name: str, seed: int = 0, **overrides) -> Workload:
    """Build the request stream of a named workload (see CONFIGS, BATCHED)."""
    if name in BATCHED:
        brc = dataclasses.replace(BATCHED[name], **overrides) if overrides else BATCHED[name]
        return _make_batched(brc, seed)
    rc = dataclasses.replace(CONFIGS[name], **overrides) if overrides else CONFIGS[name]
    rng = np.random.Generator(np.random.PCG64([seed, 104729]))
    n = rc.nvec
    leaves: List[Leaf] = []
    pools: Dict[str, List[int]] = {"M": [], "P": [], "B": []}
    shapes = {"M": (n, n), "P": (SPIN, SPIN, n, n), "B": (n, n, n)}
    for kind, cnt in (("M", rc.pool_m), ("P", rc.pool_p), ("B", rc.pool_b)):
        for _ in range(cnt):
            pools[kind].append(len(leaves))
            leaves.append(Leaf(kind, shapes[kind], len(leaves)))
    max_elems = max(int(np.prod(lf.extents)) for lf in leaves)

    diagrams: List[Tuple[List[int], list]] = []   # (item leaf indices, pending requests)
    graphs: List[Tuple[List[int], List[Tuple[int, int, int, int]]]] = []

    prefixes = []
    for _ in range(rc.prefix_pool):
        pl = int(rng.integers(2, 4))
        prefixes.append(tuple(int(pools["M"][rng.integers(len(pools["M"]))])
                              for _ in range(pl)))

    fn_diagrams: List[List[int]] = []
    for _f in range(rc.n_functions):
        roots: List[int] = []          # diagram indices of this function's terms
        nterms = int(rng.integers(rc.terms[0], rc.terms[1] + 1))
        if rc.pool_b and rng.random() < rc.p_baryon_fn:
            b1 = int(pools["B"][rng.integers(len(pools["B"]))])
            b2 = int(pools["B"][rng.integers(len(pools["B"]))])
            n_ins = int(rng.integers(0, 3))
            lines = sorted(rng.choice(3, size=n_ins, replace=False).tolist())
            ms = [int(pools["M"][rng.integers(len(pools["M"]))]) for _ in lines]
            perms = list(itertools.permutations(range(3)))
            order = rng.permutation(len(perms))[:nterms]
            for pi in order:
                perm = perms[int(pi)]
                # items: B1, inserted M's (one per chosen line), B2
                kinds = ["B"] + ["M"] * len(lines) + ["B"]
                items = [b1] + ms + [b2]
                link: Dict[Label, Label] = {}

                def tie(a, b):
                    link[a] = b
                    link[b] = a
                last = len(items) - 1
                for leg in range(3):
                    tgt = (last, "l%d" % perm[leg])
                    if leg in lines:
                        mpos = 1 + lines.index(leg)
                        tie((0, "l%d" % leg), (mpos, "din"))
                        tie((mpos, "dout"), tgt)
                    else:
                        tie((0, "l%d" % leg), tgt)
                cands = list(_all_brackets(0, len(items) - 1))
                rng.shuffle(cands)
                for br in cands:
                    pend = ring_requests(kinds, link, br, [leaves[i].extents for i in items],
                                         max_elems)
                    if pend is not None:
                        roots.append(len(diagrams))
                        diagrams.append((items, pend))
                        graphs.append((list(items), ring_edges(kinds, link)))
                        break
        else:
            kinds, seq = _meson_function(rng, rc, pools, prefixes)
            h = len(seq)
            for term in range(nterms):
                if term == 0:
                    perm = list(range(h))
                else:
                    perm = [0] + (1 + rng.permutation(h - 1)).tolist() if h > 2 else [1, 0]
                tk = [kinds[p] for p in perm]
                ti = [seq[p] for p in perm]
                link = _ring_links(tk)
                style = rc.bracket
                if style == "mixed":
                    style = "left" if rng.random() < rc.p_canonical else "random"
                br = _bracket(rng, 0, h - 1, style)
                exts = [leaves[i].extents for i in ti]
                pend = ring_requests(tk, link, br, exts, max_elems)
                if pend is None:
                    for br2 in _all_brackets(0, h - 1):
                        pend = ring_requests(tk, link, br2, exts, max_elems)
                        if pend is not None:
                            break
                if pend is not None:
                    roots.append(len(diagrams))
                    diagrams.append((ti, pend))
                    graphs.append((list(ti), ring_edges(tk, link)))
        if roots:
            fn_diagrams.append(roots)
    requests, root_of = _emit(diagrams, len(leaves), rc.emission)
    functions = [[root_of[d] for d in fn] for fn in fn_diagrams]
    return Workload(name=rc.name, lt=rc.lt, nvec=n, leaves=leaves, requests=requests,
                    functions=functions, budget_bytes=rc.budget_bytes, seed=seed,
                    graphs=graphs, graph_functions=[list(fn) for fn in fn_diagrams])


def _emit(diagrams, n_leaves: int, emission: str):
    """Flatten the diagrams' requests into one stream (operands first)."""
    keyed = []
    for d, (items, pend) in enumerate(diagrams):
        depth: List[int] = []
        for k, (lref, rref, _la, _ra) in enumerate(pend):
            dl = depth[lref[1]] if lref[0] == "req" else 0
            dr = depth[rref[1]] if rref[0] == "req" else 0
            depth.append(1 + max(dl, dr))
            keyed.append(((depth[-1] if emission == "level" else 0), d, k))
    keyed.sort()
    where: Dict[Tuple[int, int], int] = {}
    requests: List[Request] = []
    for (_dep, d, k) in keyed:
        items, pend = diagrams[d]
        lref, rref, la, ra = pend[k]

        def res(r):
            return items[r[1]] if r[0] == "leaf" else where[(d, r[1])]
        requests.append(Request(res(lref), res(rref), la, ra))
        where[(d, k)] = n_leaves + len(requests) - 1
    root_of = {d: where[(d, len(pend) - 1)] for d, (_i, pend) in enumerate(diagrams)}
    return requests, root_of
