"""Native contraction-path selection (lqc_dag_add_graphs, Sec. II-A) against
the oracle's (oracle.paths, whose pins are in test_oracle_paths.py).

* Bit-exact: the native call builds the same DAG as the oracle -- every
  node's operands and axis pairs, node ids and each graph's root -- on the
  generator's terms (meson and baryon workloads) and on seeded random tensor
  graphs (ranks 1..3, multi-edges, open axes, recurring sub-graphs).
* A planted mistake in the oracle (key value without the contraction cost)
  changes the DAG, so the comparison sees the cost term.
* Argument errors: bad offsets, vertex, axis, an axis paired twice, unequal
  extents, a disconnected graph, a frozen DAG.
* Flop count of a DAG from its node sizes equals the sum over the
  generator's contraction shapes.
* GPU: the correlators of a path-selected DAG against the oracle evaluation
  of the oracle's path-selected DAG, FP64 (<= 1e-12) and TF32x3 (<= 1e-6).
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D
from oracle import paths as PS

L = pytest.importorskip("paper_2511_02257_b300")


def _structure_native(nd):
    return [nd.node_operands(u) for u in range(nd.num_nodes())]


def _structure_oracle(od):
    return [(-1, -1, (), ()) if n.is_leaf else (n.left, n.right, tuple(n.la), tuple(n.ra))
            for n in od.nodes]


def _random_graphs(seed, n_leaves=7, n_graphs=24, n=3, lt=2):
    """Leaves of rank 1..3 (all extents n) and connected graphs over them:
    a spanning tree of edges between free axes, then extra random edges
    (multi-edges allowed), the rest of the axes left open.  Every other
    graph is followed by a copy of itself (a recurring term); the leaves
    are shared, so sub-graphs recur across different graphs too."""
    rng = np.random.default_rng(seed)
    ranks = [int(r) for r in rng.integers(1, 4, size=n_leaves)]
    graphs = []
    while len(graphs) < n_graphs:
        nv = int(rng.integers(2, 5))
        verts = [int(x) for x in rng.integers(0, n_leaves, size=nv)]
        free = {(v, a) for v in range(nv) for a in range(ranks[verts[v]])}
        edges = []
        ok = True
        for v in range(1, nv):
            mine = sorted(x for x in free if x[0] == v)
            theirs = sorted(x for x in free if x[0] < v)
            if not mine or not theirs:
                ok = False
                break
            a = mine[int(rng.integers(len(mine)))]
            b = theirs[int(rng.integers(len(theirs)))]
            free -= {a, b}
            edges.append((b[0], b[1], a[0], a[1]))
        if not ok:
            continue
        for _ in range(int(rng.integers(0, 3))):
            fl = sorted(free)
            if len(fl) < 2:
                break
            i, j = rng.choice(len(fl), size=2, replace=False)
            a, b = fl[int(i)], fl[int(j)]
            if a[0] == b[0]:
                continue
            free -= {a, b}
            edges.append((a[0], a[1], b[0], b[1]))
        graphs.append((verts, edges))
        if len(graphs) % 2 == 0 and len(graphs) < n_graphs:
            graphs.append((list(verts), list(edges)))           # a recurring term
    return ranks, graphs, n, lt


def _build_both(ranks, graphs, n, lt):
    od = D.Dag(lt)
    nd = L.Dag(lt)
    for i, r in enumerate(ranks):
        od.add_leaf((n,) * r, leaf_index=i)
        nd.add_leaf((n,) * r)
    oroots = PS.select_paths(od, graphs)
    nroots = nd.add_graphs(graphs)
    return od, oroots, nd, nroots


@pytest.mark.parametrize("name,kw", [("tiny", {}),
                                     ("multi_meson", dict(n_functions=12, nvec=6, lt=3)),
                                     ("multi_meson", dict(n_functions=40, seed=3)),
                                     ("baryon", dict(n_functions=10, nvec=5, lt=2)),
                                     ("baryon", dict(n_functions=30, seed=1)),
                                     ("memory_pressure", dict(n_functions=20)),
                                     ("batched", dict(n_dags=6, nvecs=(16, 32), lts=(4, 8),
                                                      n_functions=10))])
def test_paths_bit_exact_workloads(name, kw):
    wl = synth.make_workload(name, **kw)
    od, oroots = PS.build_with_paths(wl)
    nd, ids = L.build_dag(wl, with_data=False, paths=True)
    nl = len(wl.leaves)
    assert ids[nl:] == oroots
    assert nd.num_nodes() == len(od.nodes)
    assert _structure_native(nd) == _structure_oracle(od)
    for u in range(len(od.nodes)):
        assert nd.node_info(u)["size"] == od.size(u)


@pytest.mark.parametrize("seed", range(8))
def test_paths_bit_exact_random_graphs(seed):
    ranks, graphs, n, lt = _random_graphs(seed)
    od, oroots, nd, nroots = _build_both(ranks, graphs, n, lt)
    assert nroots == oroots
    assert _structure_native(nd) == _structure_oracle(od)
    # recurring terms share their root
    for g in range(1, len(graphs)):
        if graphs[g] == graphs[g - 1]:
            assert nroots[g] == nroots[g - 1]


def test_shared_pair_native():
    n, lt = 5, 2
    nd = L.Dag(lt)
    A, B, Cm, Dm = (nd.add_leaf((n, n)) for _ in range(4))
    ring = [(0, 1, 1, 0), (1, 1, 2, 0), (0, 0, 2, 1)]
    roots = nd.add_graphs([([A, B, Cm], ring), ([Dm, B, Cm], ring)])
    assert nd.num_nodes() == 7
    assert nd.node_operands(4) == (B, Cm, (1,), (0,))
    assert all(nd.node_info(r)["rank"] == 0 for r in roots)


def test_planted_mistake_in_oracle_is_seen(monkeypatch):
    """The oracle with the contraction cost dropped from a key's value (a
    plausible mistake: counting edge frequency only) builds another DAG than
    the native call on a workload with shapes of different cost."""
    wl = synth.make_workload("baryon", n_functions=30, seed=1)
    nd, ids = L.build_dag(wl, with_data=False, paths=True)
    good = PS._candidate

    def no_cost(dag, p, q, partner):
        c = good(dag, p, q, partner)
        return None if c is None else (c[0], 1) + tuple(c[2:])
    monkeypatch.setattr(PS, "_candidate", no_cost)
    od, _ = PS.build_with_paths(wl)
    assert _structure_native(nd) != _structure_oracle(od)


def test_add_graphs_argument_errors():
    nd = L.Dag(2)
    a = nd.add_leaf((3, 3))
    b = nd.add_leaf((3, 4))
    c = nd.add_leaf((3,))
    corr = nd.add_contraction(a, a, [0, 1], [1, 0])
    cases = [
        [([a], [(0, 0, 1, 0)])],                      # vertex index out of range
        [([a, b], [(0, 5, 1, 0)])],                   # axis out of range
        [([a, b], [(0, 0, 1, 0), (0, 0, 1, 1)])],     # an axis paired twice
        [([a, b], [(0, 1, 1, 1)])],                   # extents 3 and 4
        [([a, b, c], [(0, 0, 1, 0)])],                # c is not connected
        [([a, 99], [(0, 0, 1, 0)])],                  # not a node
        [([a, a], [(0, 0, 0, 1)])],                   # an edge within one vertex
        [([a, corr], [])],                            # a correlator (rank 0) as a vertex
        [([a, b], [(-1, 0, 1, 0)])],                  # negative vertex index
    ]
    for graphs in cases:
        with pytest.raises(L.LqcError) as ei:
            nd.add_graphs(graphs)
        assert ei.value.code == L.LQC_ERR_ARG, graphs
    # a one-vertex graph is its own root; an empty list adds nothing
    assert nd.add_graphs([([b], [])]) == [b]
    n0 = nd.num_nodes()
    assert nd.add_graphs([]) == [] and nd.num_nodes() == n0
    # a valid call after the errors
    r = nd.add_graphs([([a, a], [(0, 0, 1, 1), (0, 1, 1, 0)])])[0]
    assert nd.node_info(r)["rank"] == 0
    nd.schedule("tree", "lru", 0)
    with pytest.raises(L.LqcError) as ei:
        nd.add_graphs([([a, a], [(0, 0, 1, 0)])])
    assert ei.value.code == L.LQC_ERR_STATE


@pytest.mark.parametrize("name,kw", [("multi_meson", dict(n_functions=12, nvec=6, lt=3)),
                                     ("baryon", dict(n_functions=10, nvec=5, lt=2))])
def test_dag_flops_from_sizes(name, kw):
    from experiments import dag_contraction_flops
    from paper_2511_02257_b300.roofline import contraction_shapes
    wl = synth.make_workload(name, **kw)
    nd, ids = L.build_dag(wl, with_data=False)
    want = sum(8 * lt * m * n * k for (lt, m, n, k, _) in contraction_shapes(wl, ids).values())
    assert dag_contraction_flops(nd) == want


# ---------------------------------------------------------------- GPU
@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("tf32x3", 1e-6)])
@pytest.mark.parametrize("name,kw", [("multi_meson", dict(n_functions=12, nvec=24, lt=8)),
                                     ("baryon", dict(n_functions=10, nvec=12, lt=4))])
def test_path_selected_dag_vs_oracle(precision, tol, name, kw):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload(name, **kw)
    od, oroots = PS.build_with_paths(wl)
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index), sorted(set(oroots)))
    nd, ids = L.build_dag(wl, precision=precision, paths=True,
                          leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    assert ids[len(wl.leaves):] == oroots
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    planned = nd.schedule("tree", "lru", 0)
    nd.execute(torch.cuda.current_stream().cuda_stream)
    assert nd.stats() == planned
    errs = [np.linalg.norm(nd.read_correlator(r) - ref[r]) / np.linalg.norm(ref[r])
            for r in sorted(set(oroots))]
    assert max(errs) < tol, max(errs)


def test_paths_values_beyond_int64():
    """Extents whose contraction costs times their counts exceed 2^63: the
    native selection keeps exact values (128-bit) like the oracle's
    integers, so both pick the same keys."""
    n, lt = 1 << 20, 8
    od, nd = D.Dag(lt), L.Dag(lt)
    for i in range(4):
        od.add_leaf((n, n), leaf_index=i)
        nd.add_leaf((n, n))
    ring = [(0, 1, 1, 0), (1, 1, 2, 0), (0, 0, 2, 1)]
    graphs = [([0, 1, 2], ring), ([3, 1, 2], ring), ([0, 3, 2], ring), ([1, 2, 3], ring)]
    oroots = PS.select_paths(od, graphs)
    assert 2 * lt * n ** 3 > 2 ** 63            # count x cost of the shared pair
    assert nd.add_graphs(graphs) == oroots
    assert _structure_native(nd) == _structure_oracle(od)


def test_orientation_larger_tensor_left_native():
    n, lt = 3, 2
    for m_first in (True, False):
        nd = L.Dag(lt)
        if m_first:
            Mn, Pn = nd.add_leaf((n, n)), nd.add_leaf((4, 4, n, n))
        else:
            Pn, Mn = nd.add_leaf((4, 4, n, n)), nd.add_leaf((n, n))
        r = nd.add_graphs([([Mn, Pn], [(0, 1, 1, 2), (1, 3, 0, 0)])])[0]
        assert nd.node_operands(r) == (Pn, Mn, (2, 3), (1, 0))


def test_failed_call_leaves_the_dag_unchanged():
    """A call that fails after it began adding contractions (here: a chain
    of propagators whose products pass LQC_MAX_RANK = 8 axes) removes them
    again; a disconnected graph is rejected before anything is added.  The
    DAG then builds exactly as a fresh one does."""
    n, lt = 3, 2

    def fresh():
        d = L.Dag(lt)
        ids = [d.add_leaf((4, 4, n, n)) for _ in range(4)] + [d.add_leaf((n, n))]
        return d, ids
    good = [([0, 4], [(0, 2, 1, 1), (0, 3, 1, 0)]), ([1, 4, 2], [(0, 3, 1, 0), (1, 1, 2, 2)])]
    # P0 - P1 - P2 - P3 joined by one spin axis each: the product reaches rank 10
    chain = ([0, 1, 2, 3], [(0, 0, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0)])
    split = ([0, 1, 4], [(0, 2, 1, 2)])          # vertex 2 has no edge
    d, ids = fresh()
    n_before = d.num_nodes()
    for bad in ([good[0], chain], [good[0], split]):
        with pytest.raises(L.LqcError) as ei:
            d.add_graphs(bad)
        assert ei.value.code == L.LQC_ERR_ARG
        assert d.num_nodes() == n_before
        assert all(d.node_info(u)["is_leaf"] for u in range(d.num_nodes()))
    roots = d.add_graphs(good)
    ref, _ = fresh()
    assert roots == ref.add_graphs(good)
    assert _structure_native(d) == _structure_native(ref)
    d.schedule("tree", "lru", 0)
    ref.schedule("tree", "lru", 0)
    assert d.order() == ref.order() and d.plan() == ref.plan()


def _random_graphs_mixed(seed, n_leaves=8, n_graphs=30, lt=2):
    """Like _random_graphs, with axis extents drawn from {2, 3, 4}: edges
    pair only equal extents, so contraction costs differ and decide the
    order, not only the ties."""
    rng = np.random.default_rng(100 + seed)
    shapes = [tuple(int(e) for e in rng.integers(2, 5, size=int(rng.integers(1, 4))))
              for _ in range(n_leaves)]
    graphs = []
    tries = 0
    while len(graphs) < n_graphs and tries < 10000:
        tries += 1
        nv = int(rng.integers(2, 5))
        verts = [int(x) for x in rng.integers(0, n_leaves, size=nv)]
        free = {(v, a) for v in range(nv) for a in range(len(shapes[verts[v]]))}
        ext = lambda va: shapes[verts[va[0]]][va[1]]  # noqa: E731
        edges, ok = [], True
        for v in range(1, nv):
            pairs = [(b, a) for a in sorted(free) if a[0] == v
                     for b in sorted(free) if b[0] < v and ext(a) == ext(b)]
            if not pairs:
                ok = False
                break
            b, a = pairs[int(rng.integers(len(pairs)))]
            free -= {a, b}
            edges.append((b[0], b[1], a[0], a[1]))
        if not ok:
            continue
        graphs.append((verts, edges))
        if rng.random() < 0.4:
            graphs.append((list(verts), list(edges)))
    return shapes, graphs, lt


@pytest.mark.parametrize("seed", range(8))
def test_paths_bit_exact_random_graphs_mixed_extents(seed):
    shapes, graphs, lt = _random_graphs_mixed(seed)
    assert len(graphs) >= 20
    od, nd = D.Dag(lt), L.Dag(lt)
    for i, sh in enumerate(shapes):
        od.add_leaf(sh, leaf_index=i)
        nd.add_leaf(sh)
    oroots = PS.select_paths(od, graphs)
    assert nd.add_graphs(graphs) == oroots
    assert _structure_native(nd) == _structure_oracle(od)


def test_rarer_costlier_pair_native():
    """The hand-derived count x cost example of test_oracle_paths: the
    native selection builds the same six contractions, written out by hand
    there (the once-occurring C.B of cost 64 before the twice-occurring A.B
    of cost 8)."""
    from test_oracle_paths import COSTLY_PAIR_EXPECTED, COSTLY_PAIR_SHAPES, _ring4
    nd = L.Dag(2)
    A, B, Cm, Dm, E, F = (nd.add_leaf(s) for s in COSTLY_PAIR_SHAPES)
    roots = nd.add_graphs([_ring4(A, B, Cm, Dm), _ring4(A, B, E, F)])
    assert roots == [8, 11]
    assert [nd.node_operands(u) for u in range(6, nd.num_nodes())] == COSTLY_PAIR_EXPECTED
