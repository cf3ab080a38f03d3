"""Pins of the oracle's contraction-path selection (oracle.paths, Sec. II-A).

* Hand example: Tr(A B C) and Tr(D B C) share the adjacent pair B.C, so the
  selection contracts it first in both terms and builds 3 contractions
  (B.C and one root each) where left-deep brackets (A.B).C, (D.B).C build 4.
* Any contraction path of a term gives the same correlator: every root of a
  path-selected DAG equals the generator's own bracketing of the same term
  (whose values the brute-force pins cover), on meson and baryon terms.
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D
from oracle import paths as PS


def _ring3(x, y, z):
    # Tr(X Y Z): X.dout-Y.din, Y.dout-Z.din, Z.dout-X.din (axes din=0, dout=1)
    return [x, y, z], [(0, 1, 1, 0), (1, 1, 2, 0), (0, 0, 2, 1)]


def test_shared_pair_selected_first():
    n, lt = 5, 2
    dag = D.Dag(lt)
    A, B, Cm, Dm = (dag.add_leaf((n, n), leaf_index=i) for i in range(4))
    roots = PS.select_paths(dag, [_ring3(A, B, Cm), _ring3(Dm, B, Cm)])
    contr = [u for u in range(len(dag.nodes)) if not dag.nodes[u].is_leaf]
    assert len(contr) == 3
    first = dag.nodes[contr[0]]
    assert (first.left, first.right, first.la, first.ra) == (B, Cm, (1,), (0,))
    assert all(dag.nodes[r].extents == () for r in roots)
    # left-deep brackets of the same two terms share nothing
    ld = D.Dag(lt)
    for i in range(4):
        ld.add_leaf((n, n), leaf_index=i)
    for x in (0, 3):
        xy = ld.add_contraction(x, 1, (1,), (0,))
        ld.add_contraction(xy, 2, (1, 0), (0, 1))
    assert len(ld.non_leaf()) == 4
    # and the values agree with a direct trace
    rng = np.random.default_rng(0)
    data = [rng.standard_normal((lt, n, n)) + 1j * rng.standard_normal((lt, n, n)) for _ in range(4)]
    got = C.evaluate(dag, lambda u: data[u], roots)
    for r, x in zip(roots, (0, 3)):
        want = np.einsum("tij,tjk,tki->t", data[x], data[1], data[2])
        assert np.allclose(got[r], want, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name,kw", [("tiny", {}), ("multi_meson", dict(n_functions=12, nvec=6, lt=3)),
                                     ("baryon", dict(n_functions=10, nvec=5, lt=2)),
                                     ("batched", dict(n_dags=3, nvecs=(4, 6), lts=(2, 3),
                                                      n_functions=5))])
def test_paths_give_the_generators_values(name, kw):
    wl = synth.make_workload(name, **kw)
    od, ids = D.build_from_workload(wl)
    pd, proots = PS.build_with_paths(wl)
    assert len(proots) == len(wl.graphs)

    def lf(u):
        return synth.leaf_data(wl, u)     # leaves are the first nodes on both sides
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
    got = C.evaluate(pd, lf, proots)
    roots_in_order = [r for f in wl.functions for r in f]
    graph_roots = [ids[r] for r in roots_in_order]       # generator roots, diagram order
    assert len(graph_roots) == len(proots)
    for g, (r_ref, r_path) in enumerate(zip(graph_roots, proots)):
        a, b = ref[r_ref], got[r_path]
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a), (name, g)
    # the path-selected DAG merges at least as much as it emits
    assert len(pd.non_leaf()) <= sum(len(e) for _, e in wl.graphs)


def test_orientation_larger_tensor_left():
    """The orientation reading: the tensor with more elements is the left
    operand (M >= N), whatever the vertex order or node ids.  A meson M
    [n][n] traced against the distillation axes of a propagator P
    [4][4][n][n] leaves the spin axes open: the one contraction has P on
    the left, its pairs sorted by P's axes."""
    n, lt = 3, 2
    for m_first in (True, False):
        dag = D.Dag(lt)
        if m_first:
            Mn = dag.add_leaf((n, n), leaf_index=0)
            Pn = dag.add_leaf((4, 4, n, n), leaf_index=1)
        else:
            Pn = dag.add_leaf((4, 4, n, n), leaf_index=0)
            Mn = dag.add_leaf((n, n), leaf_index=1)
        # vertices [M, P]: M.dout - P.din, P.dout - M.din
        roots = PS.select_paths(dag, [([Mn, Pn], [(0, 1, 1, 2), (1, 3, 0, 0)])])
        node = dag.nodes[roots[0]]
        assert (node.left, node.right, node.la, node.ra) == (Pn, Mn, (2, 3), (1, 0))
        assert node.extents == (4, 4)
        rng = np.random.default_rng(1)
        mv = rng.standard_normal((lt, n, n)) + 1j * rng.standard_normal((lt, n, n))
        pv = rng.standard_normal((lt, 4, 4, n, n)) + 1j * rng.standard_normal((lt, 4, 4, n, n))
        got = C.evaluate(dag, lambda u: mv if u == Mn else pv, roots)[roots[0]]
        want = np.einsum("tab,tsuba->tsu", mv, pv)
        assert np.allclose(got, want, rtol=1e-12, atol=0)


def _ring4(w, x, y, z):
    # Tr(W X Y Z) of matrices: W.1-X.0, X.1-Y.0, Y.1-Z.0, Z.1-W.0
    return [w, x, y, z], [(0, 1, 1, 0), (1, 1, 2, 0), (2, 1, 3, 0), (3, 1, 0, 0)]


# The contractions path selection must build for Tr(A B C D) and Tr(A B E F)
# with extents a = b = c = e = 2 and d = 16 (A: a x b, B: b x c, C: c x d,
# D: d x a, E: c x e, F: e x a), derived by hand (per slice, cost = M N K):
#  1. candidates: A.B in both terms, cost 8, value 2 x 8 = 16; in the first
#     term B.C, C.D, D.A cost 64 each (value 64); in the second every pair
#     costs 8.  The largest value is 64; of the tied keys (left = the larger
#     tensor, equal sizes -> smaller id) (C,B,(0,),(1,)) < (C,D,(1,),(0,)) <
#     (D,A,(1,),(0,)), so C.B -> node 6 [d x b].  A selection by frequency
#     alone would take A.B here.
#  2. first term [A, 6, D]: 6.A, D.6, D.A all cost 64; smallest key
#     (D,A,(1,),(0,)) -> node 7 [d x b].
#  3. first term [7, 6]: both axes pair, equal sizes -> left 6:
#     (6,7,(0,1),(0,1)) -> root 8 (cost 32 > 8).
#  4. second term, every pair 8: smallest key (A,B,(1,),(0,)) -> node 9 [a x c].
#  5. [9, E, F]: keys (E,9,(0,),(1,)), (F,9,(1,),(0,)), (E,F,(1,),(0,)):
#     smallest (E,F,(1,),(0,)) -> node 10 [c x a].
#  6. [9, 10]: 9.0-10.1 (a), 9.1-10.0 (c) -> root 11 (9,10,(0,1),(1,0)).
COSTLY_PAIR_EXPECTED = [(2, 1, (0,), (1,)), (3, 0, (1,), (0,)), (6, 7, (0, 1), (0, 1)),
                        (0, 1, (1,), (0,)), (4, 5, (1,), (0,)), (9, 10, (0, 1), (1, 0))]
COSTLY_PAIR_SHAPES = [(2, 2), (2, 2), (2, 16), (16, 2), (2, 2), (2, 2)]


def test_rarer_costlier_pair_beats_frequent_cheap_one():
    """count x cost, not count: the once-occurring C.B (cost 64) is built
    before the twice-occurring A.B (cost 8); the whole DAG as derived by
    hand above, and both traces equal einsum."""
    lt = 2
    dag = D.Dag(lt)
    A, B, Cm, Dm, E, F = (dag.add_leaf(s, leaf_index=i) for i, s in enumerate(COSTLY_PAIR_SHAPES))
    roots = PS.select_paths(dag, [_ring4(A, B, Cm, Dm), _ring4(A, B, E, F)])
    got = [(dag.nodes[u].left, dag.nodes[u].right, tuple(dag.nodes[u].la), tuple(dag.nodes[u].ra))
           for u in dag.non_leaf()]
    assert got == COSTLY_PAIR_EXPECTED
    assert roots == [8, 11]
    rng = np.random.default_rng(2)
    data = [rng.standard_normal((lt,) + s) + 1j * rng.standard_normal((lt,) + s)
            for s in COSTLY_PAIR_SHAPES]
    vals = C.evaluate(dag, lambda u: data[u], roots)
    want1 = np.einsum("tab,tbc,tcd,tda->t", data[0], data[1], data[2], data[3])
    want2 = np.einsum("tab,tbc,tce,tea->t", data[0], data[1], data[4], data[5])
    assert np.allclose(vals[8], want1, rtol=1e-12, atol=0)
    assert np.allclose(vals[11], want2, rtol=1e-12, atol=0)
