"""Pins of the oracle's correlator values (oracle.contract).

* ``contract_pair`` against explicit nested Python loops on tiny tensors with
  non-trivial axis pairings (brute force, no library call).
* ``evaluate`` (node by node) against ``brute_force`` (one direct sum over
  all index labels of the tree) on the tiny workload at reduced N.
* Closed forms: identity leaves give Tr(1) = N (meson ring) or 4N (with a
  spin ring); Tr(A A^dagger) = ||A||_F^2 (real, non-negative); a ring's value
  does not depend on the bracketing or on a cyclic rotation of the ring.
* A two-matrix root equals numpy.einsum of its definition (library check).
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D


def _rand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_contract_pair_against_loops():
    rng = np.random.default_rng(1)
    lt = 2
    A = _rand(rng, (lt, 2, 3, 4))
    B = _rand(rng, (lt, 4, 5, 2))
    la, ra = (2, 0), (0, 2)      # A axis 2 (4) with B axis 0, A axis 0 (2) with B axis 2
    out = C.contract_pair(A, B, la, ra)
    assert out.shape == (lt, 3, 5)
    ref = np.zeros((lt, 3, 5), dtype=complex)
    for t in range(lt):
        for i1 in range(3):
            for j1 in range(5):
                s = 0j
                for c0 in range(4):
                    for c1 in range(2):
                        s += A[t, c1, i1, c0] * B[t, c0, j1, c1]
                ref[t, i1, j1] = s
    assert np.abs(out - ref).max() < 1e-12


def _leaf_fn(wl, dag):
    cache = {}

    def f(u):
        li = dag.nodes[u].leaf_index
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    return f


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_evaluate_matches_brute_force(seed):
    wl = synth.make_workload("tiny", seed=seed, nvec=5)
    dag, _ = D.build_from_workload(wl)
    lf = _leaf_fn(wl, dag)
    vals = C.evaluate(dag, lf)
    assert set(vals) == set(dag.roots())
    for r in dag.roots():
        bf = C.brute_force(dag, r, lf)
        assert bf.shape == (wl.lt,)
        err = np.linalg.norm(vals[r] - bf) / np.linalg.norm(bf)
        assert err < 1e-13, (r, err)


def test_evaluate_matches_brute_force_full_tiny():
    wl = synth.make_workload("tiny")
    dag, _ = D.build_from_workload(wl)
    lf = _leaf_fn(wl, dag)
    vals = C.evaluate(dag, lf)
    r = min(dag.roots(), key=lambda r: len(C.expand_tree(dag, r)[0]))
    bf = C.brute_force(dag, r, lf)
    assert np.linalg.norm(vals[r] - bf) / np.linalg.norm(bf) < 1e-13


def _ring_dag(lt, n, kinds, bracket):
    """Ring of M/P leaves (one leaf node per position) built with the
    generator's own request logic for a fixed bracketing."""
    link = synth.workloads._ring_links(kinds)
    shapes = {"M": (n, n), "P": (4, 4, n, n)}
    exts = [shapes[k] for k in kinds]
    pend = synth.ring_requests(kinds, link, bracket, exts, 10 ** 9)
    assert pend is not None
    dag = D.Dag(lt)
    for e in exts:
        dag.add_leaf(e)
    ids = []
    for (lref, rref, la, ra) in pend:
        def res(r):
            return r[1] if r[0] == "leaf" else ids[r[1]]
        ids.append(dag.add_contraction(res(lref), res(rref), la, ra))
    return dag, ids[-1]


@pytest.mark.parametrize("kinds", [("M", "M"), ("M", "M", "M"), ("M", "P", "M", "P"),
                                   ("P", "P"), ("P", "M", "P", "P", "M")])
def test_identity_ring_closed_form(kinds):
    lt, n = 3, 5
    eye_m = np.broadcast_to(np.eye(n), (lt, n, n)).astype(complex)
    eye_p = np.broadcast_to(np.einsum("ab,cd->abcd", np.eye(4), np.eye(n)), (lt, 4, 4, n, n)).astype(complex)
    for br in itertools.islice(synth.workloads._all_brackets(0, len(kinds) - 1), 6):
        dag, root = _ring_dag(lt, n, list(kinds), br)
        vals = C.evaluate(dag, lambda u: eye_p if len(dag.nodes[u].extents) == 4 else eye_m)
        expect = n * (4 if "P" in kinds else 1)
        assert np.allclose(vals[root], expect, atol=1e-12, rtol=0)


def test_trace_a_adagger_is_frobenius_norm():
    lt, n = 4, 7
    rng = np.random.default_rng(3)
    A = _rand(rng, (lt, n, n))
    Ad = np.conj(np.transpose(A, (0, 2, 1)))
    dag, root = _ring_dag(lt, n, ["M", "M"], (0, 1))
    vals = C.evaluate(dag, lambda u: A if u == 0 else Ad)
    fro = np.sum(np.abs(A) ** 2, axis=(1, 2))
    assert np.abs(vals[root] - fro).max() < 1e-11 * fro.max()
    assert np.abs(vals[root].imag).max() < 1e-11 * fro.max()


def test_bracketing_and_rotation_invariance():
    lt, n = 2, 6
    rng = np.random.default_rng(4)
    kinds = ["P", "M", "P", "M", "P"]
    data = [_rand(rng, (lt, 4, 4, n, n)) if k == "P" else _rand(rng, (lt, n, n)) for k in kinds]
    ref = None
    for rot in range(len(kinds)):
        rk = kinds[rot:] + kinds[:rot]
        rd = data[rot:] + data[:rot]
        for br in itertools.islice(synth.workloads._all_brackets(0, len(kinds) - 1), 14):
            dag, root = _ring_dag(lt, n, rk, br)
            v = C.evaluate(dag, lambda u: rd[u])[root]
            if ref is None:
                ref = v
            assert np.linalg.norm(v - ref) / np.linalg.norm(ref) < 1e-12


def test_two_matrix_root_matches_einsum():
    lt, n = 3, 9
    rng = np.random.default_rng(5)
    A, B = _rand(rng, (lt, n, n)), _rand(rng, (lt, n, n))
    dag, root = _ring_dag(lt, n, ["M", "M"], (0, 1))
    v = C.evaluate(dag, lambda u: A if u == 0 else B)[root]
    assert np.abs(v - np.einsum("tab,tba->t", A, B)).max() < 1e-12


def test_planted_transpose_mistake_caught():
    """Plant a plausible bug (right operand's pair order reversed) in the
    oracle and check that the brute-force pin catches it.  N = 4 equals the
    spin extent, so the wrong pairing still has matching shapes."""
    orig = C.contract_pair

    def buggy(A, B, la, ra):
        return orig(A, B, la, tuple(reversed(ra)))
    wl = synth.make_workload("tiny", nvec=4)
    dag, _ = D.build_from_workload(wl)
    lf = _leaf_fn(wl, dag)
    C.contract_pair = buggy
    try:
        vals = C.evaluate(dag, lf)
    finally:
        C.contract_pair = orig
    bad = 0
    for r in dag.roots():
        bf = C.brute_force(dag, r, lf)
        if np.linalg.norm(vals[r] - bf) > 1e-6 * np.linalg.norm(bf):
            bad += 1
    assert bad > 0
