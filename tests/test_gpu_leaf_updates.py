"""New leaf data between executes: a caller streaming leaves every step.

The library's host pass (normalisation and conversion, or the FP64 copy)
runs when the data is set.  New data whose largest component stays within
the leaf's power-of-two range keeps the exponent, so the program and its
CUDA graph are reused (only staged device copies are refreshed); data of a
new magnitude changes the exponent and the next execute builds a program.
Either way the correlators are those of the oracle on the new data.
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D

L = pytest.importorskip("paper_2511_02257_b300")


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _check(nd, ref, tol):
    for r in ref:
        v = nd.read_correlator(r)
        assert np.linalg.norm(v - ref[r]) <= tol * np.linalg.norm(ref[r]), r


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "tf32x3"])
@pytest.mark.parametrize("staged", [False, True])
def test_new_leaf_data_between_executes(precision, staged):
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-12 if precision == "fp64" else 1e-6
    wl = synth.make_workload("tiny", seed=0)
    od, _ = D.build_from_workload(wl)
    nd, _ = L.build_dag(wl, precision=precision,
                        leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    nd.schedule("tree", "lru", 0)
    if staged:
        nd.stage_leaves(stream)
    nd.execute(stream)
    nd.wait()
    n0 = nd.exec_info()["n_programs"]
    leaves = [u for u, n in enumerate(od.nodes) if n.is_leaf]
    rng = np.random.default_rng(5)

    def feed(factor):
        data = {}
        for u in leaves:
            x = synth.leaf_data(wl, od.nodes[u].leaf_index)
            # new values, largest component at most 0.71 of the old one's
            y = factor * 0.5 * x * np.exp(2j * np.pi * rng.random(x.shape))
            nd.set_leaf_data(u, y)
            data[u] = y
        return C.evaluate(od, lambda u: data[u])

    # same magnitude range: the program and its graph are reused
    for _ in range(2):
        ref = feed(1.0)
        nd.execute(stream)
        nd.wait()
        _check(nd, ref, tol)
        assert nd.exec_info()["n_programs"] == n0
    # 2^40 larger: a new exponent for every mixed-precision leaf, one new
    # program (FP64 stores the values as they are)
    ref = feed(2.0 ** 40)
    nd.execute(stream)
    nd.wait()
    _check(nd, ref, tol)
    assert nd.exec_info()["n_programs"] == n0 + (0 if precision == "fp64" else 1)
    nd.close()
