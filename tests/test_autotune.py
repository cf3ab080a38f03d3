"""The mixed path's autotuner (window size, fused-form limit, k-split
policy) and its options.

* host checks: state and argument errors, option ranges (no GPU needed);
* GPU: every extreme setting of the options gives correlators within the
  TF32x3 tolerance of the oracle; the autotuner times every candidate,
  applies the fastest, and the tuned DAG still matches the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D

L = pytest.importorskip("paper_2511_02257_b300")
TOL = 1e-6


def test_autotune_host_errors():
    d = L.Dag(4, "tf32x3")
    a = d.add_leaf((4, 4))
    d.add_contraction(a, a, [1], [0])
    with pytest.raises(L.LqcError) as ei:
        d.autotune()
    assert ei.value.code == L.LQC_ERR_STATE           # not scheduled
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 0)
    d.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    d.set_option(L.LQC_OPT_SPLIT_POLICY, 1)
    for opt, bad in ((L.LQC_OPT_SPLIT_POLICY, 2), (L.LQC_OPT_FUSED_MAX_N, -1)):
        with pytest.raises(L.LqcError) as ei:
            d.set_option(opt, bad)
        assert ei.value.code == L.LQC_ERR_ARG
    d64 = L.Dag(4, "fp64")
    a = d64.add_leaf((4, 4))
    d64.add_contraction(a, a, [1], [0])
    d64.schedule("tree")
    with pytest.raises(L.LqcError) as ei:
        d64.autotune()
    assert ei.value.code == L.LQC_ERR_ARG             # FP64 has nothing to tune


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _workload():
    # propagators (N' = 16*N columns: plane form by default) and mesons
    return synth.make_workload("multi_meson", n_functions=30, nvec=32, lt=8)


def _ref(wl):
    od, _ = D.build_from_workload(wl)
    return C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))


def _errs(nd, ref):
    return max(float(np.linalg.norm(nd.read_correlator(r) - ref[r]) / np.linalg.norm(ref[r]))
               for r in ref)


@pytest.mark.gpu
@pytest.mark.parametrize("window,fused,split", [(0, 0, 0), (0, 1 << 30, 1), (64, 1 << 30, 0),
                                                (64, 0, 1), (256, 64, 1)])
def test_option_extremes_match_oracle(window, fused, split):
    torch = _gpu()
    wl = _workload()
    ref = _ref(wl)
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree")
    nd.set_option(L.LQC_OPT_WINDOW, window)
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, fused)
    nd.set_option(L.LQC_OPT_SPLIT_POLICY, split)
    nd.execute(torch.cuda.current_stream().cuda_stream)
    assert _errs(nd, ref) < TOL


@pytest.mark.gpu
def test_autotune_picks_fastest_and_stays_correct():
    torch = _gpu()
    wl = _workload()
    ref = _ref(wl)
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree")
    stream = torch.cuda.current_stream().cuda_stream
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    nd.stage_leaves(stream)
    entries = nd.autotune(stream, reps=2)
    assert len(entries) == 32
    assert {(e["window"], e["fused_max_n"], e["split_policy"], e["fused_kernel"])
            for e in entries} == \
        {(w, f, s, 0) for w in (0, 64, 512, 4096) for f in (0, 64) for s in (0, 1)} | \
        {(w, 1 << 30, s, k) for w in (0, 64, 512, 4096) for s in (0, 1) for k in (0, 2)}
    assert all(e["ms"] > 0 for e in entries)
    best = entries[0]
    assert best["ms"] == min(e["ms"] for e in entries)
    nd.execute(stream)
    assert _errs(nd, ref) < TOL
