"""The memory-pressure workload at full size (Lt 128, N 128, 4,826
contractions, leaves of 32 MiB and 512 MiB in complex128) under its 24 GiB
device budget, in the launch configuration the bench times for it: TF32x3,
tree order, grouped windows, CUDA graph, leaves from the library's pinned
host store.  The oracle cannot evaluate the whole DAG in seconds, so a
seeded sample of correlators is checked, each on its own descendant
closure (<= 1e-6), and the executor's counters must equal the plan's.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D

L = pytest.importorskip("paper_2511_02257_b300")


@pytest.mark.gpu
def test_memory_pressure_full_size_sampled_roots_tf32x3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("memory_pressure")
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        leaves = list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=lambda li: leaves[li])
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    planned = nd.schedule("tree", "lru", wl.budget_bytes)
    assert planned["peak_exec"] <= wl.budget_bytes
    nd.execute(torch.cuda.current_stream().cuda_stream)
    assert nd.stats() == planned
    od, _ = D.build_from_workload(wl)
    rng = np.random.default_rng(11)
    pick = sorted(rng.choice(od.roots(), size=12, replace=False).tolist())
    ref = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index], pick)
    errs = {r: float(np.linalg.norm(nd.read_correlator(r) - ref[r]) / np.linalg.norm(ref[r]))
            for r in pick}
    assert max(errs.values()) < 1e-6, errs


@pytest.mark.gpu
def test_memory_pressure_full_size_fp64_with_evictions():
    """The same workload on the FP64 path (complex128 storage, model peak
    12.4 GiB) under an 8 GiB budget, so that the tree order evicts
    intermediates to pinned host memory and reloads them: 12 seeded roots
    against the oracle (<= 1e-12), counters equal to the plan's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("memory_pressure")
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        leaves = list(ex.map(lambda li: synth.leaf_data(wl, li), range(len(wl.leaves))))
    nd, _ = L.build_dag(wl, precision="fp64", leaf_data_fn=lambda li: leaves[li])
    planned = nd.schedule("tree", "lru", 8 << 30)
    assert planned["n_evict"] > 0 and planned["d2h_bytes"] > 0
    nd.execute(torch.cuda.current_stream().cuda_stream)
    nd.wait(600000)
    assert nd.stats() == planned
    od, _ = D.build_from_workload(wl)
    rng = np.random.default_rng(12)
    pick = sorted(rng.choice(od.roots(), size=12, replace=False).tolist())
    ref = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index], pick)
    errs = {r: float(np.linalg.norm(nd.read_correlator(r) - ref[r]) / np.linalg.norm(ref[r]))
            for r in pick}
    assert max(errs.values()) < 1e-12, errs


@pytest.mark.gpu
@pytest.mark.parametrize("budget_gib", [24, 8])
def test_arena_within_budget_all_schedulers(budget_gib):
    """The full memory-pressure workload (TF32x3 storage) under 24 and 8 GiB:
    for every scheduler the physical arena stays within the budget (the
    best-fit placement fragments; placement moves tensors to the host where
    it must), the counted figures equal the plan's, copies = plan + the
    reported extra moves, and every correlator is bit-identical to the tree
    order's at 24 GiB."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("memory_pressure")
    cache = {}

    def leaf(li):
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    nd, _ = L.build_dag(wl, precision="tf32x3", leaf_data_fn=leaf)
    budget = budget_gib << 30
    stream = torch.cuda.current_stream().cuda_stream
    base = None
    for pol in ("tree", "naive", "sibling", "rsgs", "node"):
        planned = nd.schedule(pol, "lru", budget)
        nd.execute(stream)
        vals = nd.read_all_correlators()
        info = nd.exec_info()
        assert info["arena_bytes"] <= budget, (pol, info["arena_bytes"])
        assert nd.stats() == planned, pol
        assert info["copied_h2d"] == planned["h2d_bytes"] + info["extra_h2d_bytes"]
        assert info["copied_d2h"] == planned["d2h_bytes"] + info["extra_d2h_bytes"]
        assert L.lqc_mixed_error(1) == 0
        if base is None:
            base = vals
        assert np.array_equal(vals.view(np.float64), base.view(np.float64)), pol
    nd.close()
