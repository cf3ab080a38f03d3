"""Failure paths of the executor, made on the host (no GPU fault).

* Injected failures of the library's own cudaMalloc, cudaHostAlloc and
  cudaMemcpyAsync calls (lqc_test_inject_failure): the call returns
  LQC_ERR_CUDA naming the failed step, the DAG stays destroyable, and the
  next execute (nothing armed) succeeds with correlators equal to the oracle
  -- with and without CUDA-graph capture, and for leaf staging.
* lqc_dag_wait with a 1 ms limit on a long execute returns LQC_ERR_TIMEOUT,
  then LQC_OK on a normal wait.
* The tensor-core kernels' bounded mbarrier wait: a wait that nothing
  arrives on expires after a host-set 1 ms limit, sets the device error
  word (read as LQC_ERR_TIMEOUT) and returns; the context stays usable.
* Executor-counted figures: a plan changed on the host (every FREE moved to
  the end, planned figures kept) makes the counted peak differ from the
  planned one while the results stay those of the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D

L = pytest.importorskip("paper_2511_02257_b300")

SITE_DEVICE_ALLOC, SITE_PINNED_ALLOC, SITE_COPY = 0, 1, 2


def test_inject_arguments():
    assert L.lqc_test_inject_failure(3, 0) == L.LQC_ERR_ARG
    assert L.lqc_test_inject_failure(0, -1) == L.LQC_ERR_ARG
    assert L.lqc_test_inject_failure(-2, 0) == L.LQC_ERR_ARG
    assert L.lqc_test_inject_failure(-1, 0) == L.LQC_OK
    assert L.lqc_test_expire_wait(0, None) == L.LQC_ERR_ARG
    assert L.lqc_test_expire_wait(2 * 10 ** 9, None) == L.LQC_ERR_ARG


def test_tamper_needs_an_unlimited_plan():
    d = L.Dag(2)
    a = d.add_leaf((3, 3))
    d.add_contraction(a, a, [0, 1], [1, 0])
    assert L.lqc_test_tamper_plan(d.h, 1) == L.LQC_ERR_STATE
    d.schedule("tree", "lru", 1 << 20)
    assert L.lqc_test_tamper_plan(d.h, 1) == L.LQC_ERR_ARG
    d.schedule("tree", "lru", 0)
    assert L.lqc_test_tamper_plan(d.h, 2) == L.LQC_ERR_ARG
    assert L.lqc_test_tamper_plan(d.h, 1) == L.LQC_OK


# ---------------------------------------------------------------- GPU
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _tiny(precision="fp64", seed=0):
    wl = synth.make_workload("tiny", seed=seed)
    od, _ = D.build_from_workload(wl)
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
    nd, _ = L.build_dag(wl, precision=precision, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    return wl, nd, ref


def _check(nd, ref, tol):
    for r in ref:
        v = nd.read_correlator(r)
        assert np.linalg.norm(v - ref[r]) <= tol * np.linalg.norm(ref[r]), r


@pytest.fixture
def disarm():
    yield
    L.lqc_test_inject_failure(-1, 0)


@pytest.mark.gpu
@pytest.mark.parametrize("graph", [0, 1])
@pytest.mark.parametrize("site,skip,what", [(SITE_DEVICE_ALLOC, 0, "arena"),
                                            (SITE_DEVICE_ALLOC, 1, "results"),
                                            (SITE_COPY, 0, "H2D load"),
                                            (SITE_COPY, 4, "H2D load")])
def test_injected_failure_then_recovery(site, skip, what, graph, disarm):
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    _, nd, ref = _tiny()
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, graph)
    nd.schedule("tree", "lru", 0)
    assert L.lqc_test_inject_failure(site, skip) == L.LQC_OK
    with pytest.raises(L.LqcError) as ei:
        nd.execute(stream)
    assert ei.value.code == L.LQC_ERR_CUDA
    assert what in str(ei.value)
    torch.cuda.synchronize()                  # whatever was issued before the failure
    L.lqc_test_inject_failure(-1, 0)
    nd.execute(stream)
    nd.wait()
    _check(nd, ref, 1e-12)
    nd.execute(stream)                         # and again (graph replay)
    _check(nd, ref, 1e-12)
    nd.close()


@pytest.mark.gpu
def test_injected_staging_failure(disarm):
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    _, nd, ref = _tiny()
    nd.schedule("tree", "lru", 0)
    for site in (SITE_DEVICE_ALLOC, SITE_COPY):
        L.lqc_test_inject_failure(site, 2)
        with pytest.raises(L.LqcError) as ei:
            nd.stage_leaves(stream)
        assert ei.value.code == L.LQC_ERR_CUDA
        L.lqc_test_inject_failure(-1, 0)
    nd.stage_leaves(stream)
    nd.execute(stream)
    _check(nd, ref, 1e-12)
    nd.close()


@pytest.mark.gpu
def test_injected_pinned_writeback_arena_failure(disarm):
    """A plan that writes intermediates back needs the pinned write-back
    arena; its allocation failing fails the execute, then it recovers."""
    torch = _cuda()
    from oracle import memory as M
    from oracle import schedule as S
    stream = torch.cuda.current_stream().cuda_stream
    wl = synth.make_workload("memory_pressure", lt=4, nvec=12, n_functions=30)
    od, _ = D.build_from_workload(wl)
    ref = C.evaluate(od, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
    budget = M.replay(od, S.naive(od)).stats.peak_exec // 4
    nd, _ = L.build_dag(wl, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    planned = nd.schedule("naive", "lru", budget)
    assert planned["d2h_bytes"] > 0
    L.lqc_test_inject_failure(SITE_PINNED_ALLOC, 0)
    with pytest.raises(L.LqcError) as ei:
        nd.execute(stream)
    assert ei.value.code == L.LQC_ERR_CUDA and "write-back" in str(ei.value)
    L.lqc_test_inject_failure(-1, 0)
    nd.execute(stream)
    _check(nd, ref, 1e-12)
    assert nd.stats() == planned
    nd.close()


@pytest.mark.gpu
def test_wait_timeout_then_ok():
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    wl = synth.make_workload("multi_meson", n_functions=60)
    nd, _ = L.build_dag(wl, leaf_data_fn=lambda li: synth.leaf_data(wl, li))
    nd.schedule("tree", "lru", 0)
    nd.execute(stream)
    nd.wait()                                  # first execute: program and arena
    nd.execute(stream)                         # FP64, hundreds of milliseconds
    rc = L.lqc_dag_wait(nd.h, 1)
    assert rc == L.LQC_ERR_TIMEOUT
    assert L.lqc_dag_wait(nd.h, 60000) == L.LQC_OK
    v = nd.read_all_correlators()
    assert np.all(np.isfinite(v))
    nd.close()


@pytest.mark.gpu
def test_device_bounded_wait_expires():
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    assert L.lqc_test_expire_wait(1_000_000, stream) == L.LQC_ERR_TIMEOUT
    assert L.lqc_mixed_error(0) == 0           # the probe cleared the word again
    # the context is intact: the tensor-core path still runs and is right
    _, nd, ref = _tiny("tf32x3")
    nd.set_option(L.LQC_OPT_FUSED_MAX_N, 1 << 30)
    nd.schedule("tree", "lru", 0)
    nd.execute(stream)
    nd.wait()
    _check(nd, ref, 1e-6)
    nd.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,window", [("fp64", 0), ("tf32x3", 64)])
def test_counted_figures_follow_the_executed_plan(precision, window):
    torch = _cuda()
    stream = torch.cuda.current_stream().cuda_stream
    _, nd, ref = _tiny(precision)
    nd.set_option(L.LQC_OPT_WINDOW, window)
    planned = nd.schedule("tree", "lru", 0)
    nd.execute(stream)
    assert nd.stats() == planned               # the plan as scheduled
    assert L.lqc_test_tamper_plan(nd.h, 1) == L.LQC_OK
    nd.execute(stream)
    nd.wait()
    st = nd.stats()
    # every contraction output and every leaf some contraction reads
    used = set()
    for u in range(nd.num_nodes()):
        left, right, _, _ = nd.node_operands(u)
        if left >= 0:
            used.update((u, left, right))
    total = sum(nd.node_info(u)["size"] for u in used)
    assert st["peak_exec"] > planned["peak_exec"]
    assert st["peak_exec"] == total            # nothing freed until the end
    assert {k: st[k] for k in st if k != "peak_exec"} == \
        {k: planned[k] for k in planned if k != "peak_exec"}
    _check(nd, ref, 1e-12 if precision == "fp64" else 1e-6)
    nd.close()
