"""GPU parity of the FP64 path against the CPU oracle (complex128).

Single contractions through the C-ABI entry points on device buffers, then
whole DAGs through lqc_dag_execute: every correlator within 1e-12
norm-wise relative error of the oracle (per correlator, over t), identical
bits across schedules / budgets / options, executor counters equal to the
planned figures.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D
from oracle import memory as M
from oracle import schedule as S

torch = pytest.importorskip("torch")
L = pytest.importorskip("paper_2511_02257_b300")

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def rel_err(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def _rand(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def _ext(shape):
    import ctypes
    a = np.asarray(shape, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _pairs(xs):
    import ctypes
    a = np.asarray(xs, dtype=np.intc)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


CASES = [
    # (shape A, shape B, la, ra)    -- ragged tails, permuted pairings, ranks 1..5
    ((17, 33), (33, 9), (1,), (0,)),
    ((64, 64), (64, 64), (1,), (0,)),
    ((64, 64), (64, 64), (0,), (1,)),                 # both operands transposed
    ((4, 4, 19, 21), (21, 13), (3,), (0,)),           # P x M over distillation
    ((4, 4, 24, 24), (4, 4, 24, 24), (1, 3), (0, 2)),  # P x P over spin + dist
    ((4, 4, 24, 24), (4, 4, 24, 24), (3, 1), (2, 0)),  # same pairs, other order
    ((12, 12, 12), (12, 12, 12), (1, 2), (0, 1)),     # B x B over two legs
    ((12, 12, 12), (12, 7), (2,), (0,)),              # B x M over one leg
    ((5, 3, 7, 2), (2, 7, 6), (3, 2), (0, 1)),
    ((70,), (70, 3), (0,), (0,)),                     # M = 1
    ((3, 130), (130,), (1,), (0,)),                   # N = 1
    ((129, 65), (65, 131), (1,), (0,)),               # several tiles + tails
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("lt", [1, 5])
def test_contract_fp64_vs_oracle(case, lt):
    sa, sb, la, ra = case
    rng = np.random.default_rng(hash((sa, sb, la, lt)) % 2 ** 32)
    A = _rand(rng, (lt,) + sa)
    B = _rand(rng, (lt,) + sb)
    ref = C.contract_pair(A, B, la, ra)
    dA, dB = _dev(A), _dev(B)
    dC = torch.full((lt,) + ref.shape[1:], complex("nan"), dtype=torch.complex128, device="cuda")
    ea, pa = _ext(sa)
    eb, pb = _ext(sb)
    xla, pla = _pairs(la)
    xra, pra = _pairs(ra)
    rc = L.lqc_contract_fp64(_ptr(dA), len(sa), pa, _ptr(dB), len(sb), pb, len(la), pla, pra, lt,
                             _ptr(dC), None)
    assert rc == 0
    torch.cuda.synchronize()
    got = dC.cpu().numpy()
    assert rel_err(got, ref) < TOL


@pytest.mark.parametrize("case", [((16, 16), (16, 16), (0, 1), (1, 0)),
                                  ((4, 4, 20, 20), (4, 4, 20, 20), (0, 1, 2, 3), (1, 0, 3, 2)),
                                  ((9, 10, 11), (11, 9, 10), (0, 1, 2), (1, 2, 0)),
                                  ((300,), (300,), (0,), (0,)),
                                  ((64, 64, 64), (64, 64, 64), (0, 1, 2), (0, 1, 2))])
@pytest.mark.parametrize("lt", [1, 3, 64])
def test_contract_all_fp64_vs_oracle(case, lt):
    sa, sb, la, ra = case
    rng = np.random.default_rng(7)
    A = _rand(rng, (lt,) + sa)
    B = _rand(rng, (lt,) + sb)
    ref = C.contract_pair(A, B, la, ra)
    dA, dB = _dev(A), _dev(B)
    dC = torch.zeros(lt, dtype=torch.complex128, device="cuda")
    S_ = int(np.prod(sa))
    nbytes = L.lqc_contract_all_scratch_bytes(lt, S_)
    scratch = torch.empty(max(nbytes, 16), dtype=torch.uint8, device="cuda")
    ea, pa = _ext(sa)
    eb, pb = _ext(sb)
    xla, pla = _pairs(la)
    xra, pra = _pairs(ra)
    rc = L.lqc_contract_all_fp64(_ptr(dA), len(sa), pa, _ptr(dB), len(sb), pb, len(la), pla, pra,
                                 lt, _ptr(dC), _ptr(scratch), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert rel_err(dC.cpu().numpy(), ref) < TOL


def test_contract_rejects_bad_pairs():
    ea, pa = _ext((3, 4))
    eb, pb = _ext((5, 6))
    xla, pla = _pairs((1,))
    xra, pra = _pairs((0,))
    t = torch.zeros(100, dtype=torch.complex128, device="cuda")
    rc = L.lqc_contract_fp64(_ptr(t), 2, pa, _ptr(t), 2, pb, 1, pla, pra, 1, _ptr(t), None)
    assert rc == L.LQC_ERR_ARG


# ---------------------------------------------------------------- whole DAGs
def _oracle(wl, roots=None):
    od, ids = D.build_from_workload(wl)
    cache = {}

    def lf(u):
        li = od.nodes[u].leaf_index
        if li not in cache:
            cache[li] = synth.leaf_data(wl, li)
        return cache[li]
    return od, C.evaluate(od, lf, roots)


def _native(wl, **kw):
    return L.build_dag(wl, leaf_data_fn=lambda li: synth.leaf_data(wl, li), **kw)


def _run(nd, policy="tree", evict="lru", budget=0):
    planned = nd.schedule(policy, evict, budget)
    stream = torch.cuda.current_stream().cuda_stream
    nd.execute(stream)
    nd.wait()
    vals = {r: nd.read_correlator(r) for r in nd.roots()}
    return planned, vals


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_dag_all_schedules(seed):
    wl = synth.make_workload("tiny", seed=seed)
    od, ref = _oracle(wl)
    nd, _ = _native(wl)
    base = None
    for pol in ("tree", "naive", "sibling", "rsgs", "node"):
        planned, vals = _run(nd, pol)
        assert set(vals) == set(ref)
        for r in ref:
            assert rel_err(vals[r], ref[r]) < TOL, (pol, r)
        if base is None:
            base = vals
        for r in ref:                          # schedules do not change a single bit
            assert np.array_equal(vals[r].view(np.float64), base[r].view(np.float64))
        assert nd.stats() == planned


def test_tiny_dag_brute_force_and_read_all():
    wl = synth.make_workload("tiny", nvec=6)
    od, _ = D.build_from_workload(wl)
    nd, _ = _native(wl)
    _, vals = _run(nd, "tree")
    allv = nd.read_all_correlators()
    for i, r in enumerate(nd.roots()):
        bf = C.brute_force(od, r, lambda u: synth.leaf_data(wl, od.nodes[u].leaf_index))
        assert rel_err(vals[r], bf) < TOL
        assert np.array_equal(allv[i], vals[r])


@pytest.mark.parametrize("evict", ["lru", "next_use"])
def test_budgeted_eviction_matches_oracle(evict):
    """Memory-pressure generator at reduced size; the budget forces
    evictions and write-backs for the naive order."""
    wl = synth.make_workload("memory_pressure", lt=4, nvec=12, n_functions=60)
    od, ref = _oracle(wl)
    free = M.replay(od, S.naive(od))
    budget = free.stats.peak_exec // 4
    nd, _ = _native(wl)
    base = None
    evicted = {}
    for pol in ("naive", "sibling", "tree", "rsgs", "node"):
        planned, vals = _run(nd, pol, evict, budget)
        oplan = M.replay(od, S.SCHEDULERS[pol](od), budget=budget, policy=evict)
        assert nd.order() == S.SCHEDULERS[pol](od), pol
        assert tuple(planned[k] for k in planned) == oplan.stats.as_tuple()
        assert nd.stats() == planned
        info = nd.exec_info()
        # copies = the plan's + those placement adds to keep the arena in the budget
        assert info["copied_h2d"] == planned["h2d_bytes"] + info["extra_h2d_bytes"]
        assert info["copied_d2h"] == planned["d2h_bytes"] + info["extra_d2h_bytes"]
        assert info["arena_bytes"] <= budget
        for r in ref:
            assert rel_err(vals[r], ref[r]) < TOL, (pol, r)
        if base is None:
            base = vals
        for r in ref:           # orders, budgets and evictions do not change a bit
            assert np.array_equal(vals[r].view(np.float64), base[r].view(np.float64)), pol
        evicted[pol] = planned["n_evict"]
    assert evicted["naive"] > 0


def test_naive_budget_really_evicts():
    wl = synth.make_workload("memory_pressure", lt=4, nvec=12, n_functions=60)
    od, ref = _oracle(wl)
    budget = M.replay(od, S.naive(od)).stats.peak_exec // 4
    nd, _ = _native(wl)
    planned, vals = _run(nd, "naive", "lru", budget)
    assert planned["n_evict"] > 0 and planned["n_d2h"] > 0
    nd.set_option(L.LQC_OPT_POISON, 1)         # freed / evicted memory turned to NaN
    stream = torch.cuda.current_stream().cuda_stream
    nd.execute(stream)
    for r in ref:
        v = nd.read_correlator(r)
        assert np.all(np.isfinite(v))
        assert np.array_equal(v.view(np.float64), vals[r].view(np.float64))


def test_graph_and_staged_modes_bit_identical():
    wl = synth.make_workload("tiny", seed=3)
    nd, _ = _native(wl)
    _, base = _run(nd, "tree")
    stream = torch.cuda.current_stream().cuda_stream
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
    for _ in range(2):
        nd.execute(stream)
        for r, v in base.items():
            assert np.array_equal(nd.read_correlator(r).view(np.float64), v.view(np.float64))
    nd.stage_leaves(stream)
    nd.execute(stream)
    assert nd.stats()["h2d_bytes"] == 0
    for r, v in base.items():
        assert np.array_equal(nd.read_correlator(r).view(np.float64), v.view(np.float64))
    nd.unstage_leaves()
    nd.set_option(L.LQC_OPT_CUDA_GRAPH, 0)


def test_set_leaf_data_changes_result():
    wl = synth.make_workload("tiny", seed=4)
    nd, ids = _native(wl)
    _, base = _run(nd, "tree")
    leaf0 = synth.leaf_data(wl, 0)
    nd.set_leaf_data(ids[0], 2.0 * leaf0)
    stream = torch.cuda.current_stream().cuda_stream
    nd.execute(stream)
    od, _ = D.build_from_workload(wl)
    changed = 0
    for r, v in base.items():
        new = nd.read_correlator(r)
        if 0 in od.tree(r):
            changed += 1
            # a leaf enters a ring linearly (or quadratically if it occurs twice)
            ratio = np.linalg.norm(new) / np.linalg.norm(v)
            assert min(abs(ratio - 2.0), abs(ratio - 4.0)) < 1e-9
    assert changed > 0


def test_multi_meson_full_size_all_roots():
    """The benchmark workload at full size: every correlator of the 200
    multi-meson functions against the oracle."""
    wl = synth.make_workload("multi_meson")
    od, ref = _oracle(wl)
    nd, _ = _native(wl)
    planned, vals = _run(nd, "tree")
    errs = [rel_err(vals[r], ref[r]) for r in ref]
    assert max(errs) < TOL, max(errs)
    assert nd.stats() == planned


def test_baryon_fp64_sampled_roots():
    """Baryon-like DAG (B_64 leaves contracted over one or two legs, with
    meson insertions): a seeded sample of correlators against the oracle."""
    wl = synth.make_workload("baryon")
    od, _ = D.build_from_workload(wl)
    rng = np.random.default_rng(5)
    roots = [int(r) for r in rng.choice(od.roots(), size=16, replace=False)]
    _, ref = _oracle(wl, roots)
    nd, _ = _native(wl)
    planned = nd.schedule("tree")
    nd.execute(torch.cuda.current_stream().cuda_stream)
    errs = [rel_err(nd.read_correlator(r), ref[r]) for r in roots]
    assert max(errs) < TOL, max(errs)
    assert nd.stats() == planned
