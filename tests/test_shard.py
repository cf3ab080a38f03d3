"""Batch-axis (Lt) sharding of a DAG over ranks (paper_2511_02257_b300.shard).

* Slice split: contiguous, covering, balanced; too many ranks rejected.
* Every shard of a one-batch-extent DAG gets the full DAG's order under
  every scheduler and, under the scaled budget (B // Lt) * lt_g, the full
  plan's op list, with every byte figure scaled by lt_g / Lt (a node's size
  is Lt times a per-slice size).  The oracle's simulator gives the same
  figures for a shard built on its side.
* Values: the oracle evaluated on each rank's leaf slices and assembled
  equals the oracle on the full leaves, bit for bit (no arithmetic mixes
  time slices); assembly of ragged per-root batch extents.
* The end gather on gloo ranks (world size 2 and 3).
* GPU: shards executed one after another on one device, assembled, against
  the oracle (FP64 <= 1e-12, TF32x3 <= 1e-6), including a batched DAG with
  one batch extent per part.
"""
import os
import socket
import sys

import numpy as np
import pytest

import synth
from oracle import contract as C
from oracle import dag as D
from oracle import memory as M
from oracle import schedule as S

L = pytest.importorskip("paper_2511_02257_b300")
from paper_2511_02257_b300 import shard as SH  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_lt_slices():
    for lt in (1, 7, 10, 64, 129):
        for world in range(1, min(lt, 9) + 1):
            sl = SH.lt_slices(lt, world)
            assert sl[0][0] == 0 and sl[-1][1] == lt
            assert all(sl[g][1] == sl[g + 1][0] for g in range(world - 1))
            sizes = [b - a for a, b in sl]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
            assert sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        SH.lt_slices(3, 4)
    with pytest.raises(ValueError):
        SH.lt_slices(3, 0)


def _oracle_shard(wl, rank, world):
    t0, t1 = SH.lt_slices(wl.lt, world)[rank]
    od = D.Dag(t1 - t0)
    ids = []
    for li, lf in enumerate(wl.leaves):
        a, b = SH.lt_slices(wl.leaf_lt(li), world)[rank]
        ids.append(od.add_leaf(lf.extents, leaf_index=li, lt=b - a))
    for rq in wl.requests:
        ids.append(od.add_contraction(ids[rq.left], ids[rq.right], rq.la, rq.ra))
    return od


@pytest.mark.parametrize("name,kw,world", [("multi_meson", dict(n_functions=20, lt=10), 3),
                                           ("memory_pressure", dict(n_functions=24, lt=12), 4),
                                           ("baryon", dict(n_functions=12, lt=9), 2)])
def test_shard_orders_and_plans_scale(name, kw, world):
    wl = synth.make_workload(name, **kw)
    full, _ = L.build_dag(wl, with_data=False)
    od_full, _ = D.build_from_workload(wl)
    budget = M.replay(od_full, S.naive(od_full)).stats.peak_exec // 3
    budget -= budget % wl.lt
    for sched in ("naive", "sibling", "tree", "rsgs", "node"):
        st_full = full.schedule(sched, "lru", budget)
        order, plan = full.order(), full.plan()
        for g in range(world):
            t0, t1 = SH.lt_slices(wl.lt, world)[g]
            lt_g = t1 - t0
            nd, _ = L.build_dag(wl, with_data=False, shard=(g, world))
            bg = SH.shard_budget(budget, wl.lt, lt_g)
            st = nd.schedule(sched, "lru", bg)
            assert nd.order() == order
            assert nd.plan() == plan
            for k in ("peak_paper", "peak_exec", "h2d_bytes", "d2h_bytes"):
                assert st[k] * wl.lt == st_full[k] * lt_g, (sched, k)
            for k in ("n_evict", "n_h2d", "n_d2h"):
                assert st[k] == st_full[k]
            if sched == "tree" and g == world - 1:
                od = _oracle_shard(wl, g, world)
                oplan = M.replay(od, S.SCHEDULERS["tree"](od), budget=bg, policy=M.LRU)
                assert tuple(st[k] for k in st) == oplan.stats.as_tuple()


def test_shard_values_assemble_bit_exact_oracle():
    wl = synth.make_workload("multi_meson", n_functions=8, nvec=6, lt=7)
    od, _ = D.build_from_workload(wl)
    roots = od.roots()
    leaves = {li: synth.leaf_data(wl, li) for li in range(len(wl.leaves))}
    full = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index])
    world = 3
    pieces = []
    for g in range(world):
        a, b = SH.lt_slices(wl.lt, world)[g]
        vals = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index][a:b])
        pieces.append(np.concatenate([vals[r] for r in roots]))
    got = SH.assemble(pieces, [wl.lt] * len(roots), world)
    assert got.shape == (len(roots), wl.lt)
    for i, r in enumerate(roots):
        assert np.array_equal(got[i], full[r])


def test_assemble_ragged_batch_extents():
    rng = np.random.default_rng(0)
    lts = [5, 3, 8, 4]
    world = 3
    full = [rng.standard_normal(n) + 1j * rng.standard_normal(n) for n in lts]
    pieces = []
    for g in range(world):
        parts = []
        for r, n in enumerate(lts):
            a, b = SH.lt_slices(n, world)[g]
            parts.append(full[r][a:b])
        pieces.append(np.concatenate(parts))
    got = SH.assemble(pieces, lts, world)
    assert got.ndim == 1 and np.array_equal(got, np.concatenate(full))
    with pytest.raises(ValueError):
        SH.assemble([pieces[0][:-1]] + pieces[1:], lts, world)


def test_shard_budget():
    assert SH.shard_budget(0, 64, 16) == 0
    assert SH.shard_budget(1000, 10, 3) == 300
    assert SH.shard_budget(1009, 10, 4) == 400


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gather_rank(rank, ws, port, lts, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    sys.path.insert(0, ROOT)
    from paper_2511_02257_b300 import shard
    full = [np.arange(n) * (1 + 1j) + 100 * r for r, n in enumerate(lts)]
    mine = np.concatenate([full[r][slice(*shard.lt_slices(n, ws)[rank])]
                           for r, n in enumerate(lts)])
    got = shard.gather_correlators(mine, lts, ws)
    out[rank] = bool(np.array_equal(np.asarray(got).reshape(-1), np.concatenate(full)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,lts", [(2, [6, 6, 6]), (3, [5, 9, 4])])
def test_gather_correlators_gloo(ws, lts):
    mp = pytest.importorskip("torch.multiprocessing")
    out = mp.Manager().dict()
    mp.spawn(_gather_rank, args=(ws, _free_port(), lts, out), nprocs=ws, join=True)
    assert dict(out) == {g: True for g in range(ws)}


# ---------------------------------------------------------------- GPU
def _run_shards(wl, precision, world, leaves, budget=0):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    pieces = []
    for g in range(world):
        t0, t1 = SH.lt_slices(wl.lt, world)[g]
        nd, _ = L.build_dag(wl, precision=precision, leaf_data_fn=lambda li: leaves[li],
                            shard=(g, world))
        nd.set_option(L.LQC_OPT_CUDA_GRAPH, 1)
        planned = nd.schedule("tree", "lru", SH.shard_budget(budget, wl.lt, t1 - t0))
        nd.execute(stream)
        pieces.append(np.asarray(nd.read_all_correlators()).reshape(-1))
        assert nd.stats() == planned
        roots = nd.roots()                 # the same ids on every shard
        nd.close()
    return pieces, roots


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol,world", [("fp64", 1e-12, 3), ("tf32x3", 1e-6, 2)])
def test_shards_on_one_gpu_vs_oracle(precision, tol, world):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("multi_meson", n_functions=16, nvec=32, lt=10)
    od, _ = D.build_from_workload(wl)
    leaves = [synth.leaf_data(wl, li) for li in range(len(wl.leaves))]
    ref = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index])
    pieces, roots = _run_shards(wl, precision, world, leaves)
    assert sorted(roots) == sorted(ref)
    got = SH.assemble(pieces, [wl.lt] * len(roots), world)
    errs = [np.linalg.norm(got[i] - ref[r]) / np.linalg.norm(ref[r]) for i, r in enumerate(roots)]
    assert max(errs) < tol, max(errs)


@pytest.mark.gpu
def test_shards_batched_per_part_extents_tf32x3():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    wl = synth.make_workload("batched", seed=3, n_dags=4, nvecs=(16, 32), lts=(4, 7),
                             n_functions=6)
    od, _ = D.build_from_workload(wl)
    leaves = [synth.leaf_data(wl, li) for li in range(len(wl.leaves))]
    ref = C.evaluate(od, lambda u: leaves[od.nodes[u].leaf_index])
    world = 2
    pieces, roots = _run_shards(wl, "tf32x3", world, leaves)
    root_lts = [od.nodes[r].lt for r in roots]
    assert len(set(root_lts)) > 1
    got = SH.assemble(pieces, root_lts, world)
    off = 0
    errs = []
    for r, n in zip(roots, root_lts):
        v = got[off:off + n]
        off += n
        errs.append(np.linalg.norm(v - ref[r]) / np.linalg.norm(ref[r]))
    assert max(errs) < 1e-6, max(errs)
