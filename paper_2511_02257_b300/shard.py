"""Batch-axis sharding of a contraction DAG over ranks.

No contraction ever contracts or mixes the time-slice axis Lt (Sec. II-B:
every tensor carries it as a batch axis), so the DAG splits into
independent slices.  Rank g of G holds the slices [t0, t1) of every tensor
(of every independent part, for DAGs with several batch extents), runs the
same schedule on them under a budget scaled by its share, and the only
exchange is one gather of the root values at the end.  With one batch
extent the scaled problem keeps every decision of the full one: a node's
size is Lt times a per-slice size, so the schedulers' gains and the plan's
comparisons against the budget B are those of the full DAG multiplied by
lt_g / Lt when the shard's budget is (B // Lt) * lt_g.

This module holds the host logic: the slice split, the shard budget and the
assembly of the gathered correlators; ``lqc.build_dag(..., shard=(g, G))``
builds a shard.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def lt_slices(lt: int, world: int) -> List[Tuple[int, int]]:
    """[t0, t1) of each rank: contiguous, the first lt % world ranks one
    slice longer.  Every rank needs at least one slice."""
    if world < 1 or lt < world:
        raise ValueError("cannot split %d time slices over %d ranks" % (lt, world))
    base, extra = divmod(lt, world)
    out, t = [], 0
    for g in range(world):
        n = base + (1 if g < extra else 0)
        out.append((t, t + n))
        t += n
    return out


def shard_budget(budget: int, lt: int, lt_g: int) -> int:
    """Device budget of a rank holding lt_g of lt slices (0 = unlimited).
    With one batch extent this keeps the full plan's eviction decisions: all
    sizes are lt times an integer per-slice size."""
    if budget <= 0:
        return 0
    return (budget // lt) * lt_g


def assemble(pieces: Sequence[np.ndarray], root_lts: Sequence[int], world: int) -> np.ndarray:
    """Full correlators from the ranks' pieces.  pieces[g] = rank g's
    correlators of every root in ascending root id, root r contributing its
    slices lt_slices(root_lts[r], world)[g]; returns the roots' full
    correlators concatenated in the same order (a [roots][lt] array when all
    roots share one batch extent)."""
    per_rank = [lt_slices(int(n), world) for n in root_lts]
    out = np.empty(int(sum(root_lts)), dtype=np.complex128)
    off_out = 0
    off_in = [0] * world
    for r, n in enumerate(root_lts):
        for g in range(world):
            t0, t1 = per_rank[r][g]
            m = t1 - t0
            out[off_out + t0:off_out + t1] = pieces[g][off_in[g]:off_in[g] + m]
            off_in[g] += m
        off_out += int(n)
    for g in range(world):
        if off_in[g] != np.asarray(pieces[g]).size:
            raise ValueError("rank %d sent %d values, expected %d"
                             % (g, np.asarray(pieces[g]).size, off_in[g]))
    if len(set(int(n) for n in root_lts)) == 1 and len(root_lts):
        return out.reshape(len(root_lts), int(root_lts[0]))
    return out


def gather_correlators(local: np.ndarray, root_lts: Sequence[int], world: int,
                       device: str = "cpu") -> np.ndarray:
    """All-gather of every rank's correlator piece over the default process
    group (the one exchange of a sharded execution), then `assemble`.  The
    pieces travel as float64 pairs padded to the longest piece; `device` is
    "cuda" under NCCL, "cpu" under gloo."""
    import torch
    import torch.distributed as dist
    flat = np.ascontiguousarray(local, dtype=np.complex128).reshape(-1)
    sizes = []
    for g in range(world):
        n = 0
        for lt in root_lts:
            t0, t1 = lt_slices(int(lt), world)[g]
            n += t1 - t0
        sizes.append(n)
    pad = max(sizes)
    buf = torch.zeros(2 * pad, dtype=torch.float64)
    buf[:2 * flat.size] = torch.from_numpy(flat.view(np.float64).copy())
    buf = buf.to(device)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf)
    pieces = [outs[g].cpu().numpy()[:2 * sizes[g]].view(np.complex128) for g in range(world)]
    return assemble(pieces, root_lts, world)
