"""Sharding over several GPUs: columns of the block (Section 3.1) and
independent jobs.

Column slabs.

The paper gives each process one column of the block Y: column j of
S_i = X^T A~^i Y depends only on Y[:, j], so the processes never exchange
data while they iterate, and the column sequences are gathered once before
the sigma-basis.  Here each rank (one per GPU) takes a contiguous slab of Y's
columns, computes its L x m x w slab of the sequence with
wr_sequence_slab_device, and one all-gather assembles the full L x m x n
sequence in column order on every rank.  The host logic (slab bounds, padding
of uneven slabs to a common width for the collective, reassembly) is plain
torch.distributed and runs the same on gloo (CPU) and NCCL (GPU).

Independent jobs.  Batched work (matrices x primes, rank over Q as the
maximum over primes, Section 2.5) needs no exchange while it runs: jobs are
dealt to ranks, largest first, so that the ranks' summed costs stay close,
each rank runs its share (wr_rank_batch on its GPU), and one gather brings
the ranks of every job back in job order.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch
import torch.distributed as dist


def column_slab(n: int, rank: int, world: int) -> Tuple[int, int]:
    """(first column, width) of rank's slab: n columns in world contiguous
    slabs whose widths differ by at most one, the wider ones first."""
    if not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n, world)
    w = base + (1 if rank < extra else 0)
    c0 = rank * base + min(rank, extra)
    return c0, w


def gather_columns(slab: torch.Tensor, n: int, world: int, group=None) -> torch.Tensor:
    """All-gather the L x m x w slabs of every rank into L x m x n (column
    order = rank order).  Slabs are padded to the widest width for the
    collective and cut back afterwards."""
    L, m, _ = slab.shape
    wmax = column_slab(n, 0, world)[1]
    pad = torch.zeros((L, m, wmax), dtype=slab.dtype, device=slab.device)
    pad[:, :, : slab.shape[2]] = slab
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    cols = [parts[r][:, :, : column_slab(n, r, world)[1]] for r in range(world)]
    return torch.cat(cols, dim=2).contiguous()


def sharded_sequence(compute_slab: Callable[[int, int], torch.Tensor], n: int, rank: int, world: int,
                     group=None) -> torch.Tensor:
    """The full sequence on every rank: this rank's slab from compute_slab(c0, w)
    (an L x m x w tensor), then one all-gather.  A rank whose slab is empty
    (world > n) contributes nothing and still takes part in the collective."""
    c0, w = column_slab(n, rank, world)
    slab = compute_slab(c0, w) if w > 0 else None
    if slab is None:
        raise ValueError("every rank needs at least one column (world <= n)")
    return gather_columns(slab, n, world, group)


def gpu_slab(ctx: int, mat: int, params, L: int, device: Optional[torch.device] = None):
    """compute_slab for the GPU path: wr_sequence_slab_device into a device tensor."""
    from . import wr

    def run(c0: int, w: int) -> torch.Tensor:
        out = torch.empty((L, params.m, w), dtype=torch.int32, device=device or "cuda")
        wr.wr_sequence_slab_device(ctx, mat, params, c0, w, out, L)
        return out

    return run


def deal_jobs(costs, world: int):
    """Job indices per rank: jobs taken largest cost first (ties by index),
    each to the rank with the least summed cost so far (ties by rank).  Every
    job lands on exactly one rank; a rank's list is in increasing job order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    share = [[] for _ in range(world)]
    for j in sorted(range(len(costs)), key=lambda j: (-float(costs[j]), j)):
        r = min(range(world), key=lambda r: (load[r], r))
        share[r].append(j)
        load[r] += float(costs[j])
    return [sorted(s) for s in share]


def gather_job_results(mine, results, njobs: int, world: int, group=None) -> torch.Tensor:
    """All-gather the int64 results of every rank's jobs (mine: this rank's
    job indices, results: one value each) into one tensor in job order."""
    cnt = torch.tensor([len(mine)], dtype=torch.int64)
    parts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(parts, cnt, group=group)
    counts = [int(c.item()) for c in parts]
    width = max(counts + [1])
    buf = torch.full((2, width), -1, dtype=torch.int64)
    if mine:
        buf[0, : len(mine)] = torch.tensor(list(mine), dtype=torch.int64)
        buf[1, : len(mine)] = torch.tensor(list(results), dtype=torch.int64)
    bufs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(bufs, buf, group=group)
    out = torch.full((njobs,), -1, dtype=torch.int64)
    for r in range(world):
        k = counts[r]
        out[bufs[r][0, :k]] = bufs[r][1, :k]
    if (out < 0).any():
        raise RuntimeError("a job's result is missing after the gather")
    return out
