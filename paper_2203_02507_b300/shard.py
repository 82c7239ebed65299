"""Tile sharding across GPUs (Sec. 5: different sub-regions' data sent to
different GPUs) with one final gather for stitching (Sec. 3.1, Eq. 1).

Tiles are independent (Sec. 3.1), so the reconstruction needs no exchange: each
rank reconstructs a contiguous range of every job's tiles with a plan of that
tile subset (``Plan(..., tile_first, tile_count)``: the tiles keep the geometry
they have in the whole grid), and at the end the ranks send their tiles'
spectra and pupils to one rank, which writes them into a plan of the whole grid
(``set_state``) and stitches.

The partition balances the cost of a tile's reconstruction, taken as
m^2 * L * iters (LR pixels times LED updates; the per-update work of the FFT
path grows with m^2 log m, which the m^2 proxy under-weights by at most
log2(256)/log2(64) = 4/3 between the tile sides in use).  Tiles are laid out
job after job, tile after tile, and cut at equal shares of the prefix sum of
their costs, so every rank gets one contiguous range per job and the ranks'
costs differ by at most one tile's cost.

This module holds host logic only; the reconstruction itself runs in the
library's kernels on each rank's GPU.
"""
from __future__ import annotations

import numpy as np


def tile_cost(m: int, n_leds: int, iters: int) -> int:
    """Reconstruction cost of one tile: m^2 * L * iters."""
    return int(m) * int(m) * int(n_leds) * int(iters)


def partition(costs, ranks: int):
    """Cut the list of per-tile costs into `ranks` contiguous ranges of nearly
    equal total cost.  Returns [(start, stop), ...], one per rank, covering
    0..len(costs) in order (a range may be empty when there are fewer tiles
    than ranks).  Rank r takes the tiles whose cost midpoint falls in
    [r C / ranks, (r + 1) C / ranks), C the total, so every rank's share is
    within one tile's cost of C / ranks."""
    costs = np.asarray(costs, dtype=np.float64)
    if ranks < 1:
        raise ValueError("ranks must be >= 1")
    if costs.ndim != 1 or (costs < 0).any():
        raise ValueError("costs must be a list of non-negative numbers")
    total = float(costs.sum())
    if len(costs) == 0 or total == 0.0:
        cuts = np.linspace(0, len(costs), ranks + 1).round().astype(int)
    else:
        mid = np.cumsum(costs) - 0.5 * costs            # cost midpoint of each tile
        owner = np.minimum((mid * ranks / total).astype(np.int64), ranks - 1)
        cuts = np.searchsorted(owner, np.arange(ranks + 1), side="left")
        cuts[-1] = len(costs)
    return [(int(cuts[r]), int(cuts[r + 1])) for r in range(ranks)]


def job_ranges(jobs, ranks: int):
    """Shard several jobs' tiles over `ranks` ranks.

    jobs: [(n_tiles, m, n_leds, iters), ...].  Returns, per rank, a list of
    (job index, tile_first, tile_count) with tile_count > 0: the contiguous
    range of each job's tiles that rank reconstructs."""
    costs, owner_job, owner_tile = [], [], []
    for j, (n_tiles, m, n_leds, iters) in enumerate(jobs):
        c = tile_cost(m, n_leds, iters)
        for t in range(int(n_tiles)):
            costs.append(c)
            owner_job.append(j)
            owner_tile.append(t)
    out = [[] for _ in range(ranks)]
    for r, (a, b) in enumerate(partition(costs, ranks)):
        k = a
        while k < b:
            j = owner_job[k]
            e = k
            while e < b and owner_job[e] == j:
                e += 1
            out[r].append((j, owner_tile[k], e - k))
            k = e
    return out


def rank_cost(jobs, ranges) -> float:
    """Total m^2 * L * iters of one rank's ranges."""
    return float(sum(tile_cost(*jobs[j][1:]) * cnt for j, _, cnt in ranges))


def gather_tiles(local, tile_first: int, n_tiles_total: int, ranges_by_rank, rank: int, dist, dst: int = 0):
    """Collect every rank's tile arrays on rank `dst` with point-to-point sends.

    local: host array [count, ...] (count = this rank's tiles of the job, in
    order from tile_first).  ranges_by_rank: [(tile_first, count)] of every
    rank for this job.  On `dst` returns the [n_tiles_total, ...] array of the
    whole job; elsewhere returns None.  Sizes follow from the partition, so no
    metadata is exchanged; any backend with send/recv (gloo, NCCL) serves."""
    import torch
    local = np.ascontiguousarray(local)
    # complex values travel as their float32 / float64 parts (every backend has those)
    real_dt = np.float32 if local.dtype in (np.complex64, np.float32) else np.float64
    wire = local.view(real_dt)
    if rank == dst:
        out = np.empty((n_tiles_total,) + local.shape[1:], dtype=local.dtype)
        for r, (first, count) in enumerate(ranges_by_rank):
            if count == 0:
                continue
            if r == rank:
                out[first:first + count] = local
                continue
            buf = torch.empty((count,) + wire.shape[1:], dtype=torch.float32 if real_dt is np.float32 else torch.float64)
            dist.recv(buf, src=r)
            out[first:first + count] = buf.numpy().view(local.dtype)
        return out
    if local.shape[0]:
        dist.send(torch.from_numpy(wire), dst=dst)
    return None
