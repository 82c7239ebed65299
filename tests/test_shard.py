"""Tile sharding over GPUs (Sec. 5: sub-regions sent to different GPUs) and the
final gather (host logic, on CPU): the cost-balanced partition, tile-subset plans
whose geometry is the whole grid's, and a two-rank gloo gather of tile states
reconstructed rank by rank (by the FP64 oracle here; on GPUs by the library)."""
import os
import socket

import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc

fpm = pytest.importorskip("paper_2203_02507_b300._fpm")
from paper_2203_02507_b300 import shard  # noqa: E402


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(3)
    for ranks in (1, 2, 3, 5, 8):
        costs = rng.integers(1, 50, size=137).astype(float)
        parts = shard.partition(costs, ranks)
        assert parts[0][0] == 0 and parts[-1][1] == len(costs)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(ranks - 1))
        share = costs.sum() / ranks
        for a, b in parts:
            assert abs(costs[a:b].sum() - share) <= costs.max() + 1e-9


def test_partition_degenerate_cases():
    assert shard.partition([], 3) == [(0, 0), (0, 0), (0, 0)]
    assert shard.partition([7.0], 2) in ([(0, 1), (1, 1)], [(0, 0), (0, 1)])
    assert shard.partition([1.0] * 64, 8) == [(8 * r, 8 * r + 8) for r in range(8)]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


@pytest.mark.parametrize("ranks", [2, 4, 8])
def test_uneven_batch_shards_by_tile_cost(ranks):
    """The three-job uneven batch (tiles of 128, 192 and 256 under 9x9, 13x13 and
    15x15 LEDs, 15 loops): every tile of every job on exactly one rank, each rank
    within one tile's cost (m^2 L iters) of an equal share."""
    jobs = [(64, 128, 81, 15), (64, 192, 169, 15), (64, 256, 225, 15)]
    ranges = shard.job_ranges(jobs, ranks)
    seen = [np.zeros(j[0], int) for j in jobs]
    for rr in ranges:
        for j, first, count in rr:
            seen[j][first:first + count] += 1
    assert all((s == 1).all() for s in seen)
    total = sum(shard.tile_cost(*j[1:]) * j[0] for j in jobs)
    biggest = max(shard.tile_cost(*j[1:]) for j in jobs)
    for rr in ranges:
        assert abs(shard.rank_cost(jobs, rr) - total / ranks) <= biggest


def test_subset_plan_has_the_whole_grids_geometry():
    w = synth.WORKLOADS["fov2048_m256"]
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    full = fpm.plan_for(w, defocus_um=dz, iters=2)
    s = full.schedule()
    for first, count in [(0, 9), (9, 31), (40, 24), (63, 1)]:
        sub = fpm.plan_for(w, defocus_um=dz, iters=2, tile_first=first, tile_count=count)
        t = sub.schedule()
        assert sub.n_tiles == count and sub.tile_first == first
        for k in ("shifts", "waves", "origins"):
            assert np.array_equal(t[k], s[k][first:first + count]), k
        assert np.array_equal(t["order"], s["order"])
        for i in (0, count - 1):
            assert np.array_equal(sub.initial_pupil(i), full.initial_pupil(first + i))
        sub.close()
    with pytest.raises(fpm.FpmError):
        fpm.plan_for(w, defocus_um=dz, iters=1, tile_first=60, tile_count=5)
    with pytest.raises(fpm.FpmError):
        fpm.plan_for(w, defocus_um=dz, iters=1, tile_first=3, tile_count=0)
    full.close()


SMALL = synth.Workload("shard64", sensor=208, tile=64, tiles=3, overlap=16, iters=1, epry=True,
                       optics=synth.Optics(led_side=5), defocus_um=(-10.0, 10.0), seed_offset=7700)


def _tile_state(t, images, g):
    return orc.reconstruct_tile(images[t], g.shifts[t], g.order, g.support, g.pupils[t], g.n, SMALL.iters, True)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = SMALL
    g, images = _job()
    job = [(w.n_tiles, w.tile, w.n_leds, w.iters)]
    ranges = shard.job_ranges(job, world)
    by_rank = [(rr[0][1], rr[0][2]) if rr else (0, 0) for rr in ranges]
    first, count = by_rank[rank]
    specs = np.zeros((count, g.n, g.n), np.complex64)
    pups = np.zeros((count, g.m, g.m), np.complex64)
    for i in range(count):               # this rank's tiles (a GPU rank runs a tile-subset plan here)
        s, p = _tile_state(first + i, images, g)
        specs[i], pups[i] = s, p
    all_specs = shard.gather_tiles(specs, first, w.n_tiles, by_rank, rank, dist)
    all_pups = shard.gather_tiles(pups, first, w.n_tiles, by_rank, rank, dist)
    if rank == 0:
        out["specs"], out["pups"], out["ranges"] = all_specs, all_pups, by_rank
    dist.barrier()
    dist.destroy_process_group()


def _job():
    w = SMALL
    o = w.optics
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    g = orc.geometry(w.sensor, w.sensor, w.tile, w.overlap, w.tiles, w.tiles, w.upsample, o.wavelength_um, o.na,
                     o.pixel_um, synth.led_grid(o.led_side, o.led_pitch_um), o.led_height_um, dz)
    images = np.stack([orc.forward_images(orc.fft2c(synth.hr_object(w.hr, t, w.seed_offset)), g.pupils[t],
                                          g.shifts[t], w.tile) for t in range(w.n_tiles)])
    return g, images


def test_two_rank_gather_reassembles_every_tile():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    g, images = _job()
    assert out["ranges"][0][1] > 0 and out["ranges"][1][1] > 0      # both ranks had work
    for t in range(SMALL.n_tiles):
        s, p = _tile_state(t, images, g)
        assert np.array_equal(out["specs"][t], s.astype(np.complex64))
        assert np.array_equal(out["pups"][t], p.astype(np.complex64))
