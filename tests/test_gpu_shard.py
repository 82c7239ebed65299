"""Tile sharding on the GPU (Sec. 5: sub-regions sent to different GPUs), with the
ranks emulated one after another on this one GPU (they exchange nothing while
they reconstruct): tile-subset plans reconstruct their tiles exactly as the
whole-grid plan does, and the gathered states written into a whole-grid plan
stitch (Eq. 1) to the same field of view bit for bit."""
import numpy as np
import pytest

import synth
from paper_2203_02507_b300 import shard
from tests._jobs import Job

pytestmark = pytest.mark.gpu

W = synth.Workload("shard128", sensor=512, tile=128, tiles=4, overlap=16, iters=2, epry=True,
                   optics=synth.Optics(led_side=9), defocus_um=(-20.0, 20.0), seed_offset=7800)


@pytest.fixture(scope="module")
def job():
    return Job(W)


@pytest.mark.parametrize("ranks", [2, 3])
def test_subset_plans_reassemble_the_whole_job(job, ranks):
    full = job.plan()
    full.load_tiles(job.stack, job.counts_per_unit)
    full.reconstruct(W.iters, mode="waves", graph=True)
    ref_s = [full.spectrum(t) for t in range(W.n_tiles)]
    ref_p = [full.pupil(t) for t in range(W.n_tiles)]
    ref_fov = full.stitch()
    full.close()

    ranges = shard.job_ranges([(W.n_tiles, W.tile, W.n_leds, W.iters)], ranks)
    by_rank = [(rr[0][1], rr[0][2]) if rr else (0, 0) for rr in ranges]
    specs = np.zeros((W.n_tiles, W.hr, W.hr), np.complex64)
    pups = np.zeros((W.n_tiles, W.tile, W.tile), np.complex64)
    from paper_2203_02507_b300 import plan_for
    for first, count in by_rank:             # rank r's work: a plan of its tiles only
        if count == 0:
            continue
        p = plan_for(W, defocus_um=job.defocus, iters=W.iters, tile_first=first, tile_count=count)
        p.load_tiles(job.stack, job.counts_per_unit)
        p.reconstruct(W.iters, mode="waves", graph=True)
        for i in range(count):
            specs[first + i] = p.spectrum(i)
            pups[first + i] = p.pupil(i)
        with pytest.raises(Exception):
            p.stitch()                       # a subset cannot stitch the field of view
        p.close()
    for t in range(W.n_tiles):
        assert np.array_equal(specs[t], ref_s[t]) and np.array_equal(pups[t], ref_p[t]), t

    # the gathering rank: a whole-grid plan takes every tile's state and stitches
    q = job.plan()
    q.load_tiles(job.stack, job.counts_per_unit)
    for t in range(W.n_tiles):
        q.set_state(t, specs[t], pups[t])
    assert np.array_equal(q.stitch(), ref_fov)
    q.close()
