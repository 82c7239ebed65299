"""Update-routine and EPRY variants through the C ABI (Sec. 3.2, Fig. 6): the raster
update routine, and strict-sequential EPRY (every update sees the pupil corrected
by all earlier ones; one LED per tile per wave), each against the oracle's same
mode after one loop.  Bound: max(stated bound, 4 x the float32 floor of the
oracle's steps in complex64), as for the default mode."""
import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc
from tests import _fp32
from tests._jobs import Job, rel_l2

pytestmark = pytest.mark.gpu
SPEC_TOL, PUPIL_TOL, FLOOR_FACTOR = 1e-5, 1e-4, 4.0

O9 = synth.Optics(led_side=9)
W = synth.Workload("var64", sensor=160, tile=64, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9500)
_JOB = {}


def job():
    if "j" not in _JOB:
        _JOB["j"] = Job(W)
    return _JOB["j"]


def _check_against_oracle(p, j, g, mode):
    for t in range(W.n_tiles):
        imgs = j.tile_images(t)
        spec, pup = orc.reconstruct_tile(imgs, g.shifts[t], g.order, g.support, g.pupils[t], g.n, 1, True, mode=mode)
        fs, fp = _fp32.floor(imgs, g.shifts[t], g.order, g.support, g.pupils[t], g.n, 1, True, spec, pup, mode=mode)
        assert rel_l2(p.spectrum(t), spec) < max(SPEC_TOL, FLOOR_FACTOR * fs), (t, fs)
        assert rel_l2(p.pupil(t), pup) < max(PUPIL_TOL, FLOOR_FACTOR * fp), (t, fp)


def test_sequential_epry_matches_the_oracle():
    from paper_2203_02507_b300 import plan_for
    j = job()
    p = plan_for(W, defocus_um=j.defocus, iters=1, sequential=True)
    p.load_tiles(j.stack, j.counts_per_unit)
    p.reconstruct(1, mode="waves")
    _check_against_oracle(p, j, j.g, "sequential")
    p.close()


def test_sequential_epry_is_the_same_in_every_execution_mode():
    from paper_2203_02507_b300 import plan_for
    j = job()
    outs = []
    for mode, graph in [("waves", False), ("waves", True), ("plain", False), ("persistent", True)]:
        p = plan_for(W, defocus_um=j.defocus, iters=2, sequential=True)
        p.load_tiles(j.stack, j.counts_per_unit)
        p.reconstruct(2, mode=mode, graph=graph)
        outs.append([p.spectrum(t) for t in range(W.n_tiles)] + [p.pupil(t) for t in range(W.n_tiles)])
        p.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)


def test_raster_routine_matches_the_oracle():
    from paper_2203_02507_b300 import plan_for
    j = job()
    o = W.optics
    g = orc.geometry(W.sensor, W.sensor, W.tile, W.overlap, W.tiles, W.tiles, W.upsample, o.wavelength_um, o.na,
                     o.pixel_um, j.leds, o.led_height_um, j.defocus, routine="raster")
    p = plan_for(W, defocus_um=j.defocus, iters=1, order="raster")
    assert list(p.schedule()["order"]) == list(g.order) == list(range(W.n_leds))
    p.load_tiles(j.stack, j.counts_per_unit)
    p.reconstruct(1, mode="waves")
    _check_against_oracle(p, j, g, "waves")
    p.close()


W256 = synth.Workload("var256", sensor=512, tile=256, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                      defocus_um=(-20.0, 20.0), seed_offset=9600)


@pytest.mark.parametrize("w", [W, W256], ids=["m64", "m256"])
def test_unmasked_epry_matches_the_oracle(w):
    """Non-masked EPRY (FPM_EPRY_UNMASKED): corrections, normalisers and wave
    footprints over the whole box, against the oracle run with an all-true
    support, after one loop."""
    from paper_2203_02507_b300 import plan_for
    j = job() if w is W else Job(w)
    box = np.ones((w.tile, w.tile), bool)
    p = plan_for(w, defocus_um=j.defocus, iters=1, unmasked=True)
    p.load_tiles(j.stack, j.counts_per_unit)
    p.reconstruct(1, mode="waves")
    for t in range(w.n_tiles):
        imgs = j.tile_images(t)
        g = j.g
        spec, pup = orc.reconstruct_tile(imgs, g.shifts[t], g.order, box, g.pupils[t], g.n, 1, True)
        fs, fp = _fp32.floor(imgs, g.shifts[t], g.order, box, g.pupils[t], g.n, 1, True, spec, pup)
        assert rel_l2(p.spectrum(t), spec) < max(SPEC_TOL, FLOOR_FACTOR * fs), (t, fs)
        assert rel_l2(p.pupil(t), pup) < max(PUPIL_TOL, FLOOR_FACTOR * fp), (t, fp)
        assert np.abs(p.pupil(t)[~g.support]).max() > 0          # the pupil grew outside the disc
    p.close()


def test_unmasked_epry_is_the_same_in_every_execution_mode():
    from paper_2203_02507_b300 import plan_for
    j = job()
    outs = []
    for mode, graph in [("waves", False), ("waves", True), ("plain", False), ("persistent", True)]:
        p = plan_for(W, defocus_um=j.defocus, iters=2, unmasked=True)
        p.load_tiles(j.stack, j.counts_per_unit)
        p.reconstruct(2, mode=mode, graph=graph)
        outs.append([p.spectrum(t) for t in range(W.n_tiles)] + [p.pupil(t) for t in range(W.n_tiles)])
        p.close()
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
