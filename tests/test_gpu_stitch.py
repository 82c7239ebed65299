"""Tile objects and the stitched field of view (Eq. 1, Sec. 3.1) through the C ABI.

The oracle computes the objects (FP64 inverse DFT) and stitches them pairwise,
literally, from the same spectra the GPU holds, so these tests isolate the
object transform and the stitch.  At the headline size a property replaces the
oracle: windows of one random HR field, each tile's spectrum multiplied by its
own complex factor, stitch back to the field times the first tile's factor.
Bound: rel-L2 1e-5 (FP32 transforms of N <= 1024 points per axis).
"""
import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc
from tests._jobs import Job, rel_l2

pytestmark = pytest.mark.gpu
TOL = 1e-5

O9 = synth.Optics(led_side=9)
SMALL = [
    synth.Workload("st64", sensor=192, tile=64, tiles=3, overlap=16, iters=1, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9100),
    synth.Workload("st128", sensor=256, tile=128, tiles=2, overlap=16, iters=1, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9200),
    # N = 768: the general line FFT (a radix-3 pass) with the row pass's band sums
    synth.Workload("st192", sensor=384, tile=192, tiles=2, overlap=16, iters=1, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9300),
]


@pytest.fixture(scope="module", params=SMALL, ids=[w.name for w in SMALL])
def run(request):
    w = request.param
    j = Job(w)
    p = j.plan(iters=1)
    p.load_tiles(j.stack, j.counts_per_unit)
    p.reconstruct(1, mode="waves")
    yield w, p
    p.close()


def test_objects_match_the_oracle(run):
    w, p = run
    for t in (0, w.n_tiles - 1):
        ref = orc.object_from_spectrum(p.spectrum(t).astype(np.complex128))
        assert rel_l2(p.object(t), ref) < TOL


def test_stitched_fov_matches_the_oracle(run):
    import torch
    w, p = run
    info = p.info
    ov = orc.hr_overlap(w.overlap, w.upsample)
    assert info["hr_overlap"] == ov
    objs = [orc.object_from_spectrum(p.spectrum(t).astype(np.complex128)) for t in range(w.n_tiles)]
    ref = orc.stitch_grid(objs, w.tiles, w.tiles, ov)
    assert (info["fov_h"], info["fov_w"]) == ref.shape
    got = p.stitch()
    assert rel_l2(got, ref) < TOL
    dev = torch.empty((info["fov_h"], info["fov_w"]), dtype=torch.complex64, device="cuda")
    p.stitch(out=dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), got)        # device and host destinations agree exactly


def test_full_size_windows_with_tile_factors_restitch():
    """fov2048_m256: 64 tiles of N = 1024 sharing 64 lines -> a 7744 x 7744 image."""
    import torch
    from paper_2203_02507_b300 import plan_for
    w = synth.WORKLOADS["fov2048_m256"]
    p = plan_for(w, iters=1)
    stack = torch.zeros((w.n_leds, w.sensor, w.sensor), dtype=torch.int16, device="cuda")
    p.load_tiles(stack, 1.0)
    del stack
    n, ov, tiles = p.n, p.info["hr_overlap"], w.tiles
    h, wd = p.info["fov_h"], p.info["fov_w"]
    assert (h, wd) == (n + (tiles - 1) * (n - ov),) * 2
    rng = np.random.default_rng(2024)
    field = (rng.standard_normal((h, wd), dtype=np.float32) + 1j * rng.standard_normal((h, wd), dtype=np.float32)
             + np.complex64(1.0 + 0.5j)).astype(np.complex64)
    alpha = rng.uniform(0.5, 2.0, w.n_tiles) * np.exp(1j * rng.uniform(-np.pi, np.pi, w.n_tiles))
    st = n - ov
    for t in range(w.n_tiles):
        i, j = divmod(t, tiles)
        win = field[i * st:i * st + n, j * st:j * st + n].astype(np.complex128)
        p.set_state(t, spectrum=alpha[t] * orc.fft2c(win))
    got = p.stitch()
    assert rel_l2(got, alpha[0] * field) < TOL
    p.close()
