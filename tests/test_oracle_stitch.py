"""Pins of the oracle's stitching (Eq. 1, Sec. 3.1), independent of its own code:
the paper's worked sizes, exact reassembly of windows cut from one image, removal
of an arbitrary complex factor per tile, and the exact cut line."""
import json
import os

import numpy as np
import pytest

from oracle import fpm_oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "stitch_worked.json")


def _field(h, w, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((h, w)) + 1j * rng.standard_normal((h, w)) + (2.0 + 1.0j)


def _windows(img, n, ov, ty, tx):
    st = n - ov
    return [img[i * st:i * st + n, j * st:j * st + n].copy() for i in range(ty) for j in range(tx)]


def test_paper_worked_sizes():
    g = json.load(open(GOLDEN))
    a = np.ones(g["image"], complex)
    p1 = orc.stitch_pair(a, a, g["overlap"], 0)
    assert list(p1.shape) == g["part1_output"]
    p2 = orc.stitch_pair(p1, p1, g["overlap"], 1)
    assert list(p2.shape) == g["part2_output_of_two_part1_outputs"]
    assert g["overlap"] == round(0.1 * g["image"][0])


@pytest.mark.parametrize("ty,tx,n,ov", [(2, 2, 32, 8), (3, 4, 24, 6), (1, 3, 16, 5), (3, 1, 20, 7), (2, 3, 16, 0)])
def test_windows_of_one_image_reassemble_exactly(ty, tx, n, ov):
    h, w = n + (ty - 1) * (n - ov), n + (tx - 1) * (n - ov)
    img = _field(h, w, 7)
    out = orc.stitch_grid(_windows(img, n, ov, ty, tx), ty, tx, ov)
    assert out.shape == (h, w)
    # shared bands hold equal data, so every weight is 1 up to the rounding of a complex division
    np.testing.assert_allclose(out, img, rtol=1e-13, atol=0)


def test_a_complex_factor_per_tile_is_removed():
    ty, tx, n, ov = 3, 3, 24, 8
    h, w = n + (ty - 1) * (n - ov), n + (tx - 1) * (n - ov)
    img = _field(h, w, 11)
    rng = np.random.default_rng(12)
    alpha = rng.uniform(0.5, 2.0, ty * tx) * np.exp(1j * rng.uniform(-np.pi, np.pi, ty * tx))
    tiles = [a * t for a, t in zip(alpha, _windows(img, n, ov, ty, tx))]
    out = orc.stitch_grid(tiles, ty, tx, ov)
    np.testing.assert_allclose(out, alpha[0] * img, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("axis,ov", [(0, 6), (1, 6), (0, 7), (1, 7)])
def test_cut_line_and_weight_direction(axis, ov):
    """overlap/2 is read as overlap // 2 (an odd overlap keeps the extra line from f2)."""
    n, h = 20, ov // 2
    f1 = np.full((n, n), 3.0 + 0j)
    f2 = np.full((n, n), 7.0 + 0j)
    first = (slice(0, h), slice(None)) if axis == 0 else (slice(None), slice(0, h))
    second = (slice(h, ov), slice(None)) if axis == 0 else (slice(None), slice(h, ov))
    late = (3.0 * ov - h) / (ov - h)          # band = 1 then `late`: its mean is exactly 3 like f1's
    f2[first], f2[second] = 1.0, late
    out = orc.stitch_pair(f1, f2, ov, axis)
    line = np.moveaxis(out, axis, 0)[:, 0]
    cut = n - h
    assert line.shape[0] == 2 * n - ov
    assert np.all(line[:cut] == 3.0)         # f1 up to r - overlap // 2
    assert np.all(line[cut:n] == late)       # then f2 from its line overlap // 2 on
    assert np.all(line[n:] == 7.0)
    f2s = 2j * f2                            # f2 scaled: mu1 / mu2 = 1 / 2j rescales it back
    np.testing.assert_allclose(orc.stitch_pair(f1, f2s, ov, axis), out, rtol=1e-15)


def test_hr_overlap_is_lr_overlap_times_upsampling():
    assert orc.hr_overlap(16, 4) == 64
