"""Pins of the oracle's geometry, LED order, pupil support and waves (Sec. 2.2, 3.1, 3.2)."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc

LAM, NA, DX = 0.532, 0.10, 1.625


def test_lround_halfway_away_from_zero():
    x = [0.5, -0.5, 1.5, -1.5, 2.5, -2.5, 0.49999999999999994, 2.4999999, -0.2, 0.0]
    assert list(orc.lround(x)) == [1, -1, 2, -2, 3, -3, 0, 2, 0, 0]


def test_worked_geometry_examples(golden_dir):
    gold = json.load(open(os.path.join(golden_dir, "geometry_worked.json")))
    df = 1.0 / (256 * DX)
    for case in gold["cases"]:
        s = orc.led_shifts(np.array([case["tile_centre_um"]]), np.array([case["led_xy_um"]]),
                           90000.0, LAM, df)
        assert list(s[0, 0]) == case["shift_yx"], case["_derivation"]


def test_stitch_example_span(golden_dir):
    st = json.load(open(os.path.join(golden_dir, "geometry_worked.json")))["stitch_span"]
    o = orc.tile_origins(st["m"], st["span"], st["m"], st["overlap"], 1, 2)
    assert o[0, 1] == 0 and o[1, 1] + st["m"] == st["span"]


@pytest.mark.parametrize("s,m,ov,n", [(2048, 256, 16, 8), (1536, 192, 16, 8), (5120, 128, 0, 40),
                                      (1024, 128, 16, 8), (64, 64, 0, 1)])
def test_tile_grid_properties(s, m, ov, n):
    o = orc.tile_origins(s, s, m, ov, n, n)
    xs = np.unique(o[:, 1])
    assert len(xs) == n and xs[0] >= 0 and xs[-1] + m <= s
    assert np.all(np.diff(xs) == m - ov)                 # neighbours overlap by exactly ov
    left, right = xs[0], s - (xs[-1] + m)
    assert 0 <= right - left <= 1                        # centred
    c = orc.tile_centres_um(o, m, s, s, DX)
    assert abs(c[:, 0].sum()) < 1e-6 and abs(c[:, 1].sum()) < 1e-6 or left != right


def test_centre_out_order_15x15():
    leds = synth.led_grid(15, 4000.0)
    order = orc.led_order(leds)
    assert sorted(order) == list(range(225))
    assert order[0] == 112                               # the centre LED
    assert list(order[1:5]) == [97, 111, 113, 127]       # distance 1, by index
    assert list(order[5:9]) == [96, 98, 126, 128]        # distance sqrt(2), by index
    d2 = [((i % 15) - 7) ** 2 + ((i // 15) - 7) ** 2 for i in order]
    for a, b, ia, ib in zip(d2, d2[1:], order, order[1:]):
        assert a < b or (a == b and ia < ib)
    assert list(orc.led_order(leds, "raster")) == list(range(225))


@pytest.mark.parametrize("m", [64, 128, 192, 256])
def test_pupil_support_is_the_integer_disc(m):
    """FP64 |f| <= NA/lambda agrees with an exact integer count of lattice points in the disc."""
    df = 1.0 / (m * DX)
    sup = orc.pupil_support(m, df, LAM, NA)
    r = NA / LAM / df
    r2 = r * r
    cnt = 0
    for ky in range(-m // 2, m // 2):
        for kx in range(-m // 2, m // 2):
            if ky * ky + kx * kx <= r2:
                cnt += 1
                assert sup[ky + m // 2, kx + m // 2]
    assert sup.sum() == cnt
    assert np.array_equal(sup[1:, 1:], sup[1:, 1:][::-1, ::-1])   # point symmetric about the centre
    p = orc.pupil(m, df, LAM, NA, 15.0)
    assert np.all(p[~sup] == 0) and np.allclose(np.abs(p[sup]), 1.0)
    assert abs(p[m // 2, m // 2] - 1.0) < 1e-15                    # no phase at f = 0


def test_pupil_defocus_phase_closed_form():
    m = 64
    df = 1.0 / (m * DX)
    z = 10.0
    p = orc.pupil(m, df, LAM, NA, z)
    k = (3, -4)
    f = math.hypot(k[0] * df, k[1] * df)
    want = np.exp(1j * 2 * math.pi * z * (math.sqrt(1 / LAM ** 2 - f ** 2) - 1 / LAM))
    assert abs(p[k[0] + m // 2, k[1] + m // 2] - want) < 1e-12


def _brute_waves(n, support, shifts, seq):
    fps = [set(orc.footprint(n, support, shifts[int(l)]).tolist()) for l in seq]
    w = []
    for j in range(len(seq)):
        deps = [w[i] for i in range(j) if fps[i] & fps[j]]
        w.append(1 + max(deps) if deps else 0)
    return np.array(w)


@pytest.mark.parametrize("side,iters", [(3, 2), (5, 2)])
def test_waves_match_pairwise_definition(side, iters):
    m = 16
    n = 4 * m
    df = 1.0 / (m * DX)
    leds = synth.led_grid(side, 6000.0)
    g = orc.geometry(m, m, m, 0, 1, 1, 4, LAM, NA * 2.5, DX, leds, 90000.0, [0.0])
    seq = orc.sequence(g.order, iters)
    w = orc.waves(n, g.support, g.shifts[0], seq)
    assert np.array_equal(w, _brute_waves(n, g.support, g.shifts[0], seq))
    assert w.max() < len(seq) and w.max() >= iters - 1


def test_waves_are_valid_on_config_geometry():
    """No two members of a wave share a pixel; every earlier overlapping item is in an earlier wave."""
    m = 64
    leds = synth.led_grid(15, 4000.0)
    g = orc.geometry(64, 64, m, 0, 1, 1, 4, LAM, NA, DX, leds, 90000.0, [0.0])
    seq = orc.sequence(g.order, 2)
    w = orc.waves(g.n, g.support, g.shifts[0], seq)
    owner = {}
    for j, l in enumerate(seq):
        for p in orc.footprint(g.n, g.support, g.shifts[0][int(l)]).tolist():
            key = (int(w[j]), p)
            assert key not in owner
            owner[key] = j
    last = np.full(g.n * g.n, -1)
    for j, l in enumerate(seq):
        fp = orc.footprint(g.n, g.support, g.shifts[0][int(l)])
        assert last[fp].max() < w[j]
        last[fp] = w[j]
