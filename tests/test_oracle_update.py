"""Pins of the oracle's per-LED update (Sec. 2.1 alternating projection; EPRY formulas)."""
import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc

LAM, NA, DX = 0.532, 0.10, 1.625


def _small_job(m=32, side=7, z=5.0, seed=0):
    """A small noiseless FP64 job: ground-truth spectrum, pupil, shifts, images."""
    n = 4 * m
    leds = synth.led_grid(side, 4000.0)
    g = orc.geometry(m, m, m, 0, 1, 1, 4, LAM, NA, DX, leds, 90000.0, [z])
    obj = synth.hr_object(n, 0, seed_offset=seed)
    spec = orc.fft2c(obj)
    imgs = orc.forward_images(spec, g.pupils[0], g.shifts[0], m)
    return g, spec, imgs


@pytest.mark.parametrize("epry", [False, True])
def test_fixed_point_ground_truth_is_unchanged(epry):
    """Ground-truth object and pupil with noiseless FP64 data change by < 1e-12 (relative)."""
    g, spec, imgs = _small_job()
    o, p = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n,
                                iters=1, epry=epry, spectrum0=spec)
    assert np.abs(o - spec).max() < 1e-12 * np.abs(spec).max()
    assert np.abs(p - g.pupils[0]).max() < 1e-12


def test_zero_spectrum_update_closed_form():
    """O = 0, constant image c: phi = 0 so phi' = sqrt(c); the box gains N^2 sqrt(c) conj(P(0)) at c + s."""
    m, n = 16, 64
    sup = np.zeros((m, m), bool)
    sup[4:12, 4:12] = True
    theta = 0.7
    pup = np.where(sup, np.exp(1j * theta), 0)
    spec = np.zeros((n, n), np.complex128)
    s = np.array([3, -5])
    c = 2.25
    dp = orc.update_one(spec, pup, sup, s, np.full((m, m), c))
    expect = np.zeros_like(spec)
    expect[n // 2 + s[0], n // 2 + s[1]] = n * n * np.sqrt(c) * np.exp(-1j * theta)
    np.testing.assert_allclose(spec, expect, atol=1e-9)
    assert np.all(dp == 0)          # empty box: no pupil information


def test_single_frequency_update_closed_form():
    """O = N^2 a delta at c+s+k0, P = e^{i theta} on the support, I = 4|a|^2:
    phi' = 2 phi, so O(c+s+k0) -> 2 N^2 a and dP(k0) = e^{i theta} (EPRY)."""
    m, n = 16, 64
    sup = orc.pupil_support(m, 1.0 / (m * DX), LAM, NA * 3)    # wider disc on a small grid
    theta = -0.4
    pup = np.where(sup, np.exp(1j * theta), 0)
    s = np.array([-2, 4])
    k0 = np.array([1, -2])
    a = 0.6 - 0.3j
    spec = np.zeros((n, n), np.complex128)
    spec[n // 2 + s[0] + k0[0], n // 2 + s[1] + k0[1]] = n * n * a
    ref = spec.copy()
    img = np.full((m, m), 4 * abs(a) ** 2)
    dp = orc.update_one(spec, pup, sup, s, img)
    ref[n // 2 + s[0] + k0[0], n // 2 + s[1] + k0[1]] = 2 * n * n * a
    np.testing.assert_allclose(spec, ref, atol=1e-8 * n * n)
    exp_dp = np.zeros((m, m), np.complex128)
    exp_dp[m // 2 + k0[0], m // 2 + k0[1]] = np.exp(1j * theta)
    np.testing.assert_allclose(dp, exp_dp, atol=1e-12)
    # consistent data (I = |a|^2) is a fixed point of the same update
    spec2 = ref.copy()
    spec2[n // 2 + s[0] + k0[0], n // 2 + s[1] + k0[1]] = n * n * a
    keep = spec2.copy()
    dp2 = orc.update_one(spec2, pup, sup, s, np.full((m, m), abs(a) ** 2))
    np.testing.assert_allclose(spec2, keep, atol=1e-8 * n * n)
    assert np.abs(dp2).max() < 1e-12


def test_fixed_pupil_waves_equal_sequence_bit_for_bit():
    g, spec, imgs = _small_job(z=0.0)
    init = orc.initial_spectrum(imgs[int(g.order[0])], g.n)
    a, _ = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n, 2, False,
                                mode="waves", spectrum0=init)
    b, _ = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n, 2, False,
                                mode="sequential", spectrum0=init)
    assert np.array_equal(a, b)


def test_reconstruction_error_decreases():
    """Noiseless data from a known object: the error of the spectrum on the synthesised
    band falls over iterations (a sanity check, not a pinned value)."""
    g, spec, imgs = _small_job(z=0.0, seed=11)
    band = np.zeros((g.n, g.n), bool)
    for s in g.shifts[0]:
        y0, x0 = orc.crop_origin(g.n, g.m, s)
        band[y0:y0 + g.m, x0:x0 + g.m] |= g.support
    errs = []
    for it in (1, 3, 6):
        o, _ = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n, it, False)
        # global phase is not recoverable: align it first
        ph = np.vdot(o[band], spec[band])
        ph /= abs(ph)
        errs.append(np.linalg.norm(o[band] * ph - spec[band]) / np.linalg.norm(spec[band]))
    assert errs[0] > errs[1] > errs[2]


def test_sequential_epry_equals_waves_when_every_wave_has_one_led():
    """All LEDs on one footprint: every wave holds a single LED, so wave-synchronous
    EPRY takes exactly the strict-sequential steps (a pin of the sequential mode
    through the independently pinned wave mode)."""
    g, spec, imgs = _small_job(z=3.0, seed=5)
    same = np.zeros_like(g.shifts[0])                      # every LED on the centre footprint
    init = orc.initial_spectrum(imgs[int(g.order[0])], g.n)
    w = orc.waves(g.n, g.support, same, orc.sequence(g.order, 2))
    assert list(w) == list(range(len(w)))
    a = orc.reconstruct_tile(imgs, same, g.order, g.support, g.pupils[0], g.n, 2, True, mode="waves",
                             spectrum0=init)
    b = orc.reconstruct_tile(imgs, same, g.order, g.support, g.pupils[0], g.n, 2, True, mode="sequential",
                             spectrum0=init)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_sequential_epry_differs_from_waves_when_leds_share_a_wave():
    """With disjoint footprints in a wave, sequential EPRY lets each later LED see the
    earlier corrections: the two modes then give different pupils."""
    g, spec, imgs = _small_job(z=3.0, seed=5)
    init = orc.initial_spectrum(imgs[int(g.order[0])], g.n)
    a = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n, 1, True, mode="waves",
                             spectrum0=init)
    b = orc.reconstruct_tile(imgs, g.shifts[0], g.order, g.support, g.pupils[0], g.n, 1, True,
                             mode="sequential", spectrum0=init)
    assert not np.array_equal(a[1], b[1])


def test_unmasked_epry_normaliser_is_the_box_maximum():
    """Unmasked EPRY (the update region is the whole m x m box): O holds N^2 a at
    c+s+k0 inside the pupil disc and N^2 2a at c+s+k1 outside it, P = e^{i theta}
    on the disc, I = 4|a|^2.  Only k0 is imaged, so phi' = 2 phi and D is
    N^2 a e^{i theta} at k0 alone; max|O_box|^2 over the box is |N^2 2a|^2, four
    times the disc's, so dP(k0) = e^{i theta} / 4 (e^{i theta} with the mask)."""
    m, n = 16, 64
    circ = orc.pupil_support(m, 1.0 / (m * DX), LAM, NA)           # radius ~4.9 px
    box = np.ones((m, m), bool)
    theta = 0.9
    pup = np.where(circ, np.exp(1j * theta), 0)
    s = np.array([2, -3])
    k0, k1 = np.array([1, 2]), np.array([-8, -8])          # k1: a box corner, outside the disc
    assert circ[m // 2 + k0[0], m // 2 + k0[1]] and not circ[m // 2 + k1[0], m // 2 + k1[1]]
    a = 0.5 + 0.2j
    base = np.zeros((n, n), np.complex128)
    base[n // 2 + s[0] + k0[0], n // 2 + s[1] + k0[1]] = n * n * a
    base[n // 2 + s[0] + k1[0], n // 2 + s[1] + k1[1]] = n * n * 2 * a
    img = np.full((m, m), 4 * abs(a) ** 2)
    for sup, scale in ((box, 0.25), (circ, 1.0)):
        spec = base.copy()
        dp = orc.update_one(spec, pup, sup, s, img)
        exp_dp = np.zeros((m, m), np.complex128)
        exp_dp[m // 2 + k0[0], m // 2 + k0[1]] = scale * np.exp(1j * theta)
        np.testing.assert_allclose(dp, exp_dp, atol=1e-12)
        ref = base.copy()
        ref[n // 2 + s[0] + k0[0], n // 2 + s[1] + k0[1]] = 2 * n * n * a    # the spectrum update is the same
        np.testing.assert_allclose(spec, ref, atol=1e-8 * n * n)
