"""Pins of the oracle's forward model and initial guess against closed forms (Sec. 2.1, Fig. 1)."""
import numpy as np
import pytest

from oracle import fpm_oracle as orc

LAM, NA, DX = 0.532, 0.10, 1.625


def _plane_wave(n, ky, kx, amp=1.0):
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return amp * np.exp(2j * np.pi * (ky * y + kx * x) / n)


@pytest.mark.parametrize("m", [32, 64])
def test_plane_wave_object_images_to_one_or_zero(m):
    """A plane-wave object on the HR grid images to I = |P(a - s)|^2: 1 inside the pupil, 0 outside."""
    n = 4 * m
    df = 1.0 / (m * DX)
    sup = orc.pupil_support(m, df, LAM, NA)
    pup = orc.pupil(m, df, LAM, NA, 7.5)            # phase-only on the support
    rng = np.random.default_rng(m)
    for _ in range(12):
        a = rng.integers(-m // 2, m // 2, size=2)
        s = rng.integers(-m // 2, m // 2, size=2)
        spec = orc.fft2c(_plane_wave(n, a[0], a[1]))
        img = orc.forward_images(spec, pup, s[None, :], m)[0]
        k = a - s
        inside = (-m // 2 <= k[0] < m // 2) and (-m // 2 <= k[1] < m // 2) and sup[k[0] + m // 2, k[1] + m // 2]
        np.testing.assert_allclose(img, np.full((m, m), 1.0 if inside else 0.0), atol=1e-10)


def test_two_plane_waves_give_the_closed_form_fringe():
    m, n = 32, 128
    df = 1.0 / (m * DX)
    pup = orc.pupil(m, df, LAM, NA, -12.0)
    c1, c2 = 0.8 * np.exp(0.3j), 0.45 * np.exp(-1.1j)
    a1, a2 = np.array([3, -2]), np.array([-4, 5])
    s = np.array([1, 2])
    obj = _plane_wave(n, *a1, amp=c1) + _plane_wave(n, *a2, amp=c2)
    img = orc.forward_images(orc.fft2c(obj), pup, s[None, :], m)[0]
    k1, k2 = a1 - s, a2 - s
    p1 = pup[k1[0] + m // 2, k1[1] + m // 2]
    p2 = pup[k2[0] + m // 2, k2[1] + m // 2]
    y, x = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    dk = k1 - k2
    fringe = (abs(c1 * p1) ** 2 + abs(c2 * p2) ** 2
              + 2 * np.real(c1 * p1 * np.conj(c2 * p2) * np.exp(2j * np.pi * (dk[0] * y + dk[1] * x) / m)))
    assert abs(p1) > 0.5 and abs(p2) > 0.5
    np.testing.assert_allclose(img, fringe, atol=1e-10)


def test_unit_image_initialises_unit_object():
    for m in (16, 24, 32):
        n = 4 * m
        spec = orc.initial_spectrum(np.ones((m, m)), n)
        np.testing.assert_allclose(orc.object_from_spectrum(spec), np.ones((n, n)), atol=1e-12)


def test_initial_spectrum_of_plane_wave_amplitude():
    """sqrt of a modulated image: its centred spectrum lands at the centre of the HR grid, scaled by (N/m)^2."""
    m, n = 16, 64
    y, x = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    amp = 1.0 + 0.25 * np.cos(2 * np.pi * 3 * x / m)          # sqrt(I) = amp
    spec = orc.initial_spectrum(amp ** 2, n)
    c = n // 2
    assert abs(spec[c, c] - n * n) < 1e-8
    assert abs(spec[c, c + 3] - 0.125 * n * n) < 1e-8
    assert abs(spec[c, c - 3] - 0.125 * n * n) < 1e-8
    spec[c, c] = spec[c, c + 3] = spec[c, c - 3] = 0
    assert np.abs(spec).max() < 1e-8
