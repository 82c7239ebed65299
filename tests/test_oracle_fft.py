"""Pins of the oracle's centred FFT against the DFT's definition (Sec. 3.3: FFT/IFFT)."""
import numpy as np
import pytest

from oracle import fpm_oracle as orc


def brute_dft2_centred(x, sign):
    """X[ky, kx] = sum_{y, x} x[y, x] exp(sign 2 pi i (ky y + kx x) / n), k in [-n/2, n/2).

    Written out as an explicit double sum over frequencies, with the centred
    frequency k stored at index k + n/2.
    """
    n = x.shape[0]
    ks = np.arange(n) - n // 2
    ys = np.arange(n)
    out = np.zeros((n, n), dtype=np.complex128)
    for iy, ky in enumerate(ks):
        for ix, kx in enumerate(ks):
            ph = np.exp(sign * 2j * np.pi * (ky * ys[:, None] + kx * ys[None, :]) / n)
            out[iy, ix] = np.sum(x * ph)
    return out


@pytest.mark.parametrize("n", [8, 12, 16, 24])
def test_fft2c_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ref = brute_dft2_centred(x, -1)
    np.testing.assert_allclose(orc.fft2c(x), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("n", [8, 12, 16])
def test_ifft2c_matches_brute_force_idft(n):
    rng = np.random.default_rng(100 + n)
    big = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    # inverse of the centred transform: x[y,x] = 1/n^2 sum_k X[k] exp(+2 pi i k.r / n)
    ks = np.arange(n) - n // 2
    ref = np.zeros((n, n), dtype=np.complex128)
    for y in range(n):
        for xx in range(n):
            ph = np.exp(2j * np.pi * (ks[:, None] * y + ks[None, :] * xx) / n)
            ref[y, xx] = np.sum(big * ph) / n ** 2
    np.testing.assert_allclose(orc.ifft2c(big), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n", [64, 192, 256])
def test_parseval_and_round_trip(n):
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    big = orc.fft2c(x)
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(big) ** 2) / n ** 2) < 1e-9 * np.sum(np.abs(x) ** 2)
    np.testing.assert_allclose(orc.ifft2c(big), x, atol=1e-12)


def test_dc_of_constant_is_at_centre():
    n = 16
    big = orc.fft2c(np.ones((n, n)))
    assert abs(big[n // 2, n // 2] - n * n) < 1e-9
    big[n // 2, n // 2] = 0
    assert np.abs(big).max() < 1e-9
