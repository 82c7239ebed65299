"""The float32 floor of a job: the oracle's own steps executed in complex64.

Tolerance calibration for tests only.  It reuses the oracle's geometry, waves
and conventions and repeats its update with complex64 arrays and numpy's
float32 FFTs, so the difference between this run and the FP64 oracle is what
float32 arithmetic of the same algorithm produces on that data.  Jobs whose
EPRY pupil correction is driven by many dark-field LEDs amplify that rounding
(the correction divides by a small max|O_box|^2); their GPU bound is a
multiple of this floor instead of a fixed number.
"""
import numpy as np

from oracle import fpm_oracle as orc


def _update32(spectrum, pupil_, support, shift, intensity, p_norm):
    n = spectrum.shape[0]
    m = pupil_.shape[0]
    y0, x0 = orc.crop_origin(n, m, shift)
    old = spectrum[y0:y0 + m, x0:x0 + m].copy()
    big_phi = (old * pupil_).astype(np.complex64)
    # (m/N)^2 IFFT: the constant factor cancels in phi/|phi|, the forward step restores it
    phi = np.fft.ifft2(np.fft.ifftshift(big_phi)).astype(np.complex64)     # float32 FFT
    amp = np.sqrt(np.maximum(intensity, 0)).astype(np.float32)
    mag = np.abs(phi)
    phi_new = np.where(mag > 0, amp * phi / np.where(mag > 0, mag, 1), amp).astype(np.complex64)
    big_new = (np.fft.fftshift(np.fft.fft2(phi_new)) * np.float32((n / m) ** 2)).astype(np.complex64)
    delta = (big_new - big_phi).astype(np.complex64)
    spectrum[y0:y0 + m, x0:x0 + m] = old + np.conj(pupil_) * delta / np.float32(p_norm)
    o_norm = np.max(np.abs(old[support]) ** 2)
    if o_norm == 0:
        return np.zeros_like(pupil_)
    return np.where(support, np.conj(old) * delta / o_norm, 0).astype(np.complex64)


def reconstruct_tile32(images, shifts, order, support, pupil0, n, iters, epry, mode="waves"):
    """Reconstruction of one tile in complex64 (see fpm_oracle.reconstruct_tile): wave-
    synchronous, or strict sequential (one update per wave)."""
    seq = orc.sequence(order, iters)
    w = orc.waves(n, support, shifts, seq) if mode == "waves" else np.arange(len(seq))
    spec = orc.initial_spectrum(images[int(order[0])], n).astype(np.complex64)
    p = pupil0.astype(np.complex64)
    for wid in range(int(w.max()) + 1):
        members = np.nonzero(w == wid)[0]
        p_start = p.copy()
        pn = np.max(np.abs(p_start[support]) ** 2)
        dps = [_update32(spec, p_start, support, shifts[int(seq[j])], images[int(seq[j])].astype(np.float32), pn)
               for j in members]
        if epry:
            for dp in dps:
                p = p + dp
    return spec, p


def floor(images, shifts, order, support, pupil0, n, iters, epry, ref_spec, ref_pup, mode="waves"):
    """(spectrum, pupil) rel-L2 of the complex64 run against the FP64 oracle's result."""
    s32, p32 = reconstruct_tile32(images, shifts, order, support, pupil0, n, iters, epry, mode)
    rs = float(np.linalg.norm(s32 - ref_spec) / np.linalg.norm(ref_spec))
    rp = float(np.linalg.norm(p32 - ref_pup) / np.linalg.norm(ref_pup))
    return rs, rp
