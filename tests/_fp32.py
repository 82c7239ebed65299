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


# ---------------------------------------------------------------------------
# Step-by-step attribution of the float32 floor
# ---------------------------------------------------------------------------

STEPS = ("prod", "ifft", "amp", "fft", "delta", "spec", "dp", "merge", "state")


def _r(x, on):
    """x rounded to complex64 (kept in complex128) when `on`."""
    return x.astype(np.complex64).astype(np.complex128) if on else x


def _update_mixed(spectrum, pupil_, support, shift, intensity, p_norm, f32):
    n = spectrum.shape[0]
    m = pupil_.shape[0]
    y0, x0 = orc.crop_origin(n, m, shift)
    old = spectrum[y0:y0 + m, x0:x0 + m].copy()
    scale = (m / n) ** 2
    big_phi = _r(old * pupil_, "prod" in f32)
    if "ifft" in f32:
        phi = np.fft.ifft2(np.fft.ifftshift(big_phi.astype(np.complex64))).astype(np.complex64).astype(np.complex128)
    else:
        phi = orc.ifft2c(big_phi)
    phi = scale * phi
    amp = np.sqrt(np.maximum(intensity, 0.0))
    mag = np.abs(phi)
    phi_new = _r(np.where(mag > 0.0, amp * phi / np.where(mag > 0.0, mag, 1.0), amp), "amp" in f32)
    if "fft" in f32:
        big_new = np.fft.fftshift(np.fft.fft2(phi_new.astype(np.complex64))).astype(np.complex64).astype(np.complex128)
    else:
        big_new = orc.fft2c(phi_new)
    delta = _r(big_new / scale - big_phi, "delta" in f32)
    spectrum[y0:y0 + m, x0:x0 + m] = _r(old + np.conj(pupil_) * delta / p_norm, "spec" in f32)
    o_norm = np.max(np.abs(old[support]) ** 2)
    if o_norm == 0.0:
        return np.zeros_like(pupil_)
    return _r(np.where(support, np.conj(old) * delta / o_norm, 0.0), "dp" in f32)


def reconstruct_mixed(images, shifts, order, support, pupil0, n, iters, f32):
    """The oracle's wave-synchronous EPRY with the steps named in `f32` (a subset of
    STEPS) rounded to float32 and every other step in FP64: f32 = () is the oracle
    itself, f32 = STEPS the float32 restatement above."""
    seq = orc.sequence(order, iters)
    w = orc.waves(n, support, shifts, seq)
    spec = _r(orc.initial_spectrum(images[int(order[0])], n), "state" in f32)
    p = _r(pupil0.astype(np.complex128), "state" in f32)
    for wid in range(int(w.max()) + 1):
        members = np.nonzero(w == wid)[0]
        ps = p.copy()
        pn = np.max(np.abs(ps[support]) ** 2)
        dps = [_update_mixed(spec, ps, support, shifts[int(seq[j])], images[int(seq[j])], pn, f32) for j in members]
        for dp in dps:
            p = _r(p + dp, "merge" in f32)
    return spec, p
