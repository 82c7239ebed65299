"""FP64 CPU oracle for Fourier ptychographic (FPM) tile reconstruction.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA path (``paper_2203_02507_b300``) and imports nothing from it.

It is a plain, slow, sequential restatement of what the reconstruction computes,
in float64/complex128, following the steps in the order the method takes them.
numpy's FFT serves as a library primitive.  The paper describes the method in
prose only (Sec. 2.1 and Fig. 2; the figures and formulas of the update are not
given), so each formula below is the standard published form it names, and each
choice the paper leaves open is a stated reading:

  geometry          Sec. 2.2 (LED = point source; per-sub-region angle, Fig. 3/4)
  tile grid         Sec. 3.1 (overlapping sub-regions, Fig. 5)
  update order      Sec. 3.2 (spiral/centre-out and raster routines, Fig. 6)
  pupil             Sec. 1 / Sec. 2.1 (circular low-pass set by NA and wavelength),
                    Sec. 2.2 (per-sub-region defocus)
  per-LED update    Sec. 2.1 (alternating projection, Fig. 2); formulas of the
                    embedded pupil recovery (EPRY) of Ou, Zheng and Yang,
                    Opt. Express 22(5):4960 (2014), alpha = beta = 1
  waves             Sec. 3.2 (regions that do not affect one another updated
                    in parallel, across iteration loops)
  stitching         Sec. 3.1, Eq. 1 (pairwise, weights mu1/mu2 read as the
                    complex means over the shared band)

Parity status: every function below is pinned by the CPU tests in
``tests/test_oracle_*.py`` (brute-force DFT, closed-form images, the fixed-point
invariant, brute-force wave levelling, exact integer geometry).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# Rounding and FFT conventions
# ---------------------------------------------------------------------------


def lround(x):
    """C ``lround``: nearest integer, halfway cases away from zero (exact in FP64)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.trunc(x)
    frac = np.abs(x - t)                       # exact for |x| < 2**52
    return (t + np.sign(x) * (frac >= 0.5)).astype(np.int64)


def fft2c(x):
    """Centred forward 2-D DFT: fftshift(DFT(x)), unnormalised, exp(-2 pi i nk/n)."""
    return np.fft.fftshift(np.fft.fft2(x))


def ifft2c(x):
    """Inverse of ``fft2c``: IDFT(ifftshift(x)) with the 1/n^2 factor."""
    return np.fft.ifft2(np.fft.ifftshift(x))


# ---------------------------------------------------------------------------
# Geometry (Sec. 2.2, Sec. 3.1)
# ---------------------------------------------------------------------------


@dataclass
class Geometry:
    """Everything the update needs that does not depend on the data."""
    m: int                      # LR tile side
    n: int                      # HR side = upsample * m
    df: float                   # Fourier pixel, 1 / (m * dx)
    origins: np.ndarray         # [T, 2] (y0, x0) tile origins on the sensor
    centres_um: np.ndarray      # [T, 2] (y, x) tile centres from the optical axis
    shifts: np.ndarray          # [T, L, 2] integer (sy, sx) sub-aperture shifts
    order: np.ndarray           # [L] LED visiting order
    support: np.ndarray         # [m, m] bool, circular pupil support (centred)
    pupils: np.ndarray          # [T, m, m] complex128 initial pupils


def tile_origins(sensor_h, sensor_w, m, overlap, tiles_y, tiles_x):
    """Origins of a tiles_y x tiles_x grid of m x m tiles, stride m - overlap.

    The grid is centred on the sensor; the leftover margin, floor((S - span)/2),
    is left unreconstructed (reading: the paper gives tile size and overlap, not
    the placement of the grid).
    """
    stride = m - overlap
    span_y = (tiles_y - 1) * stride + m
    span_x = (tiles_x - 1) * stride + m
    my = (sensor_h - span_y) // 2
    mx = (sensor_w - span_x) // 2
    out = np.zeros((tiles_y * tiles_x, 2), dtype=np.int64)
    for i in range(tiles_y):
        for j in range(tiles_x):
            out[i * tiles_x + j] = (my + i * stride, mx + j * stride)
    return out


def tile_centres_um(origins, m, sensor_h, sensor_w, pixel_um):
    """Tile centre in micrometres relative to the sensor centre (optical axis)."""
    o = np.asarray(origins, dtype=np.float64)
    yc = (o[:, 0] + m / 2.0 - sensor_h / 2.0) * pixel_um
    xc = (o[:, 1] + m / 2.0 - sensor_w / 2.0) * pixel_um
    return np.stack([yc, xc], axis=1)


def led_shifts(centres_um, led_xy_um, led_height_um, wavelength_um, df):
    """Integer sub-aperture shifts (sy, sx) per tile and LED (Sec. 2.2).

    The LED is a point source; over one small tile its light is taken as a plane
    wave whose direction cosines are those of the line from the tile centre to
    the LED: u = (x_led - x_c) / R, v = (y_led - y_c) / R with
    R = sqrt((x_led - x_c)^2 + (y_led - y_c)^2 + h^2).  The illumination
    spatial frequency u / lambda is expressed in Fourier pixels and rounded
    half away from zero (integer-pixel shifts; the sub-pixel rest is dropped).
    """
    t_n = len(centres_um)
    l_n = len(led_xy_um)
    out = np.zeros((t_n, l_n, 2), dtype=np.int64)
    h = float(led_height_um)
    for t in range(t_n):
        yc, xc = float(centres_um[t, 0]), float(centres_um[t, 1])
        for i in range(l_n):
            dx = float(led_xy_um[i, 0]) - xc
            dy = float(led_xy_um[i, 1]) - yc
            r = math.sqrt(dx * dx + dy * dy + h * h)
            u = dx / r
            v = dy / r
            out[t, i, 0] = lround(v / (wavelength_um * df))
            out[t, i, 1] = lround(u / (wavelength_um * df))
    return out


def led_order(led_xy_um, routine="center_out"):
    """LED visiting order (Sec. 3.2, Fig. 6).

    "center_out": the spiral-outward routine read as increasing distance of the
    LED from the array centre (the optical axis), ties by LED index.
    "raster": LED index order.
    """
    l_n = len(led_xy_um)
    idx = np.arange(l_n)
    if routine == "raster":
        return idx
    x = led_xy_um[:, 0]
    y = led_xy_um[:, 1]
    d2 = x * x + y * y
    return np.lexsort((idx, d2)).astype(np.int64)


def pupil_support(m, df, wavelength_um, na):
    """Circular pupil support: |f| <= NA / lambda, f = k * df, k in [-m/2, m/2)^2."""
    k = np.arange(m) - m // 2
    fy, fx = np.meshgrid(k * df, k * df, indexing="ij")
    return np.sqrt(fx * fx + fy * fy) <= na / wavelength_um


def pupil(m, df, wavelength_um, na, defocus_um):
    """Initial pupil of one tile: circ support times the defocus phase (Sec. 2.2).

    P = circ * exp(i 2 pi z (sqrt(1/lambda^2 - |f|^2) - 1/lambda)).  The constant
    1/lambda only removes a global phase.  Sign of z: +z (paper silent).
    """
    k = np.arange(m) - m // 2
    fy, fx = np.meshgrid(k * df, k * df, indexing="ij")
    f2 = fx * fx + fy * fy
    inv_l = 1.0 / wavelength_um
    kz = np.sqrt(np.maximum(inv_l * inv_l - f2, 0.0)) - inv_l
    circ = np.sqrt(f2) <= na / wavelength_um
    return np.where(circ, np.exp(1j * 2.0 * math.pi * defocus_um * kz), 0.0)


def geometry(sensor_h, sensor_w, m, overlap, tiles_y, tiles_x, upsample, wavelength_um,
             na, pixel_um, led_xy_um, led_height_um, defocus_um, routine="center_out"):
    """All data-independent quantities of a job, computed from the problem statement."""
    df = 1.0 / (m * pixel_um)
    origins = tile_origins(sensor_h, sensor_w, m, overlap, tiles_y, tiles_x)
    centres = tile_centres_um(origins, m, sensor_h, sensor_w, pixel_um)
    shifts = led_shifts(centres, np.asarray(led_xy_um, np.float64), led_height_um,
                        wavelength_um, df)
    order = led_order(np.asarray(led_xy_um, np.float64), routine)
    support = pupil_support(m, df, wavelength_um, na)
    pupils = np.stack([pupil(m, df, wavelength_um, na, float(z)) for z in defocus_um])
    return Geometry(m=m, n=upsample * m, df=df, origins=origins, centres_um=centres,
                    shifts=shifts, order=order, support=support, pupils=pupils)


def crop_origin(n, m, shift):
    """Top-left HR index of the m x m sub-aperture box centred at c + s, c = n/2."""
    return n // 2 + int(shift[0]) - m // 2, n // 2 + int(shift[1]) - m // 2


# ---------------------------------------------------------------------------
# Forward model (Sec. 2.1, Fig. 1)
# ---------------------------------------------------------------------------


def forward_images(spectrum, pupil_, shifts, m):
    """Clean LR intensities of one tile for every LED.

    spectrum: centred N x N HR spectrum O = fft2c(o).  For LED with shift s:
    Phi = O[box(c + s)] * P;  phi = (m/N)^2 * ifft2c(Phi);  I = |phi|^2.
    The (m/N)^2 factor makes a unit plane-wave object inside the pupil image to
    intensity 1.
    """
    n = spectrum.shape[0]
    scale = (m / n) ** 2
    out = np.zeros((len(shifts), m, m))
    for i, s in enumerate(shifts):
        y0, x0 = crop_origin(n, m, s)
        phi = scale * ifft2c(spectrum[y0:y0 + m, x0:x0 + m] * pupil_)
        out[i] = np.abs(phi) ** 2
    return out


# ---------------------------------------------------------------------------
# Initial guess
# ---------------------------------------------------------------------------


def initial_spectrum(i_centre, n):
    """Spectrum of the upsampled centre image: (N/m)^2 * zero-pad_N(fft2c(sqrt(I_c))).

    The centred m x m spectrum is placed unsplit at the centre of the N x N grid
    (its Nyquist row and column copied as they are).  A constant unit image gives
    the object o = 1.
    """
    m = i_centre.shape[0]
    small = fft2c(np.sqrt(np.maximum(i_centre, 0.0)))
    big = np.zeros((n, n), dtype=np.complex128)
    o = n // 2 - m // 2
    big[o:o + m, o:o + m] = small * (n / m) ** 2
    return big


# ---------------------------------------------------------------------------
# The per-LED update (Sec. 2.1; EPRY formulas)
# ---------------------------------------------------------------------------


def update_one(spectrum, pupil_, support, shift, intensity, p_norm=None):
    """One LED sub-aperture update, in place on ``spectrum``; returns dP.

    Steps, for the box centred at c + s:
      Phi  = O_box * P
      phi  = (m/N)^2 * ifft2c(Phi)
      phi' = sqrt(I) * phi / |phi|       (phi' = sqrt(I) where phi == 0)
      Phi' = fft2c(phi') / (m/N)^2
      D    = Phi' - Phi
      O_box <- O_box + conj(P) * D / max_support |P|^2
      dP    = support * conj(O_box_old) * D / max_support |O_box_old|^2
              (dP = 0 when that maximum is 0: an empty box says nothing about P)
    ``p_norm`` (max |P|^2 over the support) may be passed in; by default it is
    taken from ``pupil_``.  The pupil itself is not modified here.
    """
    n = spectrum.shape[0]
    m = pupil_.shape[0]
    y0, x0 = crop_origin(n, m, shift)
    old = spectrum[y0:y0 + m, x0:x0 + m].copy()
    scale = (m / n) ** 2
    big_phi = old * pupil_
    phi = scale * ifft2c(big_phi)
    amp = np.sqrt(np.maximum(intensity, 0.0))
    mag = np.abs(phi)
    safe = np.where(mag > 0.0, mag, 1.0)
    phi_new = np.where(mag > 0.0, amp * phi / safe, amp)
    big_phi_new = fft2c(phi_new) / scale
    delta = big_phi_new - big_phi
    if p_norm is None:
        p_norm = np.max(np.abs(pupil_[support]) ** 2)
    spectrum[y0:y0 + m, x0:x0 + m] = old + np.conj(pupil_) * delta / p_norm
    o_norm = np.max(np.abs(old[support]) ** 2)
    if o_norm == 0.0:            # empty box: no information for the pupil (reading)
        return np.zeros_like(pupil_)
    return np.where(support, np.conj(old) * delta / o_norm, 0.0)


# ---------------------------------------------------------------------------
# Waves (Sec. 3.2): dependency levelling of the update sequence
# ---------------------------------------------------------------------------


def footprint(n, support, shift):
    """Flat HR indices touched by the update of one LED (its support disc at c + s)."""
    m = support.shape[0]
    y0, x0 = crop_origin(n, m, shift)
    ky, kx = np.nonzero(support)
    return (y0 + ky) * n + (x0 + kx)


def sequence(order, iters):
    """The update sequence: the LED order repeated for every iteration loop."""
    return np.tile(np.asarray(order, dtype=np.int64), iters)


def waves(n, support, shifts_tile, seq):
    """Wave id of every item of ``seq`` for one tile.

    wave(j) = 0 if no earlier item's footprint meets item j's, else
    1 + max{ wave(i) : i < j, footprint(i) and footprint(j) intersect }.
    Computed with a per-pixel record of the highest wave that touched the pixel,
    which holds exactly that maximum.
    """
    last = np.full(n * n, -1, dtype=np.int64)
    fps = {}
    out = np.zeros(len(seq), dtype=np.int64)
    for j, led in enumerate(seq):
        led = int(led)
        if led not in fps:
            fps[led] = footprint(n, support, shifts_tile[led])
        fp = fps[led]
        w = int(last[fp].max()) + 1
        last[fp] = w
        out[j] = w
    return out


# ---------------------------------------------------------------------------
# Reconstruction of one tile
# ---------------------------------------------------------------------------


def reconstruct_tile(images, geom_shifts, order, support, pupil0, n, iters, epry,
                     mode="waves", spectrum0=None, return_pupil=True):
    """Reconstruct one tile; returns (spectrum, pupil).

    images: [L, m, m] measured intensities in model units (index = LED index).
    mode "waves": the sequence is split into waves (``waves``); every LED of a
      wave uses the pupil as it was at the start of the wave, and the wave's
      pupil corrections are added in ascending sequence order when the wave
      ends ("wave-synchronous EPRY").  With a fixed pupil this equals the
      strict sequence exactly.
    mode "sequential": strict sequence order, pupil corrected after every LED.
    """
    seq = sequence(order, iters)
    if spectrum0 is None:
        spectrum = initial_spectrum(images[int(order[0])], n)
    else:
        spectrum = spectrum0.copy()
    p = pupil0.copy()
    if mode == "sequential":
        for led in seq:
            dp = update_one(spectrum, p, support, geom_shifts[int(led)], images[int(led)])
            if epry:
                p = p + dp
        return spectrum, p
    w = waves(n, support, geom_shifts, seq)
    for wave_id in range(int(w.max()) + 1 if len(w) else 0):
        members = np.nonzero(w == wave_id)[0]
        p_start = p.copy()
        p_norm = np.max(np.abs(p_start[support]) ** 2)
        dps = []
        for j in members:
            led = int(seq[j])
            dps.append(update_one(spectrum, p_start, support, geom_shifts[led],
                                  images[led], p_norm=p_norm))
        if epry:
            for dp in dps:
                p = p + dp
    return spectrum, p


def tile_images_from_stack(stack, origin, m, counts_per_unit=1.0):
    """The tile's window of the sensor stack, in model units, as float64."""
    y0, x0 = int(origin[0]), int(origin[1])
    return stack[:, y0:y0 + m, x0:x0 + m].astype(np.float64) / counts_per_unit


def object_from_spectrum(spectrum):
    """HR complex object o = ifft2c(O)."""
    return ifft2c(spectrum)


# ---------------------------------------------------------------------------
# Stitching of the tile objects into one HR field of view (Eq. 1, Sec. 3.1)
# ---------------------------------------------------------------------------

def hr_overlap(overlap, upsample):
    """Lines shared by neighbouring tile objects on the HR grid.

    Reading: tiles are cut on the LR sensor with `overlap` shared pixels and
    each tile's object lives on a grid `upsample` times finer, so neighbouring
    objects share overlap * upsample lines.  (The paper's example, 256 x 256
    images sharing 26 lines, gives sizes in one pixel grid only.)
    """
    return int(overlap) * int(upsample)


def stitch_pair(f1, f2, overlap, axis):
    """Eq. 1 for one pair: f2 continues f1 along `axis`, the two sharing `overlap` lines.

    axis 0 is the paper's part 1 (f2 below f1, the condition on the row index
    x), axis 1 its part 2 (f2 right of f1, the condition on the column index y).
    With r lines in f1, output line i < r - overlap/2 is f1's line i; every
    later output line i is (mu1 / mu2) times f2's line i - (r - overlap), so the
    output has r + r2 - overlap lines.  overlap/2 is taken as overlap // 2.

    Reading of the weights: mu1 and mu2 are the complex means of f1 and f2 over
    the band both images cover (f1's last `overlap` lines, f2's first), the
    only region in which their ratio compares the same part of the sample.  A
    zero mu2 leaves f2 unscaled, and so does overlap 0 (no shared band: the
    images are placed side by side).
    """
    a = np.moveaxis(np.asarray(f1, dtype=np.complex128), axis, 0)
    b = np.moveaxis(np.asarray(f2, dtype=np.complex128), axis, 0)
    if a.shape[1:] != b.shape[1:]:
        raise ValueError("the images must agree across the stitching axis")
    r, r2 = a.shape[0], b.shape[0]
    if overlap < 0 or overlap > min(r, r2):
        raise ValueError("overlap out of range")
    w = 1.0
    if overlap > 0:
        mu1 = np.ascontiguousarray(a[r - overlap:]).mean()     # contiguous copies: one summation
        mu2 = np.ascontiguousarray(b[:overlap]).mean()         # order for both bands
        w = mu1 / mu2 if mu2 != 0 else 1.0
    cut = r - overlap // 2
    out = np.empty((r + r2 - overlap,) + a.shape[1:], dtype=np.complex128)
    out[:cut] = a[:cut]
    out[cut:] = w * b[cut - (r - overlap):]
    return np.moveaxis(out, 0, axis)


def stitch_grid(objects, tiles_y, tiles_x, overlap):
    """One field-of-view image from the tile objects (Eq. 1, Sec. 3.1).

    objects[i * tiles_x + j] is the object of the tile in grid row i, column j.
    Each column of tiles is stitched top to bottom (part 1), the running result
    being f1 of the next stitch; the column images are then stitched left to
    right the same way (part 2), the paper's part-1 output being part 2's input.
    """
    strips = []
    for j in range(tiles_x):
        s = np.asarray(objects[j], dtype=np.complex128)
        for i in range(1, tiles_y):
            s = stitch_pair(s, objects[i * tiles_x + j], overlap, 0)
        strips.append(s)
    out = strips[0]
    for j in range(1, tiles_x):
        out = stitch_pair(out, strips[j], overlap, 1)
    return out
