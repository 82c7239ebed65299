"""Workload descriptions and seeded generators for synthetic FPM data.

The paper's own data is not public (Data availability statement), so every input
here is synthetic.  The shapes follow the paper's workloads: square LR
sub-regions (256x256 in Sec. 3.1 and Sec. 4), a programmable LED array above
the sample (Sec. 2.2, Sec. 4), 12-bit camera images.

Recipe (seeded with ``numpy.random.default_rng``):
  * HR object of one tile: amplitude = white N(0,1) noise, periodic Gaussian
    smoothing (sigma = 2 HR pixels), min-max mapped to [0.5, 1]; phase = an
    independent field made the same way, mapped to [-pi/2, pi/2].
  * Per-tile defocus: uniform in [lo, hi] micrometres.
  * Camera noise: counts = Poisson(k * I0) + N(0, sigma_read^2), rounded,
    clipped to [0, 4095]; k = peak / max(I0) over the job's stack, so the
    measured intensity in model units is counts / k.
  * Seeds: amplitude 1, phase 2, noise 3, defocus 4, arrivals 5; job j adds
    1000*j; tile t of a job is drawn from SeedSequence([seed, t]).

No function here performs a Fourier transform or evaluates the imaging model:
the clean intensities I0 are produced by whoever calls ``add_noise``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

SEED_AMP, SEED_PHASE, SEED_NOISE, SEED_DEFOCUS, SEED_ARRIVAL = 1, 2, 3, 4, 5


@dataclasses.dataclass(frozen=True)
class Optics:
    """Illumination/objective description (Sec. 2.1, Sec. 2.2, Sec. 4)."""
    wavelength_um: float = 0.532
    na: float = 0.10
    pixel_um: float = 1.625          # LR pixel size in the sample plane
    led_side: int = 15               # LEDs per side of the square array
    led_pitch_um: float = 4000.0
    led_height_um: float = 90000.0


@dataclasses.dataclass(frozen=True)
class Workload:
    """One reconstruction job: sensor, tiling, optics, schedule and data model."""
    name: str
    sensor: int                      # square LR sensor side (pixels)
    tile: int                        # LR tile side m
    tiles: int                       # tiles per side
    overlap: int                     # LR overlap between adjacent tiles
    iters: int
    epry: bool
    optics: Optics
    upsample: int = 4
    defocus_um: tuple = (0.0, 0.0)   # uniform range
    image_dtype: str = "u16"         # "u16" (12-bit counts) or "f32" (noiseless)
    peak_counts: float = 3000.0
    read_sigma: float = 2.0
    seed_offset: int = 0             # 1000 * job index

    @property
    def hr(self) -> int:
        return self.upsample * self.tile

    @property
    def n_tiles(self) -> int:
        return self.tiles * self.tiles

    @property
    def n_leds(self) -> int:
        return self.optics.led_side ** 2

    @property
    def updates(self) -> int:
        """LED sub-aperture updates of the whole job."""
        return self.n_tiles * self.n_leds * self.iters

    def stack_bytes(self) -> int:
        b = 2 if self.image_dtype == "u16" else 4
        return self.n_leds * self.sensor * self.sensor * b

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


_O15 = Optics(led_side=15)
_O21 = Optics(led_side=21)

WORKLOADS = {
    # single 64x64 LR sub-region, noiseless float32 images, fixed pupil
    "tile64_plain": Workload("tile64_plain", sensor=64, tile=64, tiles=1, overlap=0,
                             iters=10, epry=False, optics=_O15, image_dtype="f32"),
    # full 2048^2 FOV, 8x8 tiles of 256, EPRY + waves, 12-bit noisy
    "fov2048_m256": Workload("fov2048_m256", sensor=2048, tile=256, tiles=8, overlap=16,
                             iters=20, epry=True, optics=_O15, defocus_um=(-20.0, 20.0)),
    # the three jobs of the uneven persistent batch
    "batch_m128": Workload("batch_m128", sensor=1024, tile=128, tiles=8, overlap=16,
                           iters=15, epry=True, optics=Optics(led_side=9),
                           defocus_um=(-20.0, 20.0), seed_offset=0),
    "batch_m192": Workload("batch_m192", sensor=1536, tile=192, tiles=8, overlap=16,
                           iters=15, epry=True, optics=Optics(led_side=13),
                           defocus_um=(-20.0, 20.0), seed_offset=1000),
    "batch_m256": Workload("batch_m256", sensor=2048, tile=256, tiles=8, overlap=16,
                           iters=15, epry=True, optics=_O15,
                           defocus_um=(-20.0, 20.0), seed_offset=2000),
    # largest single job: 5120^2 sensor, 40x40 tiles of 128, 21x21 LEDs
    "fov5120_m128": Workload("fov5120_m128", sensor=5120, tile=128, tiles=40, overlap=0,
                             iters=20, epry=True, optics=_O21, defocus_um=(-30.0, 30.0)),
}


def led_grid(side: int, pitch_um: float) -> np.ndarray:
    """LED (x, y) positions in micrometres, row-major, centred on the optical axis.

    LED index i = row * side + col; x grows with col, y with row.
    """
    c = (side - 1) / 2.0
    rows, cols = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    xy = np.stack([(cols.ravel() - c) * pitch_um, (rows.ravel() - c) * pitch_um], axis=1)
    return np.ascontiguousarray(xy, dtype=np.float64)


def _rng(seed: int, tile: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([seed, tile]))


def _smoothed(rng: np.random.Generator, n: int, sigma: float) -> np.ndarray:
    f = ndimage.gaussian_filter(rng.standard_normal((n, n)), sigma=sigma, mode="wrap")
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo)


def hr_object(n: int, tile: int, seed_offset: int = 0, sigma: float = 2.0) -> np.ndarray:
    """HR complex object of one tile: amplitude in [0.5, 1], phase in [-pi/2, pi/2]."""
    amp = 0.5 + 0.5 * _smoothed(_rng(SEED_AMP + seed_offset, tile), n, sigma)
    ph = (_smoothed(_rng(SEED_PHASE + seed_offset, tile), n, sigma) - 0.5) * math.pi
    return amp * np.exp(1j * ph)


def tile_defocus(n_tiles: int, lo: float, hi: float, seed_offset: int = 0) -> np.ndarray:
    """Per-tile defocus distances (micrometres), uniform in [lo, hi]."""
    if lo == hi:
        return np.full(n_tiles, float(lo))
    return _rng(SEED_DEFOCUS + seed_offset, 0).uniform(lo, hi, size=n_tiles)


def add_noise(i0: np.ndarray, peak: float, read_sigma: float, seed_offset: int = 0):
    """12-bit camera counts from clean intensities.

    Returns (counts as uint16, counts_per_unit k) with counts ~ Poisson(k*I0) +
    N(0, read_sigma^2), rounded and clipped to [0, 4095], k = peak / max(I0).
    """
    rng = _rng(SEED_NOISE + seed_offset, 0)
    k = float(peak / i0.max())
    c = rng.poisson(k * i0).astype(np.float64) + rng.normal(0.0, read_sigma, size=i0.shape)
    return np.clip(np.rint(c), 0, 4095).astype(np.uint16), k


def owner_windows(origins: np.ndarray, m: int, sensor: int) -> np.ndarray:
    """Which part of each tile window a tile writes into the sensor image.

    A sensor pixel covered by several tiles is taken from the tile whose centre
    is nearest; along each axis of a regular grid that is the pixel's side of
    the midpoint between neighbouring tile centres (ties go to the lower tile).
    ``origins`` is the [T, 2] (y0, x0) array of tile origins.  Returns [T, 4]
    (y_lo, y_hi, x_lo, x_hi) in tile-local coordinates, half-open.
    """
    origins = np.asarray(origins, dtype=np.int64)
    out = np.zeros((len(origins), 4), dtype=np.int64)
    for axis in (0, 1):
        starts = np.unique(origins[:, axis])
        for t, o in enumerate(origins[:, axis]):
            j = int(np.searchsorted(starts, o))
            lo, hi = 0, m
            if j > 0:   # midpoint with the previous tile: centres o_prev + m/2 and o + m/2
                mid2 = starts[j - 1] + o + m            # 2 * midpoint
                lo = max(0, (mid2 + 1) // 2 - o)        # pixels >= mid go to this tile
            if j + 1 < len(starts):
                mid2 = o + starts[j + 1] + m
                hi = min(m, (mid2 + 1) // 2 - o)
            out[t, 2 * axis] = lo
            out[t, 2 * axis + 1] = hi
    return out


def assemble_sensor(tile_images: np.ndarray, origins: np.ndarray, sensor: int) -> np.ndarray:
    """Place per-tile images [T, L, m, m] into a sensor stack [L, S, S].

    Each sensor pixel comes from the tile that owns it (``owner_windows``);
    pixels outside every tile stay zero.
    """
    t_n, l_n, m, _ = tile_images.shape
    stack = np.zeros((l_n, sensor, sensor), dtype=tile_images.dtype)
    win = owner_windows(origins, m, sensor)
    for t in range(t_n):
        y0, x0 = (int(v) for v in origins[t])
        ylo, yhi, xlo, xhi = (int(v) for v in win[t])
        stack[:, y0 + ylo:y0 + yhi, x0 + xlo:x0 + xhi] = tile_images[t, :, ylo:yhi, xlo:xhi]
    return stack


def serving_jobs(n_jobs: int = 500, rate_per_s: float = 2.0, seed: int = SEED_ARRIVAL):
    """Job stream for the serving workload: Poisson arrivals and random job shapes.

    Sensor side from {512, 1024, 1536, 2048}, tile from {64, 128, 256}, LED grid
    from {9, 13, 15} per side, defocus uniform in [-20, 20] um, 10..20 iterations.
    Returns a list of (arrival_s, Workload).
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_jobs))
    jobs = []
    for j in range(n_jobs):
        s = int(rng.choice([512, 1024, 1536, 2048]))
        m = int(rng.choice([64, 128, 256]))
        side = int(rng.choice([9, 13, 15]))
        iters = int(rng.integers(10, 21))
        w = Workload(f"job{j}", sensor=s, tile=m, tiles=s // m, overlap=16, iters=iters,
                     epry=True, optics=Optics(led_side=side), defocus_um=(-20.0, 20.0),
                     seed_offset=1000 * j)
        jobs.append((float(t[j]), w))
    return jobs
