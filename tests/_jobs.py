"""Test jobs: seeded synthetic inputs simulated by the FP64 oracle, and the
parity metrics used to compare the CUDA path with the oracle."""
from __future__ import annotations

import numpy as np

import synth
from oracle import fpm_oracle as orc


class Job:
    """A synthetic job: oracle geometry, ground truth and the sensor stack."""

    def __init__(self, w: synth.Workload, tiles_sim=None):
        self.w = w
        o = w.optics
        self.leds = synth.led_grid(o.led_side, o.led_pitch_um)
        self.defocus = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
        self.g = orc.geometry(w.sensor, w.sensor, w.tile, w.overlap, w.tiles, w.tiles, w.upsample,
                              o.wavelength_um, o.na, o.pixel_um, self.leds, o.led_height_um, self.defocus)
        m = w.tile
        imgs = np.zeros((w.n_tiles, w.n_leds, m, m))
        for t in range(w.n_tiles):
            spec = orc.fft2c(synth.hr_object(w.hr, t, w.seed_offset))
            imgs[t] = orc.forward_images(spec, self.g.pupils[t], self.g.shifts[t], m)
        if w.image_dtype == "u16":
            counts, k = synth.add_noise(imgs, w.peak_counts, w.read_sigma, w.seed_offset)
            self.stack = synth.assemble_sensor(counts, self.g.origins, w.sensor)
            self.counts_per_unit = k
        else:
            self.stack = synth.assemble_sensor(imgs.astype(np.float32), self.g.origins, w.sensor)
            self.counts_per_unit = 1.0

    def tile_images(self, t):
        return orc.tile_images_from_stack(self.stack, self.g.origins[t], self.w.tile, self.counts_per_unit)

    def oracle_tile(self, t, iters, mode="waves"):
        return orc.reconstruct_tile(self.tile_images(t), self.g.shifts[t], self.g.order, self.g.support,
                                    self.g.pupils[t], self.g.n, iters, self.w.epry, mode=mode)

    def plan(self, iters=None):
        from paper_2203_02507_b300 import plan_for
        return plan_for(self.w, defocus_um=self.defocus, iters=iters or self.w.iters)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def object_errors(spec_gpu, spec_ref):
    """(amplitude rel-L2, phase error) of the objects o = ifft2c(O).

    Phase error: RMS of the wrapped phase difference over pixels with
    |o_ref| > 0.1 max|o_ref|, divided by the RMS of the reference phase there.
    """
    og = orc.object_from_spectrum(spec_gpu.astype(np.complex128))
    orf = orc.object_from_spectrum(spec_ref)
    amp = rel_l2(np.abs(og), np.abs(orf))
    mask = np.abs(orf) > 0.1 * np.abs(orf).max()
    d = np.angle(og[mask] * np.conj(orf[mask]))
    ph = float(np.sqrt(np.mean(d ** 2)) / np.sqrt(np.mean(np.angle(orf[mask]) ** 2)))
    return amp, ph
