"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package draws random numbers and lays out geometry descriptions; it holds
none of the reconstruction's arithmetic (no Fourier transforms, pupils, shifts or
updates).  Both the FP64 oracle and the CUDA path consume what it produces.
"""
from .workloads import (  # noqa: F401
    Optics, Workload, WORKLOADS, led_grid, hr_object, tile_defocus, add_noise,
    assemble_sensor, owner_windows, serving_jobs,
)
