"""Oracle reconstructions of several tiles at once, one host process per run.

Test infrastructure: the full-run parity tests recompute sampled tiles of the
largest jobs with the FP64 oracle (and the oracle's steps in complex64, the
float32 floor of tests/_fp32.py), which takes tens of seconds per tile, so the
runs go in parallel in processes started with "spawn" (safe to start after the
parent has used the GPU; the children import only numpy, the oracle and the
float32 restatement).
"""
from __future__ import annotations

import multiprocessing as mp
import os


def _run(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    kind, images, shifts, order, support, pupil0, n, iters, epry, mode = args
    if kind == "fp64":
        from oracle import fpm_oracle as orc
        return orc.reconstruct_tile(images, shifts, order, support, pupil0, n, iters, epry, mode=mode)
    from tests import _fp32
    return _fp32.reconstruct_tile32(images, shifts, order, support, pupil0, n, iters, epry, mode=mode)


def start(jobs, processes=None):
    """Start reconstructions; jobs = [(kind, images, shifts, order, support, pupil0,
    n, iters, epry, mode), ...] with kind "fp64" (the oracle) or "fp32" (its steps
    in complex64).  Returns (pool, AsyncResult); the result's get() is the list
    of (spectrum, pupil) in job order."""
    ctx = mp.get_context("spawn")
    n = processes or min(len(jobs), max(1, (os.cpu_count() or 2) - 1))
    pool = ctx.Pool(n)
    return pool, pool.map_async(_run, jobs, chunksize=1)


def finish(pool, res, timeout=3000):
    try:
        return res.get(timeout)
    finally:
        pool.close()
        pool.join()
