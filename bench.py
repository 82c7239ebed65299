#!/usr/bin/env python
"""Benchmark of the FPM tile-reconstruction hot path on B300.

A step is one full-FOV reconstruction: the initial guess of every tile
(fpm_load_tiles) plus all iteration loops of the per-LED update with the wave
schedule (fpm_reconstruct, replayed as a CUDA graph).  The headline workload is
the 2048 x 2048 sensor cut into 8 x 8 tiles of 256 x 256 (HR 1024 x 1024),
15 x 15 LEDs, 20 loops with EPRY pupil correction: 288,000 LED sub-aperture
updates per step.  Inputs (1.9 GB image stack, 0.5 GB spectra) are larger than
L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
the host cores instead (a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "LED sub-aperture updates/sec and ms per FOV; p50/p99 job latency vs plain path"
UNIT = "updates/s"
E2E_IN_FLIGHT = 3      # FOVs in flight in the end-to-end measurement (plans on their own streams)
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 148, 128, 2.032
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3      # 76.98 TFLOP/s

# DRAM bytes per update ((mode, m, threads per CTA, CTAs per cluster) -> bytes)
# of the dominant kernel, from the latest ncu capture in profiles/ of the kernel
# as it stands; a launch scales it by the updates it processes.  Emptied
# whenever the kernel changes until re-captured.
TRAFFIC_PER_UPDATE = {
    # profiles/update_kernel_m256_4cta256_ncu_full.md: 12,634,880 + 0 B for 32 updates
    ("waves", 256, 256, 4): (12634880 + 0) / 32,
    # profiles/persistent_kernel_m256_ncu_full.md: 553,616,128 + 94,384,896 B for 3,600 updates
    ("persistent", 256, 256, 4): (553616128 + 94384896) / 3600,
}

EXTRA = {
    # many small tiles: 16 x 16 tiles of 64 on a 1024^2 sensor, 15 x 15 LEDs, 10 loops, EPRY
    "fov1024_m64": synth.Workload("fov1024_m64", sensor=1024, tile=64, tiles=16, overlap=0, iters=10, epry=True,
                                  optics=synth.Optics(led_side=15), defocus_um=(-20.0, 20.0)),
    # small cases of the same kernels for ncu captures (inputs larger than L2, well under a few GB)
    "ncu_m256": synth.Workload("ncu_m256", sensor=768, tile=256, tiles=3, overlap=16, iters=1, epry=True,
                               optics=synth.Optics(led_side=15), defocus_um=(-20.0, 20.0)),
    "ncu16_m256": synth.Workload("ncu16_m256", sensor=1024, tile=256, tiles=4, overlap=16, iters=1, epry=True,
                                 optics=synth.Optics(led_side=15), defocus_um=(-20.0, 20.0)),
    # the 5120^2 job's kernel on 8 x 8 tiles of 128, 21 x 21 LEDs, one loop (925 MB of images)
    "ncu64_m128": synth.Workload("ncu64_m128", sensor=1024, tile=128, tiles=8, overlap=0, iters=1, epry=True,
                                 optics=synth.Optics(led_side=21), defocus_um=(-30.0, 30.0)),
}


def workload(name):
    return synth.WORKLOADS.get(name) or EXTRA[name]


def support_px(w):
    m, o = w.tile, w.optics
    df = 1.0 / (m * o.pixel_um)
    k = np.arange(m) - m // 2
    fy, fx = np.meshgrid(k * df, k * df, indexing="ij")
    return int((np.sqrt(fx * fx + fy * fy) <= o.na / o.wavelength_um).sum())


def flops_per_update(w):
    """Algorithmic FLOPs of one update: two m x m 2-D FFTs at 5 n log2 n (n = m^2),
    10 flop per pixel for the amplitude step, and 18 (fixed pupil) or 36 (EPRY)
    flop per support pixel for the box products and the corrections."""
    m = w.tile
    a = support_px(w)
    return 2 * 5 * m * m * math.log2(m * m) + 10 * m * m + (36 if w.epry else 18) * a


def bytes_per_update(w):
    """Algorithmic HBM bytes of one update: the LR image once, the spectrum's
    support disc read and written (16 B/px), the pupil disc read (8 B/px) and,
    with EPRY, its correction written (8 B/px)."""
    m = w.tile
    a = support_px(w)
    img = 2 if w.image_dtype == "u16" else 4
    return img * m * m + 16 * a + (16 if w.epry else 8) * a


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# synthetic data on the device
# ---------------------------------------------------------------------------

def gpu_objects(torch, dev, n, tiles, seed, sigma=2.0):
    """HR objects made on the GPU with the recipe's statistics: seeded N(0,1) fields,
    periodic Gaussian smoothing (sigma = 2 HR px, applied in the Fourier domain),
    min-max mapped to amplitude [0.5, 1] and phase [-pi/2, pi/2].  Used for the
    large auxiliary workloads, where drawing every tile on the host would dominate."""
    g = torch.Generator(device=dev).manual_seed(seed)
    f = torch.fft.fftfreq(n, device=dev)
    gauss = torch.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    out = torch.empty((tiles, n, n), dtype=torch.complex64, device=dev)
    for t in range(tiles):
        a, p = (torch.fft.ifft2(torch.fft.fft2(torch.randn((n, n), generator=g, device=dev)) * gauss).real
                for _ in range(2))
        a = 0.5 + 0.5 * (a - a.min()) / (a.max() - a.min())
        p = ((p - p.min()) / (p.max() - p.min()) - 0.5) * math.pi
        out[t] = torch.polar(a, p)
    return out


def device_stack(plan, w, torch, dev, fast=False):
    """Sensor stack [L, S, S] of 12-bit counts (int16 bits) simulated on the GPU."""
    t_n, n, m, l_n = w.n_tiles, w.hr, w.tile, w.n_leds
    if fast:
        objs = gpu_objects(torch, dev, n, t_n, 1 + w.seed_offset)
    else:
        objs = torch.empty((t_n, n, n), dtype=torch.complex64, device=dev)
        for t in range(t_n):
            objs[t].copy_(torch.from_numpy(synth.hr_object(n, t, w.seed_offset).astype(np.complex64)))
    imgs = torch.empty((t_n, l_n, m, m), dtype=torch.float32, device=dev)
    plan.simulate(objs, imgs)
    del objs
    if w.image_dtype == "f32":
        stack = torch.zeros((l_n, w.sensor, w.sensor), dtype=torch.float32, device=dev)
        k = 1.0
        counts = imgs
    else:
        g = torch.Generator(device=dev).manual_seed(synth.workloads.SEED_NOISE + w.seed_offset)
        k = float(w.peak_counts / imgs.max().item())
        counts = torch.poisson(imgs * k, generator=g)
        counts += torch.randn(counts.shape, generator=g, device=dev) * w.read_sigma
        counts = counts.round_().clamp_(0, 4095).to(torch.int16)
        stack = torch.zeros((l_n, w.sensor, w.sensor), dtype=torch.int16, device=dev)
    origins = plan.schedule()["origins"]
    win = synth.owner_windows(origins, m, w.sensor)
    for t in range(t_n):
        y0, x0 = (int(v) for v in origins[t])
        ylo, yhi, xlo, xhi = (int(v) for v in win[t])
        stack[:, y0 + ylo:y0 + yhi, x0 + xlo:x0 + xhi] = counts[t, :, ylo:yhi, xlo:xhi]
    del imgs, counts
    torch.cuda.synchronize()
    return stack, k


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure; only this leg of bench.py uses it)
# ---------------------------------------------------------------------------

def _oracle_worker(args):
    name, tile, iters = args
    from oracle import fpm_oracle as orc
    if iters == 0:                      # pool warm-up: imports only
        return 0.0, 0
    w = workload(name)
    o = w.optics
    leds = synth.led_grid(o.led_side, o.led_pitch_um)
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    g = orc.geometry(w.sensor, w.sensor, w.tile, w.overlap, w.tiles, w.tiles, w.upsample, o.wavelength_um, o.na,
                     o.pixel_um, leds, o.led_height_um, dz)
    imgs = orc.forward_images(orc.fft2c(synth.hr_object(w.hr, tile, w.seed_offset)), g.pupils[tile],
                              g.shifts[tile], w.tile)
    t0 = time.perf_counter()
    orc.reconstruct_tile(imgs, g.shifts[tile], g.order, g.support, g.pupils[tile], g.n, iters, w.epry)
    return time.perf_counter() - t0, iters * w.n_leds


def cpu_baseline(name, tiles=1, iters=1, procs=1):
    """Oracle updates/s on host cores: `procs` processes, one tile each (the paper's
    one-sub-region-per-CPU strategy), `iters` loops."""
    jobs = [(name, t, iters) for t in range(tiles)]
    if procs == 1:
        res = [_oracle_worker(j) for j in jobs]
        wall = sum(r[0] for r in res)
    else:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        with ctx.Pool(procs) as pool:
            pool.map(_oracle_worker, [(name, 0, 0)] * procs)          # import warm-up
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, jobs)
            wall = time.perf_counter() - t0
    upd = sum(r[1] for r in res)
    return upd / wall, upd, wall


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload)
    procs = max(1, min(os.cpu_count() or 1, w.n_tiles, 32))
    times, ups = [], 0
    for s in range(args.warmup + args.steps):
        v, upd, wall = cpu_baseline(args.workload, tiles=procs, iters=1, procs=procs)
        if s >= args.warmup:
            times.append(wall)
            ups = upd
    value = ups / statistics.mean(times)
    sample = f"{procs} tiles x 1 loop ({ups} updates) per step, one process per tile"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * w.updates / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sensor": w.sensor, "tile": w.tile, "tiles": w.n_tiles,
                       "leds": w.n_leds, "iters": w.iters, "epry": w.epry},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def aggregate(ms_local, updates_local, dist=None, device=None):
    """Whole-job result of N independent replicas: the slowest rank's time and the
    units all ranks processed.  Returns (ms, total_updates, updates_per_s)."""
    import torch
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        u = torch.tensor([updates_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms_local, updates_local = float(t.item()), float(u.item())
    return ms_local, updates_local, updates_local / (ms_local / 1e3)


def shard_gather_and_stitch(plan, w, stack, k, by_rank, rank, world, dist, torch, stream):
    """After a sharded run (Sec. 5): every rank sends its tiles' spectra and pupils
    to rank 0 (point-to-point), which writes them into a plan of the whole grid
    and stitches the field of view (Eq. 1).  Returns the timings on rank 0."""
    from paper_2203_02507_b300 import plan_for, shard
    first, count = by_rank[rank]
    specs = np.zeros((count, w.hr, w.hr), np.complex64)
    pups = np.zeros((count, w.tile, w.tile), np.complex64)
    for i in range(count):
        specs[i] = plan.spectrum(i)
        pups[i] = plan.pupil(i)
    t0 = time.perf_counter()
    all_s = shard.gather_tiles(specs, first, w.n_tiles, by_rank, rank, dist)
    all_p = shard.gather_tiles(pups, first, w.n_tiles, by_rank, rank, dist)
    gather_s = time.perf_counter() - t0
    if rank != 0:
        return None
    q = plan_for(w)
    q.load_tiles(stack, k)
    for t in range(w.n_tiles):
        q.set_state(t, all_s[t], all_p[t])
    fov = torch.empty((q.info["fov_h"], q.info["fov_w"]), dtype=torch.complex64, device=stack.device)
    q.stitch(fov)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    q.stitch(fov)
    e1.record(stream)
    torch.cuda.synchronize()
    q.close()
    return {"ranks": world, "tiles_by_rank": by_rank, "gather_s": gather_s,
            "gather_bytes": int(w.n_tiles * (w.hr * w.hr + w.tile * w.tile) * 8),
            "stitch_ms": e0.elapsed_time(e1),
            "how": "tile states (spectrum + pupil) copied to the host and sent to rank 0 point to point "
                   "after the timed steps; rank 0 writes them into a whole-grid plan and stitches"}


# ---------------------------------------------------------------------------
# batched and served forms
# ---------------------------------------------------------------------------

def hbm_peak_gbs():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json, copy bandwidth)"
    except (OSError, KeyError, ValueError):
        return 6400.0, "fallback"


def sequential_timing(torch, stack, k, w, steps=2):
    """Strict-sequential EPRY (FPM_SEQUENTIAL: one LED per tile per wave) on the same FOV,
    the whole job per step as in the headline, both execution paths."""
    from paper_2203_02507_b300 import plan_for
    p = plan_for(w, sequential=True)
    s = torch.cuda.current_stream()
    out = {"waves_per_tile": p.info["max_waves"], "updates_per_step": w.updates}
    for mode in ("waves", "persistent"):
        p.load_tiles(stack, k)
        p.reconstruct(w.iters, mode=mode, graph=True)          # warm-up (graph capture)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            p.load_tiles(stack, k)
            p.reconstruct(w.iters, mode=mode, graph=True)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[mode] = {"updates_per_s": w.updates / (ms / 1e3), "ms_per_step": ms}
    p.close()
    return out


def unmasked_timing(torch, stack, k, w, steps=2):
    """Non-masked EPRY (FPM_EPRY_UNMASKED: corrections and footprints over the whole
    box) on the same FOV, the whole job per step, wave by wave with 8 graph branches
    (the persistent kernel cannot hold the whole box at m = 256)."""
    from paper_2203_02507_b300 import plan_for
    prev = os.environ.get("FPM_WAVE_BRANCHES")
    os.environ["FPM_WAVE_BRANCHES"] = "8"
    p = plan_for(w, unmasked=True)
    p.load_tiles(stack, k)
    if prev is None:
        del os.environ["FPM_WAVE_BRANCHES"]
    else:
        os.environ["FPM_WAVE_BRANCHES"] = prev
    s = torch.cuda.current_stream()
    out = {"waves_per_tile": p.info["max_waves"], "updates_per_step": w.updates, "mode": "waves+graph, 8 branches",
           "threads": p.info["threads"], "cluster": p.info["cluster"]}
    p.reconstruct(w.iters, mode="waves", graph=True)          # warm-up (graph capture)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        p.load_tiles(stack, k)
        p.reconstruct(w.iters, mode="waves", graph=True)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out.update({"updates_per_s": w.updates / (ms / 1e3), "ms_per_step": ms})
    p.close()
    return out


def online_timing(plan, torch, host_stack, k, w):
    """Online ingestion (Sec. 3.4): the FOV's images pushed one at a time from page-locked
    host memory in the LED order, as fast as the host issues them.  Per image: device
    time from its push to the end of the work it released (copy wait, gather, ready
    wave steps); tail: the remaining loops after the last image."""
    order = plan.schedule()["order"]
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in order]
    end = torch.cuda.Event(enable_timing=True)
    for warm in (True, False):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.online_begin(w.iters, dtype="u16", counts_per_unit=k)
        before_last = 0
        for i, led in enumerate(order):
            if i == len(order) - 1:
                before_last = plan.stats(check=False)["online_launched"]
            ev[i][0].record(s)
            plan.online_push(int(led), host_stack[int(led)])
            ev[i][1].record(s)
        plan.online_finish()
        end.record(s)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    per = sorted(a.elapsed_time(b) for a, b in ev[:-1])          # images before the last one
    total_steps = plan.stats(check=False)["online_steps"]
    return {"images": len(order), "per_image_ms_p50": per[len(per) // 2],
            "per_image_ms_p99": per[int(0.99 * (len(per) - 1))], "per_image_ms_max": per[-1],
            "last_image_to_done_ms": ev[-1][0].elapsed_time(end),
            "device_ms_first_push_to_done": ev[0][0].elapsed_time(end), "wall_ms": wall * 1e3,
            "steps_launched_before_last_image": before_last, "steps": total_steps,
            "updates_per_s": w.updates / (ev[0][0].elapsed_time(end) / 1e3),
            "how": "page-locked host images pushed in LED order without pacing; per image: device time of the "
                   "work its push released (copy wait, gather, ready wave steps); the schedule is the offline "
                   "one, so the result equals it bit for bit (tests/test_gpu_online.py)"}


def stitch_timing(plan, torch, dev, stack, k, w, reps=3):
    """fpm_stitch of the reconstructed FOV into a device image (Eq. 1): device time and
    bandwidth on its algorithmic bytes (every spectrum read once, the image written once)."""
    plan.load_tiles(stack, k)
    plan.reconstruct(1, mode="waves", graph=True)
    info = plan.info
    out = torch.empty((info["fov_h"], info["fov_w"]), dtype=torch.complex64, device=dev)
    plan.stitch(out=out)                                   # warm-up
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan.stitch(out=out)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nbytes = w.n_tiles * w.hr * w.hr * 8 + info["fov_h"] * info["fov_w"] * 8
    peak, src = hbm_peak_gbs()
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"ms": ms, "fov": [info["fov_h"], info["fov_w"]], "hr_overlap": info["hr_overlap"],
            "algorithmic_bytes": nbytes, "gbs": gbs, "hbm_peak_gbs": peak, "frac": gbs / peak, "peak_source": src,
            "includes": "one tile column at a time: row transforms of its spectra (with each row's band values), "
                        "its band sums and Eq. 1 weights on the device, column transforms writing weight x object "
                        "straight into the image; two row buffers, so the next column's row transforms run "
                        "while this column's weights and column transforms run on a second stream; scratch "
                        "kept with the plan"}


def uneven_batch(torch, dev, steps=3):
    """Three jobs (128/192/256 tiles, 9x9/13x13/15x15 LEDs, 15 loops, EPRY) run together
    each step: one persistent launch over all their updates, and every job an independent
    graph branch (its tiles in 4 branches); returns updates/s and ms per step of both."""
    from paper_2203_02507_b300 import plan_for, reconstruct_batch
    ws = [synth.WORKLOADS[k] for k in ("batch_m128", "batch_m192", "batch_m256")]
    prev = os.environ.get("FPM_WAVE_BRANCHES")
    os.environ["FPM_WAVE_BRANCHES"] = "4"
    plans, stacks = [], []
    for w in ws:
        p = plan_for(w)
        st, k = device_stack(p, w, torch, dev, fast=True)
        p.load_tiles(st, k)
        plans.append(p)
        stacks.append((st, k))
    if prev is None:
        del os.environ["FPM_WAVE_BRANCHES"]
    else:
        os.environ["FPM_WAVE_BRANCHES"] = prev
    upd = sum(w.updates for w in ws)
    out = {"updates_per_step": upd, "steps": steps, "jobs": [w.name for w in ws]}
    for mode in ("persistent", "waves"):
        def step():
            for p, (st, k) in zip(plans, stacks):
                p.load_tiles(st, k)
            reconstruct_batch(plans, [w.iters for w in ws], graph=True, mode=mode)

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        for p in plans:
            assert p.stats()["device_error"] == 0
        out[mode] = {"value": upd / (ms / 1e3), "unit": UNIT, "ms_per_step": ms}
    for p in plans:
        p.close()
    out["value"] = out["persistent"]["value"]
    out["mode"] = ("value: one persistent launch per step (graph); waves: every job a graph branch "
                   "with its tiles in 4 branches")
    return out


def config_extra(name, torch, dev, peak, steps=2, tune_iters=2):
    """Another configuration of the benchmark set, measured like the headline: the
    path the autotuner picks on `tune_iters` loops of the job's own data, then the
    whole job (load + initial guess + all loops) timed with CUDA events, and the
    update kernel's per-launch roofline from one more, per-launch-timed step."""
    from paper_2203_02507_b300 import plan_for
    w = synth.WORKLOADS[name]
    plan = plan_for(w)
    stack, k = device_stack(plan, w, torch, dev, fast=w.n_tiles > 64)
    plan.load_tiles(stack, k)
    entries, best = plan.autotune(iters=tune_iters)
    mode = entries[best]["mode"]

    def step():
        plan.load_tiles(stack, k)
        plan.reconstruct(w.iters, mode=mode, graph=True)

    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    assert plan.stats()["device_error"] == 0
    out = {"value": w.updates / (ms / 1e3), "unit": UNIT, "ms_per_job": ms, "steps": steps,
           "updates_per_job": w.updates, "mode": mode + "+graph", "tuned": entries[best],
           "config": {"sensor": w.sensor, "tile": w.tile, "tiles": w.n_tiles, "leds": w.n_leds, "iters": w.iters,
                      "epry": w.epry, "image": w.image_dtype}}
    # per-launch roofline of the update kernel (wave launches of the tuned variant, one branch)
    plan.load_tiles(stack, k)
    plan.reconstruct(w.iters, mode="waves", graph=True, timed=True)
    torch.cuda.synchronize()
    st = plan.stats()
    t_l = st["update_ms"] / 1e3 / st["update_launches"]
    u_l = st["updates"] / st["update_launches"]
    fpu = flops_per_update(w)
    out["roofline"] = {"bound": "alu", "achieved": fpu * u_l / t_l / 1e12, "peak": peak, "unit": "TFLOP/s",
                       "frac": fpu * u_l / t_l / 1e12 / peak, "avg_launch_us": t_l * 1e6,
                       "updates_per_launch": u_l, "flop_per_update": fpu,
                       "kernel_variant": {"threads": st["run_threads"], "cluster": st["run_cluster"]},
                       "job_frac": fpu * w.updates / (ms / 1e3) / 1e12 / peak}
    plan.close()
    del stack
    torch.cuda.synchronize()
    return out


def plain_rate(torch, dev, w):
    """Updates/s of the plain path (one tile at a time, one LED per launch) on one loop of `w`."""
    from paper_2203_02507_b300 import plan_for
    p = plan_for(w, iters=1)
    st, k = device_stack(p, w, torch, dev, fast=True)
    p.load_tiles(st, k)
    p.reconstruct(1, mode="waves")
    p.load_tiles(st, k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.reconstruct(1, mode="plain")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    p.close()
    return w.n_tiles * w.n_leds / dt


def serving(torch, dev, n_jobs, budget=120 << 30):
    """The first n_jobs of the serving stream (Poisson arrivals at 2 jobs/s) through
    the server in real time; latency = submit -> done."""
    from paper_2203_02507_b300 import Server, plan_for
    stream = synth.serving_jobs(500)[:n_jobs]
    prepared = []
    for arrival, w in stream:
        p = plan_for(w)
        st, k = device_stack(p, w, torch, dev, fast=True)
        prepared.append((arrival, w, p, st, k))
    torch.cuda.synchronize()
    srv = Server(budget)
    ids = []
    t0 = time.perf_counter()
    for arrival, w, p, st, k in prepared:
        while time.perf_counter() - t0 < arrival:
            time.sleep(0.0005)
        ids.append(srv.submit(p, w.iters, stack=st, counts_per_unit=k))
    while True:
        states = [srv.poll(i) for i in ids]
        if all(s[0] in ("done", "failed") for s in states):
            break
        time.sleep(0.002)
    t_end = time.perf_counter() - t0
    srv.close()
    assert all(s[0] == "done" for s in states), states
    lat = np.array([s[2] for s in states])
    upd = sum(w.updates for _, w, _, _, _ in prepared)
    # throughput: completed updates over the time the server had admitted work on
    # the GPU (union of every job's admit -> done interval)
    spans = sorted((arrival + s[1], arrival + s[2]) for (arrival, *_), s in zip(prepared, states))
    busy, cur0, cur1 = 0.0, None, None
    for a0, a1 in spans:
        if cur1 is None or a0 > cur1:
            if cur1 is not None:
                busy += cur1 - cur0
            cur0, cur1 = a0, a1
        else:
            cur1 = max(cur1, a1)
    if cur1 is not None:
        busy += cur1 - cur0
    # plain path, same arrivals: one job at a time (FIFO), each at the plain rate measured for its tile size
    rates = {}
    for m in sorted({w.tile for _, w, _, _, _ in prepared}):
        rates[m] = plain_rate(torch, dev, synth.Workload(f"plain{m}", sensor=4 * m, tile=m, tiles=4, overlap=0,
                                                         iters=1, epry=True, optics=synth.Optics(led_side=15)))
    free_at, plain_lat = 0.0, []
    for arrival, w, _, _, _ in prepared:
        start = max(arrival, free_at)
        free_at = start + w.updates / rates[w.tile]
        plain_lat.append(free_at - arrival)
    for _, _, p, _, _ in prepared:
        p.close()
    plain_lat = np.array(plain_lat)
    return {"jobs": n_jobs, "arrivals": "Poisson 2 jobs/s (first jobs of the 500-job stream)",
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "updates_per_s": upd / busy, "updates": upd, "wall_s": t_end,
            "busy_s": busy, "offered_updates_per_s": upd / t_end,
            "throughput_how": "completed updates / GPU-busy time (union of the jobs' admit -> done intervals); "
                              "offered_updates_per_s = updates / wall time of the arrival stream",
            "plain_path_model": {"p50_s": float(np.percentile(plain_lat, 50)),
                                 "p99_s": float(np.percentile(plain_lat, 99)),
                                 "plain_updates_per_s_by_tile": {str(k): v for k, v in rates.items()},
                                 "how": "FIFO, one job at a time at the plain path's measured per-tile-size rate"},
            "budget_gb": budget / (1 << 30)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fov2048_m256")
    ap.add_argument("--mode", default="auto", choices=["auto", "waves", "persistent"],
                    help="auto: fpm_autotune picks the fastest path on one loop of the data")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, plain path and CPU baseline")
    ap.add_argument("--serving-jobs", type=int, default=40, help="jobs of the serving sample (0 to skip)")
    ap.add_argument("--shard", action="store_true",
                    help="split one FOV's tiles over the ranks by cost (strong scaling, Sec. 5) and gather the "
                         "tile states on rank 0 for stitching, instead of one FOV replica per rank")
    ap.add_argument("--only", choices=["stitch", "online", "sequential", "unmasked"],
                    help="time only this part on the workload (profiling aid) and print its JSON")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2203_02507_b300 import plan_for

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload(args.workload)

    plan = plan_for(w)
    stack, k = device_stack(plan, w, torch, dev)
    stream = torch.cuda.current_stream()
    units_local = w.updates
    shard_range = None
    if args.shard:
        # this rank's contiguous share of the FOV's tiles, balanced by m^2 L iters (all
        # tiles cost the same here); the stack stays whole, each tile reads its window
        from paper_2203_02507_b300 import shard
        ranges = shard.job_ranges([(w.n_tiles, w.tile, w.n_leds, w.iters)], world)
        shard_by_rank = [(rr[0][1], rr[0][2]) if rr else (0, 0) for rr in ranges]
        shard_range = shard_by_rank[rank]
        plan.close()
        plan = plan_for(w, tile_first=shard_range[0], tile_count=max(shard_range[1], 1))
        units_local = shard_range[1] * w.n_leds * w.iters
        args.no_extras = True
    if args.only:
        if args.only == "stitch":
            part = stitch_timing(plan, torch, dev, stack, k, w)
        elif args.only == "sequential":
            part = sequential_timing(torch, stack, k, w)
        elif args.only == "unmasked":
            part = unmasked_timing(torch, stack, k, w)
        else:
            host_stack = torch.empty(stack.shape, dtype=stack.dtype, pin_memory=True)
            host_stack.copy_(stack)
            part = online_timing(plan, torch, host_stack, k, w)
        print(json.dumps({"part": args.only, "workload": w.name, args.only: part}))
        return
    tune = None
    if args.mode == "auto":
        plan.load_tiles(stack, k)
        entries, best = plan.autotune(iters=w.iters)     # the whole job, as timed below
        tune = {"entries": entries, "best": best}
        args.mode = entries[best]["mode"]

    # one step = initial guess of every tile + all loops of the update
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(i=None, timed=False):
        plan.load_tiles(stack, k)
        if i is not None:
            ev[i][0].record(stream)
        if args.mode == "persistent":
            plan.reconstruct(w.iters, mode="persistent", graph=True)
        else:
            plan.reconstruct(w.iters, mode="waves", graph=True, timed=timed)
        if i is not None:
            ev[i][1].record(stream)

    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    from paper_2203_02507_b300 import fp32_peak
    peak = fp32_peak()          # measured FP32 FFMA throughput of this device, this run (roofline denominator)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    run_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    st_timed = plan.stats()          # launch counts of the timed steps' configuration
    instr_ms = None
    if args.mode != "persistent":
        # per-launch events around each of the step's ~900 update launches cost ~6% of
        # the step (and run the wave steps as one branch), so they are recorded in one
        # more step after the timed region
        l0, i0, i1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        l0.record(stream)
        plan.load_tiles(stack, k)
        i0.record(stream)
        plan.reconstruct(w.iters, mode="waves", graph=True, timed=True)
        i1.record(stream)
        torch.cuda.synchronize()
        instr_ms = i0.elapsed_time(i1)
        load_ms = l0.elapsed_time(i0)
    st = plan.stats()
    ms, _, value = aggregate(ms, units_local * args.steps, dist if world > 1 else None, dev)
    ms_per_step = ms / args.steps
    launches = (st_timed["load_launches"] + st_timed["run_launches"]) * args.steps

    # roofline of the dominant kernel, from the CUDA events of the timed region
    fpu, bpu = flops_per_update(w), bytes_per_update(w)
    if args.mode == "persistent":
        per_launch_s, upl, kname, n_launch = run_ms / 1e3, w.updates, "fpm::persistent_kernel", 1
        share = run_ms / ms_per_step
        kernel_timing = "CUDA events around the persistent launch of every timed step"
    else:
        per_launch_s = st["update_ms"] / 1e3 / st["update_launches"]
        upl, kname, n_launch = st["updates"] / st["update_launches"], "fpm::update_kernel", st["update_launches"]
        share = st["update_ms"] / (st["update_ms"] + st["merge_ms"] + load_ms)
        kernel_timing = ("CUDA events around each update launch of one more step (one graph branch) run right "
                         "after the timed region; share = update time / (update + merge + load time) of that step, "
                         "the serialised kernel-time share an ncu launch list gives")
    kkey = (args.mode, w.tile, st["run_threads"], st["run_cluster"])     # the kernel variant that ran
    achieved = fpu * upl / per_launch_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (TRAFFIC_PER_UPDATE[kkey] * upl if kkey in TRAFFIC_PER_UPDATE else None),
            "traffic_source": "ncu dram__bytes_read+write per update on a 16-tile case (profiles/), "
                              "scaled by this launch's updates",
            "kernel": kname, "kernel_variant": {"threads": st["run_threads"], "cluster": st["run_cluster"]},
            "launches_per_step": n_launch, "updates_per_launch": upl,
            "avg_launch_us": per_launch_s * 1e6, "flop_per_update": fpu, "hbm_bytes_per_update": bpu,
            "hbm_gbs_algorithmic": bpu * upl / per_launch_s / 1e9, "kernel_share_of_step": share,
            "peak_source": "measured: fpm_fp32_peak (chains of FFMA on every FP32 lane, this device, this run)",
            "peak_nominal": FP32_PEAK_TFLOPS, "kernel_timing": kernel_timing,
            "job_achieved": fpu * units_local / (run_ms / 1e3) / 1e12,
            "job_frac": fpu * units_local / (run_ms / 1e3) / 1e12 / peak,
            "job_timing": "the job's algorithmic work over the timed steps' reconstruction time (CUDA events "
                          "around fpm_reconstruct; for wave launches with graph branches the kernels of "
                          "different tile groups overlap)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 1), "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "sensor": w.sensor, "tile": w.tile, "hr": w.hr, "tiles": w.n_tiles,
                       "leds": w.n_leds, "iters": w.iters, "epry": w.epry, "updates_per_step": w.updates,
                       "mode": args.mode + "+graph", "ms_per_fov": ms_per_step, "autotune": tune,
                       "graph_branches": (tune["entries"][tune["best"]]["branches"] if tune
                                          else int(os.environ.get("FPM_WAVE_BRANCHES", "1"))),
                       "clusters": st["persistent_clusters"] if args.mode == "persistent" else None,
                       "l2": "inputs larger than L2 (1.9 GB stack, 0.5 GB spectra); no flush",
                       "parallelism": f"{world} independent FOV replicas" if world > 1 else "1 GPU"},
            "roofline": roof, "gpu_launches": launches, "clocks": clk,
            "step_parts": {"reconstruct_ms": run_ms, "load_ms": ms_per_step - run_ms,
                           "how": "CUDA events around fpm_reconstruct in every timed step; load = the rest of "
                                  "the step (fpm_load_tiles: tile-image gather and initial guess)"}}

    if args.shard:
        line["scaling"] = "strong"
        line["config"]["parallelism"] = f"{world} GPU(s), the FOV's {w.n_tiles} tiles split by cost"
        line["shard"] = shard_gather_and_stitch(plan, w, stack, k, shard_by_rank, rank, world,
                                                dist if world > 1 else None, torch, stream)
    if not args.no_extras and rank == 0:
        # e2e through the public API with host buffers: per FOV the H2D of its stack (page-locked),
        # the whole job, and the D2H of every spectrum
        host_stack = torch.empty(stack.shape, dtype=stack.dtype, pin_memory=True)
        host_stack.copy_(stack)
        host_out = [torch.empty((w.n_tiles, w.hr, w.hr), dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        k_e2e = max(2, args.steps)       # FOVs per plan; the stream fills and drains once over all of them
        # one FOV at a time
        plan.load_tiles(host_stack, k)
        plan.reconstruct(w.iters, mode=args.mode, graph=True)
        plan.spectra(host_out[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            plan.load_tiles(host_stack, k)
            plan.reconstruct(w.iters, mode=args.mode, graph=True)
            plan.spectra(host_out[0])
            torch.cuda.synchronize()
        serial_s = (time.perf_counter() - t0) / k_e2e
        # E2E_IN_FLIGHT FOVs in flight: as many plans on as many streams, so some FOVs' copies
        # overlap the others' compute
        extra = [plan_for(w) for _ in range(E2E_IN_FLIGHT - 1)]
        plans = [plan] + extra
        streams = [torch.cuda.Stream() for _ in plans]
        while len(host_out) < len(plans):
            host_out.append(torch.empty((w.n_tiles, w.hr, w.hr), dtype=torch.complex64, pin_memory=True))
        # the other plans run the timed plan's kernel variant and branch count (read when their
        # device state is made, at the first load)
        env = {"FPM_WAVE_BRANCHES": str(line["config"]["graph_branches"])}
        if tune:
            best = tune["entries"][tune["best"]]
            env["FPM_UPDATE_THREADS"] = f"{best['threads']}x{best['cluster']}"
        prev_env = {key: os.environ.get(key) for key in env}
        os.environ.update(env)
        for q in extra:
            q.load_tiles(stack, k)
        for key, v in prev_env.items():
            if v is None:
                del os.environ[key]
            else:
                os.environ[key] = v
        torch.cuda.synchronize()
        for j in range(len(plans)):
            plans[j].load_tiles(host_stack, k, stream=streams[j])
            plans[j].reconstruct(w.iters, mode=args.mode, graph=True, stream=streams[j])
            plans[j].spectra(host_out[j], stream=streams[j])
        torch.cuda.synchronize()
        n_fov = len(plans) * k_e2e
        t0 = time.perf_counter()
        for i in range(n_fov):
            j = i % len(plans)
            plans[j].load_tiles(host_stack, k, stream=streams[j])
            plans[j].reconstruct(w.iters, mode=args.mode, graph=True, stream=streams[j])
            plans[j].spectra(host_out[j], stream=streams[j])
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / n_fov
        for q in extra:
            q.close()
        line["e2e"] = {"value": w.updates / e2e_s, "unit": UNIT,
                       "h2d_bytes_per_step": int(host_stack.numel() * host_stack.element_size()),
                       "d2h_bytes_per_step": int(host_out[0].numel() * host_out[0].element_size()),
                       "ms_per_step": e2e_s * 1e3, "steps": n_fov,
                       "how": f"{E2E_IN_FLIGHT} plans on {E2E_IN_FLIGHT} streams, {E2E_IN_FLIGHT} FOVs in flight: "
                              "every FOV's H2D, whole job and D2H in the timed region, copies overlapping the "
                              "other FOVs' compute",
                       "serial": {"value": w.updates / serial_s, "ms_per_step": serial_s * 1e3, "steps": k_e2e}}
        # plain path: one tile at a time, one LED per launch (bounded: one loop)
        plan.load_tiles(stack, k)
        plan.reconstruct(1, mode="waves")          # builds the one-loop schedule lists
        plan.load_tiles(stack, k)
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        plan.reconstruct(1, mode="plain")
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - p0
        plain_upd = w.n_tiles * w.n_leds
        line["plain_path"] = {"value": plain_upd / plain_s, "unit": UNIT,
                              "sample": f"one loop of all {w.n_tiles} tiles ({plain_upd} updates), no graph",
                              "speedup_of_batched": value / (plain_upd / plain_s)}
        # the same FOV step in the other execution mode
        other = "waves" if args.mode == "persistent" else "persistent"
        plan.load_tiles(stack, k)
        plan.reconstruct(w.iters, mode=other, graph=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            plan.load_tiles(stack, k)
            plan.reconstruct(w.iters, mode=other, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / args.steps
        alt = {"value": w.updates / (pms / 1e3), "unit": UNIT, "ms_per_step": pms}
        if other == "waves":
            plan.load_tiles(stack, k)                  # per-launch events: one more, untimed step
            plan.reconstruct(w.iters, mode="waves", graph=True, timed=True)
            torch.cuda.synchronize()
            s2 = plan.stats()
            t_l = s2["update_ms"] / 1e3 / s2["update_launches"]
            u_l = s2["updates"] / s2["update_launches"]
            alt["update_kernel"] = {"avg_launch_us": t_l * 1e6, "updates_per_launch": u_l,
                                    "achieved_tflops": fpu * u_l / t_l / 1e12,
                                    "frac": fpu * u_l / t_l / 1e12 / peak,
                                    "share_of_step": s2["update_ms"] / pms}
        line[other + "_path"] = alt
        line["online"] = online_timing(plan, torch, host_stack, k, w)
        del host_stack, host_out
        line["sequential_epry"] = sequential_timing(torch, stack, k, w)
        line["unmasked_epry"] = unmasked_timing(torch, stack, k, w)
        line["stitch"] = stitch_timing(plan, torch, dev, stack, k, w)
        line["uneven_batch"] = uneven_batch(torch, dev)
        for extra_name in ("tile64_plain", "fov5120_m128"):
            line[extra_name] = config_extra(extra_name, torch, dev, peak)
        if args.serving_jobs > 0:
            line["serving"] = serving(torch, dev, args.serving_jobs)
        if world == 1:
            v, upd, wall = cpu_baseline(w.name, tiles=1, iters=4, procs=1)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"1 tile x 4 loops ({upd} updates, {wall:.1f} s), FP64 numpy"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
