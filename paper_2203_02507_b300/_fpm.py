"""ctypes binding of libfpm (include/fpm.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
Python/numpy/torch arguments to the C ABI and raises on a non-zero status.
Importing it fails loudly when the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfpm.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"libfpm.so not built at {LIB_PATH}: run `python -m paper_2203_02507_b300.build`")
_lib = C.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, EBUDGET, ETIMEOUT, ECUDA, EBUSY, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
ORDER = {"center_out": 0, "raster": 1}
EPRY = 1
SEQUENTIAL = 2
EPRY_UNMASKED = 4
U16, F32 = 0, 1
RUN = {"plain": 0, "waves": 1, "persistent": 2, "auto": 3}
RUN_GRAPH = 0x100
RUN_TIMED = 0x200
RUN_FAULT_TEST = 0x400
JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}
TUNE_MAX_ENTRIES = 64    # FPM_TUNE_MAX_ENTRIES


class FpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fpm status {code}: {msg}")
        self.code = code


class PlanDesc(C.Structure):
    _fields_ = [
        ("sensor_h", C.c_int32), ("sensor_w", C.c_int32),
        ("tile", C.c_int32), ("overlap", C.c_int32),
        ("tiles_y", C.c_int32), ("tiles_x", C.c_int32),
        ("upsample", C.c_int32),
        ("wavelength_um", C.c_double), ("na", C.c_double), ("pixel_um", C.c_double),
        ("n_leds", C.c_int32), ("led_xy_um", C.POINTER(C.c_double)),
        ("led_height_um", C.c_double),
        ("defocus_um", C.POINTER(C.c_double)),
        ("order", C.c_int32), ("iters", C.c_int32), ("flags", C.c_uint32),
        ("tile_first", C.c_int32), ("tile_count", C.c_int32),
    ]


class PlanInfo(C.Structure):
    _fields_ = [
        ("m", C.c_int32), ("n", C.c_int32), ("n_tiles", C.c_int32), ("n_leds", C.c_int32),
        ("iters", C.c_int32), ("support_px", C.c_int32), ("support_rows", C.c_int32),
        ("max_waves", C.c_int32), ("max_wave_width", C.c_int32), ("total_waves", C.c_int64),
        ("device_bytes", C.c_int64), ("cluster", C.c_int32), ("threads", C.c_int32),
        ("image_elems", C.c_int64), ("hr_overlap", C.c_int32), ("fov_h", C.c_int32), ("fov_w", C.c_int32),
        ("tile_first", C.c_int32), ("band", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneEntry(C.Structure):
    _fields_ = [("mode", C.c_int32), ("threads", C.c_int32), ("cluster", C.c_int32), ("branches", C.c_int32),
                ("ms", C.c_double), ("lanes", C.c_int32), ("radix_a", C.c_int32), ("radix_b", C.c_int32),
                ("pad0", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("load_launches", C.c_int64), ("run_launches", C.c_int64), ("update_launches", C.c_int64),
                ("updates", C.c_int64), ("update_ms", C.c_double), ("device_error", C.c_int32),
                ("persistent_clusters", C.c_int32), ("run_threads", C.c_int32), ("online_launched", C.c_int32),
                ("online_steps", C.c_int32), ("run_cluster", C.c_int32), ("merge_ms", C.c_double),
                ("run_lanes", C.c_int32), ("pad0", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _i32, _i64, _f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
_SIGS = {
    "fpm_plan_create": [C.POINTER(PlanDesc), C.POINTER(_vp)],
    "fpm_plan_destroy": [_vp],
    "fpm_plan_get_info": [_vp, C.POINTER(PlanInfo)],
    "fpm_get_schedule": [_vp, _vp, _vp, _vp, _vp],
    "fpm_load_tiles": [_vp, _vp, _i32, _i32, _i64, _i64, _f32, _vp],
    "fpm_reconstruct": [_vp, _i32, _i32, _vp],
    "fpm_get_spectrum": [_vp, _i32, _vp, _i32, _vp],
    "fpm_get_pupil": [_vp, _i32, _vp, _i32, _vp],
    "fpm_set_state": [_vp, _i32, _vp, _vp, _vp],
    "fpm_initial_pupil": [_vp, _i32, _vp],
    "fpm_get_stats": [_vp, C.POINTER(Stats)],
    "fpm_autotune": [_vp, _i32, _vp, C.POINTER(TuneEntry), _i32, C.POINTER(_i32), C.POINTER(_i32)],
    "fpm_simulate": [_vp, _vp, _vp, _vp],
    "fpm_server_create": [C.c_size_t, C.POINTER(_vp)],
    "fpm_submit": [_vp, _vp, _i32, _vp, _i32, _i32, _i64, _i64, _f32, C.POINTER(_i64)],
    "fpm_poll": [_vp, _i64, C.POINTER(_i32), C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "fpm_server_destroy": [_vp],
    "fpm_reconstruct_batch": [C.POINTER(_vp), C.POINTER(_i32), _i32, _i32, _vp],
    "fpm_update_tile_static": [_vp, _i32, _vp, _i32, _vp, _i32, _i32, C.c_double, C.c_double, C.c_double, _i32, _vp],
    "fpm_fp32_peak": [C.POINTER(C.c_double), _vp],
    "fpm_get_object": [_vp, _i32, _vp, _i32, _vp],
    "fpm_stitch": [_vp, _vp, _i32, _vp],
    "fpm_online_begin": [_vp, _i32, _i32, _f32, _vp],
    "fpm_online_push": [_vp, _i32, _vp, _i32, _i64, _vp],
    "fpm_online_finish": [_vp, _vp],
    "fpm_get_spectra": [_vp, _vp, _i32, _vp],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.fpm_last_error.argtypes = []
_lib.fpm_last_error.restype = C.c_char_p

EXPORTED = sorted(list(_SIGS) + ["fpm_last_error"])


def _check(rc: int):
    if rc != OK:
        raise FpmError(rc, _lib.fpm_last_error().decode())


def _ptr(x):
    """Raw address of a numpy array or torch tensor (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Plan:
    """An FPM job: geometry, schedule, and (after load_tiles) device state."""

    def __init__(self, *, sensor, tile, overlap, tiles, upsample, wavelength_um, na, pixel_um,
                 led_xy_um, led_height_um, defocus_um=None, order="center_out", iters=1, epry=False,
                 sequential=False, unmasked=False, tile_first=0, tile_count=0):
        sh, sw = (sensor, sensor) if np.isscalar(sensor) else sensor
        ty, tx = (tiles, tiles) if np.isscalar(tiles) else tiles
        self._leds = np.ascontiguousarray(led_xy_um, dtype=np.float64).reshape(-1, 2)
        self._defocus = None if defocus_um is None else np.ascontiguousarray(defocus_um, dtype=np.float64)
        d = PlanDesc()
        d.sensor_h, d.sensor_w = int(sh), int(sw)
        d.tile, d.overlap, d.tiles_y, d.tiles_x = int(tile), int(overlap), int(ty), int(tx)
        d.upsample = int(upsample)
        d.wavelength_um, d.na, d.pixel_um = float(wavelength_um), float(na), float(pixel_um)
        d.n_leds = len(self._leds)
        d.led_xy_um = self._leds.ctypes.data_as(C.POINTER(C.c_double))
        d.led_height_um = float(led_height_um)
        d.defocus_um = (self._defocus.ctypes.data_as(C.POINTER(C.c_double))
                        if self._defocus is not None else None)
        d.order = ORDER[order]
        d.iters = int(iters)
        d.flags = (EPRY if epry else 0) | (SEQUENTIAL if sequential else 0) | (EPRY_UNMASKED if unmasked else 0)
        d.tile_first, d.tile_count = int(tile_first), int(tile_count)
        h = _vp()
        _check(_lib.fpm_plan_create(C.byref(d), C.byref(h)))
        self._h = h
        info = PlanInfo()
        _check(_lib.fpm_plan_get_info(self._h, C.byref(info)))
        self.info = info.as_dict()
        self.m, self.n = info.m, info.n
        self.n_tiles, self.n_leds, self.iters = info.n_tiles, info.n_leds, info.iters
        self.epry = bool(epry)
        self.tile_first = info.tile_first
        self._stack_ref = None

    # -- host-only queries -------------------------------------------------
    def schedule(self):
        order = np.zeros(self.n_leds, np.int32)
        shifts = np.zeros((self.n_tiles, self.n_leds, 2), np.int32)
        waves = np.zeros((self.n_tiles, self.iters * self.n_leds), np.int32)
        origins = np.zeros((self.n_tiles, 2), np.int32)
        _check(_lib.fpm_get_schedule(self._h, _ptr(order), _ptr(shifts), _ptr(waves), _ptr(origins)))
        return {"order": order, "shifts": shifts, "waves": waves, "origins": origins}

    def initial_pupil(self, tile: int) -> np.ndarray:
        out = np.zeros((self.m, self.m), np.complex64)
        _check(_lib.fpm_initial_pupil(self._h, int(tile), _ptr(out)))
        return out

    # -- device work --------------------------------------------------------
    def load_tiles(self, stack, counts_per_unit: float = 1.0, stream=None):
        """stack: [L, H, W] uint16/int16 (12-bit counts) or float32, numpy (host) or torch (device)."""
        dt = str(stack.dtype)
        if dt.endswith("uint16") or dt.endswith("int16"):
            code = U16
        elif dt.endswith("float32"):
            code = F32
        else:
            raise TypeError(f"stack dtype {dt} not supported (uint16 or float32)")
        l_n, h, w = stack.shape
        on_dev = 1 if _is_device(stack) else 0
        _check(_lib.fpm_load_tiles(self._h, _ptr(stack), code, on_dev, int(h * w), int(w),
                                   float(counts_per_unit), _stream(stream)))
        self._stack_ref = stack if on_dev else None   # borrowed device memory stays alive

    def reconstruct(self, iters: int | None = None, mode: str = "waves", graph: bool = False, timed: bool = False,
                    stream=None, fault_test: bool = False):
        flag = (RUN[mode] | (RUN_GRAPH if graph else 0) | (RUN_TIMED if timed else 0)
                | (RUN_FAULT_TEST if fault_test else 0))
        _check(_lib.fpm_reconstruct(self._h, int(iters or self.iters), flag, _stream(stream)))

    def autotune(self, iters: int | None = None, stream=None):
        """Time every execution path on `iters` loops (default: the plan's loop count)
        of the loaded data and keep the fastest (for mode="auto"); returns
        ([{mode, threads, cluster, ms}], best index)."""
        iters = self.info["iters"] if iters is None else iters
        ent = (TuneEntry * TUNE_MAX_ENTRIES)()
        n, best = _i32(), _i32()
        _check(_lib.fpm_autotune(self._h, int(iters), _stream(stream), ent, TUNE_MAX_ENTRIES, C.byref(n),
                                 C.byref(best)))
        names = {v: k for k, v in RUN.items()}
        out = [{"mode": names[e.mode], "threads": e.threads, "cluster": e.cluster, "branches": e.branches,
                "lanes": e.lanes, "split": (e.radix_a, e.radix_b), "ms": e.ms} for e in ent[:n.value]]
        return out, best.value

    def stats(self, check: bool = True) -> dict:
        st = Stats()
        rc = _lib.fpm_get_stats(self._h, C.byref(st))
        if check:
            _check(rc)
        return st.as_dict()

    def spectrum(self, tile: int, out=None, stream=None):
        if out is None:
            out = np.zeros((self.n, self.n), np.complex64)
        _check(_lib.fpm_get_spectrum(self._h, int(tile), _ptr(out), 1 if _is_device(out) else 0, _stream(stream)))
        return out

    def spectra(self, out, stream=None):
        """All tiles' spectra into `out` ([T, N, N] complex64, host or device), one copy
        enqueued on the stream and not waited for (fpm_get_spectra)."""
        _check(_lib.fpm_get_spectra(self._h, _ptr(out), 1 if _is_device(out) else 0, _stream(stream)))
        return out

    def pupil(self, tile: int, out=None, stream=None):
        if out is None:
            out = np.zeros((self.m, self.m), np.complex64)
        _check(_lib.fpm_get_pupil(self._h, int(tile), _ptr(out), 1 if _is_device(out) else 0, _stream(stream)))
        return out

    # -- online ingestion (images one at a time) ---------------------------
    def online_begin(self, iters=None, dtype="u16", counts_per_unit=1.0, stream=None):
        iters = self.iters if iters is None else iters
        _check(_lib.fpm_online_begin(self._h, int(iters), U16 if dtype == "u16" else F32, float(counts_per_unit),
                                     _stream(stream)))

    def online_push(self, led: int, image, stream=None):
        """image: [sensor_h, sensor_w] (rows may be strided) uint16/int16 or float32,
        numpy (host) or torch (host or device)."""
        if hasattr(image, "stride"):
            stride_row = image.stride()[0] if callable(image.stride) else image.strides[0] // image.itemsize
        else:
            stride_row = image.strides[0] // image.itemsize
        if hasattr(image, "data_ptr"):
            ptr = image.data_ptr()
        else:
            if not image.flags.c_contiguous and image.strides[1] != image.itemsize:
                raise ValueError("image rows must be contiguous")
            ptr = image.ctypes.data
        _check(_lib.fpm_online_push(self._h, int(led), ptr, 1 if _is_device(image) else 0, int(stride_row),
                                    _stream(stream)))

    def online_finish(self, stream=None):
        _check(_lib.fpm_online_finish(self._h, _stream(stream)))

    def object(self, tile: int, out=None, stream=None):
        """The tile's HR complex object (fpm_get_object)."""
        if out is None:
            out = np.zeros((self.n, self.n), np.complex64)
        _check(_lib.fpm_get_object(self._h, int(tile), _ptr(out), 1 if _is_device(out) else 0, _stream(stream)))
        return out

    def stitch(self, out=None, stream=None):
        """The whole field of view as one HR complex image (fpm_stitch, Eq. 1)."""
        if out is None:
            out = np.zeros((self.info["fov_h"], self.info["fov_w"]), np.complex64)
        _check(_lib.fpm_stitch(self._h, _ptr(out), 1 if _is_device(out) else 0, _stream(stream)))
        return out

    def set_state(self, tile: int, spectrum=None, pupil=None, stream=None):
        s = None if spectrum is None else np.ascontiguousarray(spectrum, np.complex64)
        p = None if pupil is None else np.ascontiguousarray(pupil, np.complex64)
        _check(_lib.fpm_set_state(self._h, int(tile), _ptr(s), _ptr(p), _stream(stream)))

    def simulate(self, objects, out, stream=None):
        """objects: device complex64 [T, N, N]; out: device float32 [T, L, m, m]."""
        _check(_lib.fpm_simulate(self._h, _ptr(objects), _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.fpm_plan_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server for many plans (fpm_server_*)."""

    def __init__(self, hbm_budget_bytes: int):
        h = _vp()
        _check(_lib.fpm_server_create(int(hbm_budget_bytes), C.byref(h)))
        self._h = h

    def submit(self, plan: Plan, iters: int | None = None, stack=None, counts_per_unit: float = 1.0) -> int:
        """Queue a job.  With `stack` ([L, H, W] uint16/float32, host or device) the
        server loads the images at admission; keep `stack` alive until the job ends."""
        job = _i64()
        if stack is None:
            args = (None, 0, 0, 0, 0, 1.0)
        else:
            code = F32 if str(stack.dtype).endswith("float32") else U16
            l_n, h, w = stack.shape
            args = (_ptr(stack), code, 1 if _is_device(stack) else 0, int(h * w), int(w), float(counts_per_unit))
            plan._stack_ref = stack
        _check(_lib.fpm_submit(self._h, plan._h, int(iters or plan.iters), *args, C.byref(job)))
        return job.value

    def poll(self, job: int):
        st, w, lat = _i32(), C.c_double(), C.c_double()
        _check(_lib.fpm_poll(self._h, int(job), C.byref(st), C.byref(w), C.byref(lat)))
        return JOB_STATES[st.value], w.value, lat.value

    def close(self):
        if getattr(self, "_h", None):
            _check(_lib.fpm_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_batch(plans, iters=None, graph: bool = False, stream=None, mode: str = "persistent"):
    """Run several loaded plans together (fpm_reconstruct_batch): mode "persistent" (one
    persistent launch over all their updates) or "waves" (each plan an independent branch)."""
    n = len(plans)
    hs = (_vp * n)(*[p._h.value for p in plans])
    its = (_i32 * n)(*[int(i) for i in (iters or [p.iters for p in plans])])
    _check(_lib.fpm_reconstruct_batch(hs, its, n, RUN[mode] | (RUN_GRAPH if graph else 0), _stream(stream)))


def update_tile_static(spectrum, pupil, image, shift, wavelength_um, na, pixel_um, epry, stream=None):
    """One LED update of one tile with no device allocation (fpm_update_tile_static).

    spectrum: device complex64 [N, N]; pupil: device complex64 [m, m]; image:
    device float32 [m, m]; shift: (sy, sx).  Updates spectrum (and pupil if
    epry) in place, stream-ordered.  The C call cannot see the tensors' sizes,
    so they are checked here: every argument must be a contiguous CUDA tensor of
    the stated type and square shape, all three on one device; ValueError
    otherwise, before anything reaches the library.
    """
    for name, t, dt in (("spectrum", spectrum, "complex64"), ("pupil", pupil, "complex64"),
                        ("image", image, "float32")):
        if not hasattr(t, "is_cuda") or str(t.dtype) != f"torch.{dt}":
            raise ValueError(f"{name} must be a torch {dt} tensor, got {getattr(t, 'dtype', type(t))}")
        if t.dim() != 2 or t.shape[0] != t.shape[1]:
            raise ValueError(f"{name} must be square [side, side], got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if not _is_device(t):
            raise ValueError(f"{name} must be a CUDA tensor")
    n, m = int(spectrum.shape[0]), int(pupil.shape[0])
    if tuple(image.shape) != (m, m):
        raise ValueError(f"image must be [{m}, {m}] like the pupil, got {tuple(image.shape)}")
    if not (spectrum.device == pupil.device == image.device):
        raise ValueError("spectrum, pupil and image must be on one device")
    _check(_lib.fpm_update_tile_static(_ptr(spectrum), n, _ptr(pupil), m, _ptr(image), int(shift[0]),
                                       int(shift[1]), float(wavelength_um), float(na), float(pixel_um),
                                       1 if epry else 0, _stream(stream)))


def fp32_peak(stream=None) -> float:
    """Measured FP32 throughput of the current device in TFLOP/s (fpm_fp32_peak)."""
    v = C.c_double(0.0)
    _check(_lib.fpm_fp32_peak(C.byref(v), _stream(stream)))
    return v.value


def plan_for(workload, defocus_um=None, iters=None, sequential=False, order="center_out",
             unmasked=False, tile_first=0, tile_count=0) -> Plan:
    """Plan of a synth.Workload (square sensor and grid)."""
    from synth import led_grid, tile_defocus
    o = workload.optics
    if defocus_um is None:
        lo, hi = workload.defocus_um
        defocus_um = tile_defocus(workload.n_tiles, lo, hi, workload.seed_offset)
    return Plan(sensor=workload.sensor, tile=workload.tile, overlap=workload.overlap, tiles=workload.tiles,
                upsample=workload.upsample, wavelength_um=o.wavelength_um, na=o.na, pixel_um=o.pixel_um,
                led_xy_um=led_grid(o.led_side, o.led_pitch_um), led_height_um=o.led_height_um,
                defocus_um=defocus_um, iters=iters or workload.iters, epry=workload.epry, sequential=sequential,
                order=order, unmasked=unmasked, tile_first=tile_first, tile_count=tile_count)
