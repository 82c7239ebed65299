"""B300 (sm_103a) FPM tile reconstruction: C-ABI library libfpm + ctypes binding.

The binding is loaded on first use of any of its names; that import fails when
libfpm.so has not been built (there is no CPU fallback).  Build it with
``python -m paper_2203_02507_b300.build``.
"""
_NAMES = ("EXPORTED", "FpmError", "Plan", "Server", "plan_for", "update_tile_static", "reconstruct_batch", "fp32_peak",
          "LIB_PATH")


def __getattr__(name):
    if name in _NAMES:
        from . import _fpm
        return getattr(_fpm, name)
    raise AttributeError(name)
