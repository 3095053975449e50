"""ctypes mirror of include/splat2d.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

c_int32, c_int64, c_float, c_uint32, c_size_t, c_void_p = (
    ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_void_p)

OK = 0
ERR_INVALID_ARG = -1
ERR_WORKSPACE_TOO_SMALL = -2
ERR_CUDA = -3
ERR_CAPACITY = -4
ERR_TIMEOUT = -5
ERR_NO_DEVICE = -6
ERR_BOUNDS = -7
FLAG_NO_STATS = 1
FLAG_DEPTH_RAY = 2
SORT_NOALLOC_MAX_PAIRS = 1 << 20


class View(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("Rt", c_float * 12), ("surfel_offset", c_int64), ("surfel_count", c_int64),
                ("pixel_offset", c_int64)]


class Surfels(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacity", c_void_p),
                ("rgb", c_void_p), ("n", c_int64)]


class Grads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacity", c_void_p),
                ("rgb", c_void_p), ("pose", c_void_p)]


class Config(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("chunk", c_int32), ("alpha_min", c_float),
                ("alpha_max", c_float), ("t_min", c_float), ("lowpass_sigma", c_float), ("z_near", c_float),
                ("bg", c_float * 3), ("flags", c_uint32), ("bwd_chunk", c_int32)]


class SurfelBuffers(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p), ("opacity", c_void_p),
                ("rgb", c_void_p)]


class Problem(ctypes.Structure):
    _fields_ = [("views", ctypes.POINTER(View)), ("n_views", c_int32), ("n_surfels", c_int64),
                ("instance_capacity", c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("status", c_int64), ("needed_capacity", c_int64), ("n_instances", c_int64),
                ("n_visible", c_int64), ("fwd_pairs_evaluated", c_int64), ("fwd_pairs_blended", c_int64),
                ("bwd_pairs_evaluated", c_int64), ("bwd_pairs_blended", c_int64), ("sort_passes", c_int64),
                ("bwd_terms_outside", c_int64), ("reserved", c_int64 * 6)]


class Layout(ctypes.Structure):
    _fields_ = [("records", c_size_t), ("ntiles", c_size_t), ("keys", c_size_t), ("vals", c_size_t),
                ("ranges", c_size_t), ("tfinal", c_size_t), ("last", c_size_t), ("total", c_size_t),
                ("n_records", c_int64), ("n_tiles", c_int64), ("n_pixels", c_int64)]


# every symbol include/splat2d.h declares, with its ctypes signature
SIGNATURES = {
    "splat2d_default_config": (None, [ctypes.POINTER(Config)]),
    "splat2d_workspace_size": (c_size_t, [ctypes.POINTER(Config), ctypes.POINTER(Problem)]),
    "splat2d_preprocess": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), ctypes.POINTER(Surfels),
                                          c_void_p, c_size_t, c_void_p]),
    "splat2d_bin_sort": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p, c_size_t,
                                        c_void_p]),
    "splat2d_render_fwd": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p, c_size_t,
                                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "splat2d_render_bwd": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), ctypes.POINTER(Surfels),
                                          c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p,
                                          ctypes.POINTER(Grads), c_void_p]),
    "splat2d_render_bwd_tiles": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p,
                                                c_size_t, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "splat2d_render_fwd_dist": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p, c_size_t,
                                               c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "splat2d_render_bwd_dist": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem),
                                               ctypes.POINTER(Surfels), c_void_p, c_size_t, c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p, ctypes.POINTER(Grads), c_void_p]),
    "splat2d_render_bwd_tiles_dist": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p,
                                                     c_size_t, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                                     c_void_p]),
    "splat2d_preprocess_bwd": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem),
                                              ctypes.POINTER(Surfels), c_void_p, c_size_t, ctypes.POINTER(Grads),
                                              c_void_p]),
    "splat2d_max_error": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem), c_void_p, c_size_t,
                                         c_void_p, c_void_p, c_void_p]),
    "splat2d_accum_gate_tmp_size": (c_size_t, [c_int64]),
    "splat2d_accum_gate": (ctypes.c_int, [c_void_p, c_int64, ctypes.c_float, c_void_p, c_void_p, c_void_p, c_size_t,
                                          c_void_p]),
    "splat2d_voxelize_tmp_size": (c_size_t, [ctypes.c_int32, ctypes.c_int32]),
    "splat2d_voxelize": (ctypes.c_int, [ctypes.POINTER(Surfels), ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                        ctypes.POINTER(SurfelBuffers), c_void_p, c_void_p, c_void_p, c_size_t,
                                        c_void_p]),
    "splat2d_sim3_apply": (ctypes.c_int, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "splat2d_launch_count": (ctypes.c_uint64, []),
    "splat2d_stats": (ctypes.c_int, [c_void_p, ctypes.POINTER(Stats), c_void_p]),
    "splat2d_status": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64), c_void_p]),
    "splat2d_workspace_layout": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Problem),
                                                ctypes.POINTER(Layout)]),
    "splat2d_sort_tmp_size": (c_size_t, [c_int64]),
    "splat2d_sort_pairs": (ctypes.c_int, [c_void_p, c_void_p, c_int64, ctypes.c_int, c_void_p, c_size_t,
                                          c_void_p]),
    "splat2d_sort_pairs_noalloc": (ctypes.c_int, [c_void_p, c_void_p, c_int64, ctypes.c_int, c_void_p]),
    "splat2d_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True):
    """Load libsplat2d (building it first if needed).  Raises if it cannot
    be built or loaded: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libsplat2d not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def strerror(code: int) -> str:
    return load().splat2d_strerror(int(code)).decode()


class Splat2DError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


def check(code: int, what: str = ""):
    if code != OK:
        raise Splat2DError(code, what)
