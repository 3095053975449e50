"""FP64 CPU oracle for the 2DGS rasterizer -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg
may import this package.  It wraps `splat2d_oracle.c` (plain C, FP64), which
states the image-formation model of Sec. 3 (Eq. 1) with the 2DGS ray-splat
intersection and its analytic gradient; see that file's header for the
readings it takes.  Nothing here shares code with the CUDA library.

Pinning: every function here is checked by `tests/test_oracle_pins.py`
against closed forms, Eq. 1 in its screen-space form, an independent ray-
plane intersection, invariants and FP64 central differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splat2d_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libsplat2d_oracle.so")
_lock = threading.Lock()
_lib = None

NREC = 20
ST_VISIBLE, ST_OPACITY, ST_NEAR, ST_EMPTY, ST_INVALID = 0, 1, 2, 3, 4
SF_TILE_AMBIG, SF_NEAR_AMBIG, SF_PIX_AMBIG = 1, 2, 4
PF_ALPHA_MIN, PF_T_MIN, PF_RECT, PF_NEAR, PF_ALPHA_MAX, PF_BRANCH = 1, 2, 4, 8, 16, 32
# pixel flags that make a forward value legitimately differ between FP32 and FP64
PF_FORWARD = PF_ALPHA_MIN | PF_T_MIN | PF_RECT | PF_NEAR


def build(force: bool = False, openmp: bool = True) -> str:
    """Compile the oracle with gcc into oracle/_lib (no fused multiply-add
    contraction, so x86 and Arm give the same FP64 results)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        cmds = ([base[:1] + ["-fopenmp"] + base[1:]] if openmp else []) + [base]
        err = None
        for cmd in cmds:
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode == 0:
                os.replace(tmp, _LIB)
                return _LIB
            err = r.stderr
        raise RuntimeError(f"oracle build failed:\n{err}")


def _load():
    global _lib
    if _lib is None:
        path = build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.oracle_preprocess.argtypes = [i64] + [P] * 7 + [P] * 7
        lib.oracle_render.argtypes = [ctypes.c_int, i64] + [P] * 8 + [P] * 5
        lib.oracle_render_pixels.argtypes = [ctypes.c_int, i64] + [P] * 8 + [i64, P] + [P] * 4
        lib.oracle_render_bwd.argtypes = [ctypes.c_int, i64] + [P] * 9 + [i64, P, P, P]
        lib.oracle_render_dist.argtypes = [ctypes.c_int, i64] + [P] * 8 + [P]
        lib.oracle_chain.argtypes = [i64] + [P] * 12
        lib.oracle_render_pixels_variants.argtypes = ([ctypes.c_int, i64] + [P] * 8
                                                      + [ctypes.c_int, ctypes.c_int, i64, P, P])
        lib.oracle_max_error.argtypes = [ctypes.c_int, i64] + [P] * 8 + [P, P]
        lib.oracle_bin_sort.argtypes = [ctypes.c_int] + [P] * 9 + [i64]
        lib.oracle_bin_sort.restype = i64
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Config:
    """Rasterizer constants (readings: alpha clamp 0.99, skip 1/255, stop
    1e-4, low-pass sigma sqrt(1/2) px, near plane 0.01)."""
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    sigma_lp: float = 0.70710678118654752
    z_near: float = 0.01
    bg: tuple = (0.0, 0.0, 0.0)
    tile_w: int = 16
    tile_h: int = 16
    # how close (relative / in pixels) a decision must be to be reported ambiguous
    eps_alpha: float = 2e-5
    eps_t: float = 2e-5
    eps_px: float = 2e-5
    eps_z: float = 1e-5
    # depth output: False = the surfel center's depth (Eq. 1), True = the depth
    # of the ray-splat intersection where the object-space term decides
    depth_ray: bool = False
    # binned mode: which pixel rect decides whether a pair counts (0 = the
    # extent's; 1 / 2 = the widest / narrowest that rounding could give)
    rect_variant: int = 0

    def array(self) -> np.ndarray:
        f32 = lambda x: float(np.float32(x))  # the library receives FP32 constants
        return np.array([f32(self.alpha_min), f32(self.alpha_max), f32(self.t_min), f32(self.sigma_lp),
                         f32(self.z_near), f32(self.bg[0]), f32(self.bg[1]), f32(self.bg[2]),
                         self.tile_w, self.tile_h, self.eps_alpha, self.eps_t, self.eps_px, self.eps_z,
                         1.0 if self.depth_ray else 0.0, float(self.rect_variant)],
                        dtype=np.float64)


def cam_array(view) -> np.ndarray:
    Rt = np.asarray(view.Rt, np.float32).astype(np.float64)
    f32 = lambda x: float(np.float32(x))
    return np.concatenate([[view.width, view.height, f32(view.fx), f32(view.fy), f32(view.cx), f32(view.cy)],
                           Rt.reshape(-1)]).astype(np.float64)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


@dataclass
class Prep:
    rec: np.ndarray       # (n, 20) float64
    status: np.ndarray    # (n,) int32
    pixrect: np.ndarray   # (n, 4) int32 inclusive x0 y0 x1 y1
    tilerect: np.ndarray  # (n, 4) int32
    amb: np.ndarray       # (n, 8) int32 widest / narrowest pixel rect
    zbits: np.ndarray     # (n,) uint32
    sflags: np.ndarray    # (n,) uint32
    cam: np.ndarray
    cfg: np.ndarray


def preprocess(means, scales, quats, opacity, rgb, view, cfg: Config, cam: Optional[np.ndarray] = None) -> Prep:
    """Per-surfel records of one view.  `cam` (W, H, fx, fy, cx, cy, Rt[12])
    in FP64 overrides `view`, for finite differences of the pose."""
    lib = _load()
    means, scales, quats = _c(means, np.float32), _c(scales, np.float32), _c(quats, np.float32)
    opacity, rgb = _c(opacity, np.float32), _c(rgb, np.float32)
    n = means.shape[0]
    rec = np.zeros((n, NREC)); status = np.zeros(n, np.int32)
    pr = np.zeros((n, 4), np.int32); tr = np.zeros((n, 4), np.int32); amb = np.zeros((n, 8), np.int32)
    zb = np.zeros(n, np.uint32); sf = np.zeros(n, np.uint32)
    cam = cam_array(view) if cam is None else np.ascontiguousarray(cam, np.float64)
    cf = cfg.array()
    lib.oracle_preprocess(n, _p(means), _p(scales), _p(quats), _p(opacity), _p(rgb), _p(cam), _p(cf),
                          _p(rec), _p(status), _p(pr), _p(tr), _p(amb), _p(zb), _p(sf))
    return Prep(rec, status, pr, tr, amb, zb, sf, cam, cf)


def preprocess_scene_view(scene, v: int, cfg: Config) -> Prep:
    off, cnt = scene.view_ranges()[v]
    sl = slice(off, off + cnt)
    return preprocess(scene.means[sl], scene.scales[sl], scene.quats[sl], scene.opacity[sl],
                      scene.rgb[sl], scene.views[v], cfg)


@dataclass
class Image:
    out: np.ndarray     # (8, H, W): r, g, b, depth, nx, ny, nz, alpha
    tfinal: np.ndarray  # (H, W)
    nblend: np.ndarray  # (H, W)
    pflags: np.ndarray  # (H, W) uint32
    phash: np.ndarray   # (H, W) uint64 decision signature

    @property
    def rgb(self):
        return self.out[0:3]

    @property
    def depth(self):
        return self.out[3]

    @property
    def normal(self):
        return self.out[4:7]

    @property
    def alpha(self):
        return self.out[7]


def render(prep: Prep, mode: int = 1) -> Image:
    """mode 0: definition (every surfel at every pixel); mode 1: binned."""
    lib = _load()
    W, H = int(prep.cam[0]), int(prep.cam[1])
    n = prep.rec.shape[0]
    out = np.zeros((8, H, W)); tf = np.zeros((H, W)); nb = np.zeros((H, W), np.int32)
    pf = np.zeros((H, W), np.uint32); ph = np.zeros((H, W), np.uint64)
    lib.oracle_render(mode, n, _p(prep.rec), _p(prep.status), _p(prep.pixrect), _p(prep.amb), _p(prep.zbits),
                      _p(prep.sflags), _p(prep.cam), _p(prep.cfg), _p(out), _p(tf), _p(nb), _p(pf), _p(ph))
    return Image(out, tf, nb, pf, ph)


def render_pixels(prep: Prep, pix: np.ndarray, mode: int = 1):
    """Outputs (8, npix), tfinal, nblend, pflags at the listed flat pixel indices."""
    lib = _load()
    pix = _c(pix, np.int64)
    m = pix.shape[0]
    out = np.zeros((8, m)); tf = np.zeros(m); nb = np.zeros(m, np.int32); pf = np.zeros(m, np.uint32)
    lib.oracle_render_pixels(mode, prep.rec.shape[0], _p(prep.rec), _p(prep.status), _p(prep.pixrect),
                             _p(prep.amb), _p(prep.zbits), _p(prep.sflags), _p(prep.cam), _p(prep.cfg), m,
                             _p(pix), _p(out), _p(tf), _p(nb), _p(pf))
    return out, tf, nb, pf


def max_error(prep: Prep, err: np.ndarray, mode: int = 1, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Per surfel, the largest err[y, x] over the pixels that blend it
    (raised into `out` if given, else into zeros)."""
    lib = _load()
    W, H = int(prep.cam[0]), int(prep.cam[1])
    err = _c(np.broadcast_to(err, (H, W)), np.float64)
    n = prep.rec.shape[0]
    out = np.zeros(n) if out is None else out
    lib.oracle_max_error(mode, n, _p(prep.rec), _p(prep.status), _p(prep.pixrect), _p(prep.amb), _p(prep.zbits),
                         _p(prep.sflags), _p(prep.cam), _p(prep.cfg), _p(err), _p(out))
    return out


def accum_gate(alpha: np.ndarray, tau: float) -> np.ndarray:
    """Insertion gate of map fusion (Sec. 4.3, "Map Fusion"): new per-pixel
    primitives go only where the accumulated alpha rendered from the global
    map is below tau.  Ascending indices i with alpha[i] < tau (NaN never)."""
    a = np.asarray(alpha).reshape(-1)
    return np.nonzero(a < tau)[0]


@dataclass
class Grads:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacity: np.ndarray
    rgb: np.ndarray
    pose: np.ndarray  # (6,) d rho, d phi


def render_dist(prep: Prep, mode: int = 1) -> np.ndarray:
    """Depth distortion per pixel (H, W): 2 sum_i sum_{j<i} w_i w_j (z_i - z_j)
    over the pixel's blended entries in blending order."""
    lib = _load()
    W, H = int(prep.cam[0]), int(prep.cam[1])
    out = np.zeros((H, W))
    lib.oracle_render_dist(mode, prep.rec.shape[0], _p(prep.rec), _p(prep.status), _p(prep.pixrect), _p(prep.amb),
                           _p(prep.zbits), _p(prep.sflags), _p(prep.cam), _p(prep.cfg), _p(out))
    return out


def render_bwd(means, scales, quats, prep: Prep, g8: np.ndarray, mode: int = 1,
               pix: Optional[np.ndarray] = None, grads: Optional[Grads] = None,
               g_dist: Optional[np.ndarray] = None) -> Grads:
    """Gradients of sum(g8 * outputs) (+ sum(g_dist * distortion)) for one
    view; accumulated into `grads`."""
    lib = _load()
    means, scales, quats = _c(means, np.float32), _c(scales, np.float32), _c(quats, np.float32)
    n = prep.rec.shape[0]
    g8 = _c(g8, np.float64)
    gd = None if g_dist is None else _c(g_dist, np.float64)
    grec = np.zeros((n, NREC))
    if pix is None:
        lib.oracle_render_bwd(mode, n, _p(prep.rec), _p(prep.status), _p(prep.pixrect), _p(prep.amb),
                              _p(prep.zbits), _p(prep.sflags), _p(prep.cam), _p(prep.cfg), _p(g8), -1, None,
                              _p(grec), None if gd is None else _p(gd))
    else:
        pix = _c(pix, np.int64)
        lib.oracle_render_bwd(mode, n, _p(prep.rec), _p(prep.status), _p(prep.pixrect), _p(prep.amb),
                              _p(prep.zbits), _p(prep.sflags), _p(prep.cam), _p(prep.cfg), _p(g8),
                              pix.shape[0], _p(pix), _p(grec), None if gd is None else _p(gd))
    if grads is None:
        grads = Grads(np.zeros((n, 3)), np.zeros((n, 2)), np.zeros((n, 4)), np.zeros(n), np.zeros((n, 3)),
                      np.zeros(6))
    lib.oracle_chain(n, _p(means), _p(scales), _p(quats), _p(prep.status), _p(prep.cam), _p(grec),
                     _p(grads.means), _p(grads.scales), _p(grads.quats), _p(grads.opacity), _p(grads.rgb),
                     _p(grads.pose))
    grads.grec = grec
    return grads


def bin_sort(preps, tile_bases, tiles_x, surfel_offsets, cap: Optional[int] = None):
    """Keys and values of every view's instances, stably sorted by key."""
    lib = _load()
    counts = np.array([p.rec.shape[0] for p in preps], np.int64)
    status = np.concatenate([p.status for p in preps]).astype(np.int32)
    tr = np.concatenate([p.tilerect for p in preps]).astype(np.int32)
    zb = np.concatenate([p.zbits for p in preps]).astype(np.uint32)
    sidx = np.concatenate([np.arange(c, dtype=np.int64) + o for c, o in zip(counts, surfel_offsets)])
    tb = np.asarray(tile_bases, np.int64)
    tx = np.asarray(tiles_x, np.int32)
    need = lib.oracle_bin_sort(len(preps), _p(counts), _p(status), _p(tr), _p(zb), _p(sidx), _p(tb), _p(tx),
                               None, None, 0)
    keys = np.zeros(max(need, 1), np.uint64)
    vals = np.zeros(max(need, 1), np.uint32)
    lib.oracle_bin_sort(len(preps), _p(counts), _p(status), _p(tr), _p(zb), _p(sidx), _p(tb), _p(tx),
                        _p(keys), _p(vals), need)
    return keys[:need], vals[:need]


def render_pixels_either_side(prep: Prep, pix: np.ndarray, mode: int = 1) -> np.ndarray:
    """Outputs (k, 8, npix) at the listed pixels under every combination of
    the outcomes of the decisions this oracle reports as within rounding:
    alpha_min and t_min moved just past their flag margins either way (so a
    pair whose alpha, or a stop whose transmittance, is within the margin is
    decided the other way), and the pixel rect of the extent, the widest or
    the narrowest that rounding could give.  A result computed at lower
    precision that took some of these decisions the other way should match
    one of the k outputs; k = 27 (the unmodified result is among them)."""
    lib = _load()
    base = np.asarray(prep.cfg, np.float64)
    ea, et = base[10], base[11]
    rows = []
    for sa in (0, -1, 1):
        for st in (0, -1, 1):
            for rv in (0, 1, 2):
                c = base.copy()
                c[0] = base[0] * (1.0 + 1.25 * sa * ea)
                c[2] = base[2] * (1.0 + 1.25 * st * et)
                c[15] = rv
                rows.append(c)
    cfgs = np.ascontiguousarray(np.stack(rows))
    pix = _c(pix, np.int64)
    out = np.zeros((len(rows), 8, pix.shape[0]))
    if pix.shape[0]:
        lib.oracle_render_pixels_variants(mode, prep.rec.shape[0], _p(prep.rec), _p(prep.status),
                                          _p(prep.pixrect), _p(prep.amb), _p(prep.zbits), _p(prep.sflags),
                                          _p(prep.cam), _p(cfgs), cfgs.shape[0], cfgs.shape[1], pix.shape[0],
                                          _p(pix), _p(out))
    return out
