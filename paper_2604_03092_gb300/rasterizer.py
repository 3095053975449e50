"""Python binding of libsplat2d: argument marshalling around the C ABI.

Every step of the rasterizer runs in the CUDA library; this module only
turns torch tensors into device pointers, owns the workspace tensor and
wraps the backward in a `torch.autograd.Function`.  There is no fallback:
if the library cannot be loaded, or a tensor is not on a CUDA device, the
calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import List, NamedTuple, Optional, Sequence

import torch

from . import _abi

__all__ = ["RasterConfig", "Rasterizer", "Images", "SurfelGrads", "Splat2DRender", "Splat2DRenderDist", "render",
           "accum_gate"]


@dataclasses.dataclass
class RasterConfig:
    """Constants of the rasterizer (see splat2d_config in include/splat2d.h)."""

    tile_w: int = 8
    tile_h: int = 8
    chunk: int = 128
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    lowpass_sigma: float = math.sqrt(0.5)
    z_near: float = 0.01
    bg: tuple = (0.0, 0.0, 0.0)
    stats: bool = True
    fwd_tail: int = 0  # 0: default; 255: forward always shares pixels across warps
    bwd_chunk: int = 64  # 0: same as chunk
    depth_ray: bool = False  # depth output from the ray-splat intersection (SPLAT2D_FLAG_DEPTH_RAY)

    @classmethod
    def for_problem(cls, views: Sequence, n_surfels: int, **kw) -> "RasterConfig":
        """The default constants with the launch shape the autotuner keeps
        for this problem's bucket (the user's cache, else the shipped GB300
        measurement, else the defaults)."""
        from . import autotune
        cfg = cls(**kw)
        tuned = autotune.lookup(views, n_surfels)
        if tuned:
            cfg.tile_w, cfg.tile_h, cfg.chunk, cfg.bwd_chunk = tuned
        return cfg

    def to_c(self) -> _abi.Config:
        c = _abi.Config()
        c.tile_w, c.tile_h, c.chunk = int(self.tile_w), int(self.tile_h), int(self.chunk)
        c.alpha_min, c.alpha_max, c.t_min = self.alpha_min, self.alpha_max, self.t_min
        c.lowpass_sigma, c.z_near = self.lowpass_sigma, self.z_near
        for i in range(3):
            c.bg[i] = float(self.bg[i])
        c.flags = ((0 if self.stats else _abi.FLAG_NO_STATS) | (_abi.FLAG_DEPTH_RAY if self.depth_ray else 0)
                   | ((int(self.fwd_tail) & 0xFF) << 8))
        c.bwd_chunk = int(self.bwd_chunk)
        return c


class Images(NamedTuple):
    rgb: torch.Tensor     # [V, 3, H, W] for equal-size views, else packed [3 * P]
    depth: torch.Tensor   # [V, H, W] or packed [P]
    normal: torch.Tensor  # [V, 3, H, W] or packed [3 * P]
    alpha: torch.Tensor   # [V, H, W] or packed [P]


class SurfelGrads(NamedTuple):
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacity: torch.Tensor
    rgb: torch.Tensor
    pose: torch.Tensor  # [V, 6] dL/d(rho, phi) of T_cw <- Exp(xi) T_cw at xi = 0


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsplat2d takes CUDA tensors only")
    if t.dtype != torch.float32:
        raise ValueError(f"expected float32, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Rasterizer:
    """One rasterization problem: a set of views, a surfel count, the
    constants, and the workspace that holds every intermediate buffer.

    `views` are `scenes.View`-like objects (width, height, fx, fy, cx, cy,
    Rt (3x4 world->camera), surfel_offset, surfel_count).  Images of the
    views are packed one after another.  A forward and its backward must use
    the same Rasterizer with no other forward in between.
    """

    def __init__(self, views: Sequence, n_surfels: int, config: Optional[RasterConfig] = None,
                 capacity: Optional[int] = None, device=None):
        self.lib = _abi.load()
        # no config: the autotuned launch shape of this problem's bucket
        self.config = config or RasterConfig.for_problem(views, n_surfels)
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("the rasterizer runs on CUDA devices only")
        self.n_surfels = int(n_surfels)
        self.n_views = len(views)
        if self.n_views < 1:
            raise ValueError("at least one view is required")
        self._cviews = (_abi.View * self.n_views)()
        self.sizes = []
        pix = 0
        for i, v in enumerate(views):
            cv = self._cviews[i]
            cv.width, cv.height = int(v.width), int(v.height)
            cv.fx, cv.fy, cv.cx, cv.cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
            Rt = [float(x) for x in (v.Rt.reshape(-1).tolist() if hasattr(v.Rt, "reshape") else v.Rt)]
            for k in range(12):
                cv.Rt[k] = Rt[k]
            cnt = getattr(v, "surfel_count", -1)
            off = getattr(v, "surfel_offset", 0)
            cv.surfel_offset = int(off)
            cv.surfel_count = int(self.n_surfels - off if cnt is None or cnt < 0 else cnt)
            cv.pixel_offset = pix
            self.sizes.append((cv.height, cv.width))
            pix += cv.width * cv.height
        self.n_pixels = pix
        self.uniform = len(set(self.sizes)) == 1
        self.n_records = sum(int(self._cviews[i].surfel_count) for i in range(self.n_views))
        self._cfg = self.config.to_c()
        # bumped by every preprocess: the workspace then holds another
        # forward's records, lists and per-pixel state
        self.generation = 0
        cap = capacity if capacity is not None else max(1 << 16, int(1.5 * self.n_records))
        self._alloc(cap)

    # -- workspace ---------------------------------------------------------
    def _problem(self, cap: int) -> _abi.Problem:
        p = _abi.Problem()
        p.views = ctypes.cast(self._cviews, ctypes.POINTER(_abi.View))
        p.n_views = self.n_views
        p.n_surfels = self.n_surfels
        p.instance_capacity = int(cap)
        return p

    def _alloc(self, cap: int):
        self.capacity = int(min(cap, 0xFFFFFFFF))
        self._prob = self._problem(self.capacity)
        size = self.lib.splat2d_workspace_size(ctypes.byref(self._cfg), ctypes.byref(self._prob))
        if size == 0:
            raise ValueError("invalid rasterizer problem (check views, surfel ranges and the config)")
        self.ws_bytes = int(size)
        self.ws = None
        # zero-filled once: the library keeps its gradient records zero between iterations
        self.ws = torch.zeros(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        lay = _abi.Layout()
        _abi.check(self.lib.splat2d_workspace_layout(ctypes.byref(self._cfg), ctypes.byref(self._prob),
                                                     ctypes.byref(lay)), "workspace layout")
        self.layout = lay

    def ws_tensor(self, offset: int, count: int, dtype: torch.dtype) -> torch.Tensor:
        """A typed view of `count` elements at byte `offset` of the workspace."""
        start = self._ws_ptr - self.ws.data_ptr() + int(offset)
        nbytes = int(count) * torch.empty((), dtype=dtype).element_size()
        return self.ws[start:start + nbytes].view(dtype)

    def set_capacity(self, cap: int):
        if int(cap) != self.capacity:
            self._alloc(int(cap))

    def set_config(self, config: RasterConfig):
        self.config = config
        self._cfg = config.to_c()
        self._alloc(self.capacity)

    # -- buffers -----------------------------------------------------------
    def new_images(self) -> Images:
        P = self.n_pixels
        dev = self.device
        return Images(torch.empty(3 * P, device=dev), torch.empty(P, device=dev), torch.empty(3 * P, device=dev),
                      torch.empty(P, device=dev))

    def shaped(self, im: Images) -> Images:
        """[V,3,H,W] / [V,H,W] views of packed images when all views share a size."""
        if not self.uniform:
            return im
        H, W = self.sizes[0]
        V = self.n_views
        return Images(im.rgb.view(V, 3, H, W), im.depth.view(V, H, W), im.normal.view(V, 3, H, W),
                      im.alpha.view(V, H, W))

    def view_images(self, im: Images, v: int) -> Images:
        """Images of view v as ([3,H,W], [H,W], [3,H,W], [H,W])."""
        H, W = self.sizes[v]
        o = int(self._cviews[v].pixel_offset)
        flat = [t.reshape(-1) for t in im]
        return Images(flat[0][3 * o:3 * o + 3 * H * W].view(3, H, W), flat[1][o:o + H * W].view(H, W),
                      flat[2][3 * o:3 * o + 3 * H * W].view(3, H, W), flat[3][o:o + H * W].view(H, W))

    @staticmethod
    def _surfels(means, scales, quats, opacity, rgb) -> _abi.Surfels:
        s = _abi.Surfels()
        s.means, s.scales, s.quats = _ptr(means), _ptr(scales), _ptr(quats)
        s.opacity, s.rgb = _ptr(opacity), _ptr(rgb)
        s.n = means.shape[0]
        return s

    # -- calls -------------------------------------------------------------
    def set_view_pose(self, v: int, Rt):
        """Replace view v's world-to-camera pose (3x4, row-major); takes
        effect from the next preprocess.  A pose step along the tangent the
        backward returns is T_cw <- Exp(xi) T_cw, folded in by the caller."""
        vals = [float(x) for x in (Rt.reshape(-1).tolist() if hasattr(Rt, "reshape") else Rt)]
        if len(vals) != 12:
            raise ValueError("Rt: 12 values (3x4 row-major)")
        for k in range(12):
            self._cviews[v].Rt[k] = vals[k]

    def preprocess(self, means, scales, quats, opacity, rgb):
        if means.shape[0] != self.n_surfels:
            raise ValueError(f"expected {self.n_surfels} surfels, got {means.shape[0]}")
        self.generation += 1
        self._sf = self._surfels(means, scales, quats, opacity, rgb)
        _abi.check(self.lib.splat2d_preprocess(ctypes.byref(self._cfg), ctypes.byref(self._prob),
                                               ctypes.byref(self._sf), self._ws_ptr, self.ws_bytes, _stream()),
                   "splat2d_preprocess")

    def bin_sort(self):
        _abi.check(self.lib.splat2d_bin_sort(ctypes.byref(self._cfg), ctypes.byref(self._prob), self._ws_ptr,
                                             self.ws_bytes, _stream()), "splat2d_bin_sort")

    def render_fwd(self, out: Images, dist: Optional[torch.Tensor] = None):
        """Forward compositing into `out`; with `dist` (one float per packed
        pixel) also the depth distortion."""
        _abi.check(self.lib.splat2d_render_fwd_dist(ctypes.byref(self._cfg), ctypes.byref(self._prob), self._ws_ptr,
                                                    self.ws_bytes, _ptr(out.rgb), _ptr(out.depth), _ptr(out.normal),
                                                    _ptr(out.alpha), _ptr(dist), _stream()), "splat2d_render_fwd")

    def render_bwd(self, means, scales, quats, opacity, rgb, d_out: Sequence[Optional[torch.Tensor]],
                   grads: SurfelGrads, d_dist: Optional[torch.Tensor] = None):
        sf = self._surfels(means, scales, quats, opacity, rgb)
        g = _abi.Grads()
        g.means, g.scales, g.quats = _ptr(grads.means), _ptr(grads.scales), _ptr(grads.quats)
        g.opacity, g.rgb, g.pose = _ptr(grads.opacity), _ptr(grads.rgb), _ptr(grads.pose)
        d = [None if t is None else _ptr(t) for t in d_out]
        _abi.check(self.lib.splat2d_render_bwd_dist(ctypes.byref(self._cfg), ctypes.byref(self._prob),
                                                    ctypes.byref(sf), self._ws_ptr, self.ws_bytes, d[0], d[1], d[2],
                                                    d[3], _ptr(d_dist), ctypes.byref(g), _stream()),
                   "splat2d_render_bwd")

    def render_bwd_tiles(self, d_out: Sequence[Optional[torch.Tensor]], d_dist: Optional[torch.Tensor] = None):
        """Tile adjoint only: record gradients stay in the workspace."""
        d = [None if t is None else _ptr(t) for t in d_out]
        _abi.check(self.lib.splat2d_render_bwd_tiles_dist(ctypes.byref(self._cfg), ctypes.byref(self._prob),
                                                          self._ws_ptr, self.ws_bytes, d[0], d[1], d[2], d[3],
                                                          _ptr(d_dist), _stream()), "splat2d_render_bwd_tiles")

    def max_error(self, err: torch.Tensor, max_err: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Map-fusion pruning input: per surfel, the largest err over the
        pixels that blended it in the last forward (err packed like the
        alpha output).  Raised into `max_err` (zeros if not given)."""
        err = err.contiguous().view(-1)
        if err.numel() != self.n_pixels or err.dtype != torch.float32:
            raise ValueError("err: one float32 per packed pixel")
        if max_err is None:
            max_err = torch.zeros(self.n_surfels, device=self.device)
        _abi.check(self.lib.splat2d_max_error(ctypes.byref(self._cfg), ctypes.byref(self._prob), self._ws_ptr,
                                              self.ws_bytes, _ptr(err), _ptr(max_err), _stream()),
                   "splat2d_max_error")
        return max_err

    def preprocess_bwd(self, means, scales, quats, opacity, rgb, grads: SurfelGrads):
        """Chain rule from the workspace's record gradients to `grads`."""
        sf = self._surfels(means, scales, quats, opacity, rgb)
        g = _abi.Grads()
        g.means, g.scales, g.quats = _ptr(grads.means), _ptr(grads.scales), _ptr(grads.quats)
        g.opacity, g.rgb, g.pose = _ptr(grads.opacity), _ptr(grads.rgb), _ptr(grads.pose)
        _abi.check(self.lib.splat2d_preprocess_bwd(ctypes.byref(self._cfg), ctypes.byref(self._prob), ctypes.byref(sf),
                                                   self._ws_ptr, self.ws_bytes, ctypes.byref(g), _stream()),
                   "splat2d_preprocess_bwd")

    def launch_count(self) -> int:
        return int(self.lib.splat2d_launch_count())

    def stats(self) -> dict:
        """Synchronises; device status and pair counters of the last iteration."""
        st = _abi.Stats()
        self.lib.splat2d_stats(self._ws_ptr, ctypes.byref(st), _stream())
        return {k: getattr(st, k) for k, _ in _abi.Stats._fields_ if k != "reserved"}

    def status(self) -> int:
        need = ctypes.c_int64(0)
        rc = self.lib.splat2d_status(self._ws_ptr, ctypes.byref(need), _stream())
        self._needed = int(need.value)
        return int(rc)

    def forward(self, means, scales, quats, opacity, rgb, out: Optional[Images] = None, check: bool = True,
                max_retries: int = 3, dist: Optional[torch.Tensor] = None) -> Images:
        """preprocess -> bin_sort -> render_fwd.  With check=True the device
        status is read (a synchronisation) and an instance-capacity overflow
        is repaired by growing the workspace and running again."""
        out = out or self.new_images()
        for _ in range(max_retries + 1):
            self.preprocess(means, scales, quats, opacity, rgb)
            self.bin_sort()
            self.render_fwd(out, dist)
            if not check:
                return out
            rc = self.status()
            if rc == _abi.OK:
                return out
            if rc != _abi.ERR_CAPACITY:
                raise _abi.Splat2DError(rc, "device status")
            self.set_capacity(int(self._needed * 1.25) + 1024)
        raise _abi.Splat2DError(_abi.ERR_CAPACITY, "instance capacity")

    def new_grads(self) -> SurfelGrads:
        n, dev = self.n_surfels, self.device
        z = lambda *s: torch.zeros(*s, device=dev)
        return SurfelGrads(z(n, 3), z(n, 2), z(n, 4), z(n), z(n, 3), z(self.n_views, 6))

    def backward(self, means, scales, quats, opacity, rgb, d_out: Sequence[Optional[torch.Tensor]],
                 grads: Optional[SurfelGrads] = None, d_dist: Optional[torch.Tensor] = None) -> SurfelGrads:
        """Gradients of sum(d_out . outputs) (+ sum(d_dist . distortion));
        accumulated into `grads` (zeros if not given).  d_out = (d_rgb,
        d_depth, d_normal, d_alpha), packed like the forward outputs; None
        entries count as zero."""
        grads = grads or self.new_grads()
        flat = [None if t is None else t.contiguous().view(-1) for t in d_out]
        dd = None if d_dist is None else d_dist.contiguous().view(-1)
        self.render_bwd(means, scales, quats, opacity, rgb, flat, grads, dd)
        return grads


def accum_gate(alpha: torch.Tensor, tau: float):
    """Map-fusion insertion gate: (keep_idx, n_keep) with keep_idx[:n_keep]
    the ascending indices of the pixels whose accumulated alpha is below
    tau; n_keep is a device tensor (read it to slice; no sync here)."""
    lib = _abi.load()
    alpha = alpha.contiguous().view(-1)
    if alpha.dtype != torch.float32 or not alpha.is_cuda:
        raise ValueError("alpha: float32 CUDA tensor")
    n = alpha.numel()
    keep = torch.empty(max(n, 1), dtype=torch.int32, device=alpha.device)
    n_keep = torch.zeros(1, dtype=torch.int64, device=alpha.device)
    tmp = torch.empty(max(int(lib.splat2d_accum_gate_tmp_size(n)), 4), dtype=torch.uint8, device=alpha.device)
    _abi.check(lib.splat2d_accum_gate(_ptr(alpha), n, float(tau), keep.data_ptr(), n_keep.data_ptr(),
                                      tmp.data_ptr(), tmp.numel(), _stream()), "splat2d_accum_gate")
    return keep, n_keep


class Splat2DRender(torch.autograd.Function):
    """Differentiable render of all views of `rast`: returns (rgb, depth,
    normal, alpha).

    `pose_tangent` ([V, 6]) receives dL/dxi of each view's pose under the
    left perturbation T_cw <- Exp(xi) T_cw, evaluated at xi = 0.  Its value
    does not enter the render: the poses are the rasterizer's views, so a
    caller that refines poses folds each step into them
    (`Rasterizer.set_view_pose`) and keeps xi at zero.

    The intermediate state the backward needs (records, sorted lists,
    per-pixel transmittance) lives in `rast`'s one workspace, so a second
    render with the same rasterizer overwrites it: the first render's
    backward then raises instead of returning gradients of the wrong forward.
    Use one Rasterizer per render that must stay differentiable."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, means, scales, quats, opacity, rgb, pose_tangent, check: bool = True):
        params = [t.contiguous() for t in (means, scales, quats, opacity, rgb)]
        out = rast.forward(*params, check=check)
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.save_for_backward(*params)
        shaped = rast.shaped(out)
        return tuple(shaped)

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_normal, g_alpha):
        rast: Rasterizer = ctx.rast
        if rast.generation != ctx.generation:
            raise RuntimeError("Splat2DRender: the rasterizer ran another forward after this one, so its "
                               "workspace no longer holds this render's state; use one Rasterizer per "
                               "render that is differentiated")
        params = ctx.saved_tensors
        grads = rast.backward(*params, (g_rgb, g_depth, g_normal, g_alpha))
        return (None, grads.means, grads.scales, grads.quats, grads.opacity, grads.rgb, grads.pose, None)


class Splat2DRenderDist(torch.autograd.Function):
    """Splat2DRender that also returns the depth distortion map (the 2DGS
    regulariser, see splat2d_render_fwd_dist): (rgb, depth, normal, alpha,
    dist), dist shaped like alpha.  The same rules on the workspace apply."""

    @staticmethod
    def forward(ctx, rast: Rasterizer, means, scales, quats, opacity, rgb, pose_tangent, check: bool = True):
        params = [t.contiguous() for t in (means, scales, quats, opacity, rgb)]
        dist = torch.empty(rast.n_pixels, device=rast.device)
        out = rast.forward(*params, check=check, dist=dist)
        ctx.rast = rast
        ctx.generation = rast.generation
        ctx.save_for_backward(*params)
        shaped = rast.shaped(out)
        if rast.uniform:
            H, W = rast.sizes[0]
            dist = dist.view(rast.n_views, H, W)
        return (*shaped, dist)

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_normal, g_alpha, g_dist):
        rast: Rasterizer = ctx.rast
        if rast.generation != ctx.generation:
            raise RuntimeError("Splat2DRenderDist: the rasterizer ran another forward after this one, so its "
                               "workspace no longer holds this render's state; use one Rasterizer per "
                               "render that is differentiated")
        params = ctx.saved_tensors
        grads = rast.backward(*params, (g_rgb, g_depth, g_normal, g_alpha), d_dist=g_dist)
        return (None, grads.means, grads.scales, grads.quats, grads.opacity, grads.rgb, grads.pose, None)


def render(rast: Rasterizer, means, scales, quats, opacity, rgb, pose_tangent=None, check: bool = True,
           distortion: bool = False):
    """Functional form of Splat2DRender (with distortion=True, of
    Splat2DRenderDist: the depth distortion map is a fifth output)."""
    if pose_tangent is None:
        pose_tangent = torch.zeros(rast.n_views, 6, device=means.device, requires_grad=False)
    fn = Splat2DRenderDist if distortion else Splat2DRender
    return fn.apply(rast, means, scales, quats, opacity, rgb, pose_tangent, check)
