"""Map maintenance around the rasterizer (Flash-Mono backend, Sec. 4.3):
adaptive voxelization of a keyframe's per-pixel surfels and Sim(3)
transforms for insertion into the world map and for loop correction.
Argument marshalling only: the work runs in libsplat2d's kernels."""
from __future__ import annotations

from typing import Optional, Tuple

import torch

from . import _abi
from .rasterizer import _stream

__all__ = ["voxelize", "sim3_apply"]


def _f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name}: contiguous float32 CUDA tensor expected")
    return t


def voxelize(means, quats, scales, opacity, rgb, width: int, height: int, tau_d: float
             ) -> Tuple[Tuple[torch.Tensor, ...], torch.Tensor, torch.Tensor]:
    """2x2 block merge of a per-pixel map (primitive y * width + x, centers
    in the keyframe's camera frame).  Returns ((means, quats, scales,
    opacity, rgb) buffers of capacity width*height, block index per output,
    n_out as a device int64 tensor); the first n_out rows are valid."""
    lib = _abi.load()
    n = width * height
    ins = [_f32(t, k) for t, k in zip((means, scales, quats, opacity, rgb), ("means", "scales", "quats", "opacity",
                                                                              "rgb"))]
    if any(t.shape[0] != n for t in ins):
        raise ValueError("one primitive per pixel expected")
    dev = means.device
    out = [torch.empty_like(t) for t in ins]
    block = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    tmp = torch.empty(max(int(lib.splat2d_voxelize_tmp_size(width, height)), 4), dtype=torch.uint8, device=dev)
    sf = _abi.Surfels(*[t.data_ptr() for t in ins], n)
    ob = _abi.SurfelBuffers(*[t.data_ptr() for t in out])
    _abi.check(lib.splat2d_voxelize(sf, width, height, float(tau_d), ob, block.data_ptr(), n_out.data_ptr(),
                                    tmp.data_ptr(), tmp.numel(), _stream()), "splat2d_voxelize")
    m, s, q, o, c = out
    return (m, q, s, o, c), block, n_out


def sim3_apply(means: Optional[torch.Tensor], quats: Optional[torch.Tensor], scales: Optional[torch.Tensor],
               sim3: torch.Tensor, index: Optional[torch.Tensor] = None) -> None:
    """In place: mu <- s R mu + t, r <- q r, scales <- s scales, with the
    row (qw, qx, qy, qz, tx, ty, tz, s) of `sim3` chosen per primitive by
    `index` (int32) or row 0."""
    lib = _abi.load()
    present = [t for t in (means, quats, scales) if t is not None]
    if not present:
        return
    n = present[0].shape[0]
    for t, k in ((means, "means"), (quats, "quats"), (scales, "scales")):
        if t is not None:
            _f32(t, k)
            if t.shape[0] != n:
                raise ValueError("all arrays need the same number of primitives")
    _f32(sim3, "sim3")
    if index is not None and not (index.is_cuda and index.dtype == torch.int32 and index.numel() == n):
        raise ValueError("index: int32 CUDA tensor, one per primitive")
    ptr = lambda t: None if t is None else t.data_ptr()
    _abi.check(lib.splat2d_sim3_apply(n, ptr(means), ptr(quats), ptr(scales), sim3.data_ptr(), ptr(index), _stream()),
               "splat2d_sim3_apply")
