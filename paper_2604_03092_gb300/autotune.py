"""Autotuner for the rasterizer's launch shape: tile shape (8x8, 16x16, 32x8)
and the shared-memory chunk depths (64, 128, 256) of the forward and of the
backward compositing pass.

A candidate is timed over a few full forward + backward iterations of the
caller's own problem; the fastest is cached in a JSON file keyed by the
problem's image-size bucket (log2 of the mean view pixel count) and its
density bucket (log2 of the mean number of surfels per pixel per view), so
that problems of the same shape reuse the choice without re-timing.  Buckets
that were measured on GB300 when the library was built ship with it
(SHIPPED) and answer lookups that the user's cache cannot.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

Candidate = Tuple[int, int, int, int]  # tile_w, tile_h, chunk, backward chunk

CANDIDATES: List[Candidate] = [(16, 16, 256, 256), (16, 16, 128, 128), (16, 16, 256, 128), (8, 8, 64, 64),
                               (8, 8, 128, 128), (8, 8, 128, 64), (8, 8, 256, 64), (32, 8, 256, 256),
                               (32, 8, 128, 128)]

# Best launch shapes measured on GB300 by tune() with cuda_runner (forward +
# backward step time over the candidates above), by bucket: one 512x384
# keyframe seen from 8 views (img18_dens0), 64 uneven submaps at
# 320x240..640x480 (img18_dens1: 8x8/64/64 91.8 ms, 8x8/128/64 93.2 ms),
# 8- and 32-keyframe submaps at 512x384 (img18_dens3, img18_dens5:
# 8x8/64/64 66.8 ms, 8x8/128/64 68.2 ms, 16x16/256/256 102.1 ms), the
# 150-keyframe map seen at 640x480 (img18_dens7: 8x8/64/64 59.7 ms,
# 8x8/128/64 60.4 ms, 16x16/256/256 79.6 ms).
SHIPPED: Dict[str, Candidate] = {"img18_dens0": (8, 8, 128, 64), "img18_dens1": (8, 8, 64, 64),
                                 "img18_dens3": (8, 8, 64, 64), "img18_dens5": (8, 8, 64, 64),
                                 "img18_dens7": (8, 8, 64, 64)}


def _candidate(x) -> Candidate:
    t = tuple(int(v) for v in x)
    return t if len(t) == 4 else (t[0], t[1], t[2], t[2])  # type: ignore[return-value]

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("SPLAT2D_AUTOTUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "splat2d", "autotune.json")


def bucket_key(views: Sequence, n_surfels: int) -> str:
    pix = [int(v.width) * int(v.height) for v in views]
    counts = []
    for v in views:
        c = getattr(v, "surfel_count", -1)
        counts.append(n_surfels - getattr(v, "surfel_offset", 0) if c is None or c < 0 else c)
    mean_pix = sum(pix) / max(len(pix), 1)
    density = sum(counts) / max(sum(pix), 1)
    return f"img{round(math.log2(max(mean_pix, 1)))}_dens{round(math.log2(max(density, 1e-6)))}"


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: Dict[str, dict]):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(views: Sequence, n_surfels: int, path: Optional[str] = None,
           shipped: bool = True) -> Optional[Candidate]:
    """The cached best (tile_w, tile_h, chunk, backward chunk) for this
    problem's bucket; else the shipped measurement for it (if `shipped`)."""
    key = bucket_key(views, n_surfels)
    entry = _load(path or cache_path()).get(key)
    if entry:
        return _candidate(entry["best"])
    if shipped and key in SHIPPED:
        return _candidate(SHIPPED[key])
    return None


def tune(views: Sequence, n_surfels: int, run: Callable[[Candidate], float],
         candidates: Iterable[Candidate] = CANDIDATES, path: Optional[str] = None,
         force: bool = False) -> Tuple[Candidate, Dict[str, float]]:
    """Time every candidate with `run(candidate) -> milliseconds per
    iteration` (lower is better), cache and return the fastest.  A cached
    entry is returned without timing unless force=True."""
    path = path or cache_path()
    key = bucket_key(views, n_surfels)
    with _lock:
        table = _load(path)
        if not force and key in table:
            return _candidate(table[key]["best"]), table[key]["ms"]
    results: Dict[str, float] = {}
    best, best_ms = None, math.inf
    for c in candidates:
        c = _candidate(c)
        ms = float(run(c))
        results["x".join(map(str, c))] = ms
        if ms < best_ms:
            best, best_ms = c, ms
    if best is None:
        raise ValueError("no candidates")
    with _lock:
        table = _load(path)
        table[key] = {"best": list(best), "ms": results}
        _store(path, table)
    return best, results


def cuda_runner(views, params, d_out, steps: int = 3, warmup: int = 1, capacity: Optional[int] = None):
    """A `run` function for tune(): full forward + backward iterations on the
    GPU, timed with CUDA events."""
    import torch

    from .rasterizer import RasterConfig, Rasterizer

    n = params[0].shape[0]

    def timed(c: Candidate) -> float:
        cfg = RasterConfig(tile_w=c[0], tile_h=c[1], chunk=c[2], bwd_chunk=c[3])
        rast = Rasterizer(views, n, cfg, capacity=capacity)
        rast.forward(*params)  # sizes the capacity
        grads = rast.new_grads()
        out = rast.new_images()
        for _ in range(warmup):
            rast.forward(*params, out=out, check=False)
            rast.backward(*params, d_out, grads=grads)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            rast.forward(*params, out=out, check=False)
            rast.backward(*params, d_out, grads=grads)
        b.record()
        torch.cuda.synchronize()
        if rast.status() != 0:
            return math.inf
        return a.elapsed_time(b) / steps

    def run(c: Candidate) -> float:
        # each candidate's workspace is released before the next one (a large
        # problem's workspace can be a good part of the device); a candidate
        # that does not fit scores as infinitely slow
        try:
            return timed(c)
        except torch.cuda.OutOfMemoryError:
            return math.inf
        finally:
            torch.cuda.synchronize()
            torch.cuda.empty_cache()

    return run
