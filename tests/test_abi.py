"""The C-ABI library builds, loads and exports every entry point that
include/splat2d.h declares; host-side argument checks work without a GPU
(no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2604_03092_gb300 import _abi, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "splat2d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(splat2d_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert set(_declared()) == set(_abi.SIGNATURES), (set(_declared()) ^ set(_abi.SIGNATURES))


def test_library_exports_every_declared_symbol():
    lib = _abi.load()
    for name in _declared():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {_abi._build.LIB}").read()
    for name in _declared():
        assert re.search(rf"\bT {name}\b", out), name


def _problem(views, n, cap=1000):
    arr = (_abi.View * len(views))()
    for i, v in enumerate(views):
        arr[i].width, arr[i].height = v.width, v.height
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = v.fx, v.fy, v.cx, v.cy
        for k, x in enumerate(v.Rt.reshape(-1)):
            arr[i].Rt[k] = float(x)
        arr[i].surfel_offset = v.surfel_offset
        arr[i].surfel_count = n - v.surfel_offset if v.surfel_count < 0 else v.surfel_count
        arr[i].pixel_offset = sum(w.width * w.height for w in views[:i])
    p = _abi.Problem()
    p.views = ctypes.cast(arr, ctypes.POINTER(_abi.View))
    p.n_views, p.n_surfels, p.instance_capacity = len(views), n, cap
    p._keep = arr
    return p


def test_workspace_size_and_argument_checks():
    lib = _abi.load()
    cfg = _abi.Config()
    lib.splat2d_default_config(ctypes.byref(cfg))
    assert (cfg.tile_w, cfg.tile_h, cfg.chunk, cfg.bwd_chunk) == (8, 8, 128, 64)
    assert cfg.alpha_max == pytest.approx(0.99) and cfg.t_min == pytest.approx(1e-4)
    sc = scenes.random_scene(n=100, width=40, height=30, f=30.0, seed=0, n_views=2)
    p = _problem(sc.views, sc.n)
    size = lib.splat2d_workspace_size(ctypes.byref(cfg), ctypes.byref(p))
    # 80 B record + 80 B gradient + 4 B count per (view, surfel), 24 B per instance of capacity
    assert size >= 2 * 100 * 164 + 1000 * 24
    bad = _abi.Config.from_buffer_copy(cfg)
    bad.tile_w = 12
    assert lib.splat2d_workspace_size(ctypes.byref(bad), ctypes.byref(p)) == 0
    bad = _abi.Config.from_buffer_copy(cfg)
    bad.chunk = 100
    assert lib.splat2d_workspace_size(ctypes.byref(bad), ctypes.byref(p)) == 0
    bad = _abi.Config.from_buffer_copy(cfg)
    bad.bwd_chunk = 512  # 512-entry chunks need 256-pixel tiles
    assert lib.splat2d_workspace_size(ctypes.byref(bad), ctypes.byref(p)) == 0
    ok = _abi.Config.from_buffer_copy(cfg)
    ok.bwd_chunk = 0  # 0: the forward's chunk
    assert lib.splat2d_workspace_size(ctypes.byref(ok), ctypes.byref(p)) > 0
    p2 = _problem(sc.views, sc.n)
    p2._keep[1].surfel_offset = 50
    p2._keep[1].surfel_count = 60  # beyond n
    assert lib.splat2d_workspace_size(ctypes.byref(cfg), ctypes.byref(p2)) == 0
    # calls reject a missing or misaligned workspace before touching the GPU
    rc = lib.splat2d_bin_sort(ctypes.byref(cfg), ctypes.byref(p), None, 0, None)
    assert rc == _abi.ERR_INVALID_ARG
    rc = lib.splat2d_bin_sort(ctypes.byref(cfg), ctypes.byref(p), 256, 16, None)
    assert rc == _abi.ERR_WORKSPACE_TOO_SMALL
    assert lib.splat2d_strerror(_abi.ERR_CAPACITY).decode() == "instance capacity exceeded"
    assert lib.splat2d_sort_pairs(None, None, -1, 8, None, 0, None) == _abi.ERR_INVALID_ARG


def test_layout_offsets_are_aligned_and_inside():
    lib = _abi.load()
    cfg = _abi.Config()
    lib.splat2d_default_config(ctypes.byref(cfg))
    sc = scenes.random_scene(n=333, width=50, height=37, f=30.0, seed=0, n_views=3)
    p = _problem(sc.views, sc.n, cap=12345)
    lay = _abi.Layout()
    assert lib.splat2d_workspace_layout(ctypes.byref(cfg), ctypes.byref(p), ctypes.byref(lay)) == 0
    assert lay.n_records == 3 * 333 and lay.n_pixels == 3 * 50 * 37
    tx, ty = -(-50 // cfg.tile_w), -(-37 // cfg.tile_h)
    assert lay.n_tiles == 3 * tx * ty
    for f in ("records", "ntiles", "keys", "vals", "ranges", "tfinal", "last"):
        off = getattr(lay, f)
        assert off % 256 == 0 and off < lay.total, f
