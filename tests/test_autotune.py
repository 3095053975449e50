"""Host logic of the autotuner (CPU, with a fake timer)."""
from paper_2604_03092_gb300 import autotune, scenes


def test_tune_picks_fastest_and_caches(tmp_path):
    sc = scenes.random_scene(n=1000, width=64, height=48, f=50.0, seed=0, n_views=2)
    path = str(tmp_path / "cache.json")
    calls = []

    def fake(c):
        calls.append(c)
        return {(8, 8, 128, 64): 1.5}.get(c, 2.0 + c[2] / 1000)

    best, res = autotune.tune(sc.views, sc.n, fake, path=path)
    assert best == (8, 8, 128, 64)
    assert len(calls) == len(autotune.CANDIDATES) and len(res) == len(calls)
    assert autotune.lookup(sc.views, sc.n, path=path) == (8, 8, 128, 64)
    # cached: no re-timing
    best2, _ = autotune.tune(sc.views, sc.n, lambda c: 1 / 0, path=path)
    assert best2 == (8, 8, 128, 64)
    # a different bucket is not served from the cache
    big = scenes.random_scene(n=1000, width=640, height=480, f=500.0, seed=0)
    assert autotune.lookup(big.views, big.n, path=path) is None


def test_bucket_key_separates_image_size_and_density():
    a = scenes.random_scene(n=1000, width=64, height=48, seed=0)
    b = scenes.random_scene(n=100000, width=64, height=48, seed=0, with_target=False)
    c = scenes.random_scene(n=1000, width=512, height=384, seed=0, with_target=False)
    ka, kb, kc = (autotune.bucket_key(s.views, s.n) for s in (a, b, c))
    assert len({ka, kb, kc}) == 3


def test_lookup_reads_three_field_entries_and_shipped_table(tmp_path, monkeypatch):
    import json
    sc = scenes.random_scene(n=1000, width=64, height=48, f=50.0, seed=0, n_views=2)
    key = autotune.bucket_key(sc.views, sc.n)
    path = tmp_path / "old.json"
    path.write_text(json.dumps({key: {"best": [16, 16, 128], "ms": {}}}))
    assert autotune.lookup(sc.views, sc.n, path=str(path)) == (16, 16, 128, 128)
    empty = str(tmp_path / "none.json")
    monkeypatch.setitem(autotune.SHIPPED, key, (8, 8, 128, 64))
    assert autotune.lookup(sc.views, sc.n, path=empty) == (8, 8, 128, 64)
    assert autotune.lookup(sc.views, sc.n, path=empty, shipped=False) is None


def test_shipped_shapes_are_candidates_the_library_accepts():
    # tile shapes and chunk depths the C library's config check takes
    tiles = {(16, 16), (8, 8), (32, 8)}
    for key, c in autotune.SHIPPED.items():
        assert c in autotune.CANDIDATES, (key, c)
        tw, th, ch, bch = c
        assert (tw, th) in tiles
        for depth in (ch, bch):
            assert depth in (64, 128, 256) or (depth == 512 and tw * th == 256)


def test_tune_on_the_gpu(tmp_path):
    """The tuner times every candidate launch shape on the GPU with real
    forward + backward iterations, caches the fastest, and a rasterizer built
    without a config takes it; every candidate renders the same images."""
    import math

    import numpy as np
    import pytest
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer
    sc = scenes.keyframe_scene(seed=1005, width=128, height=96, f=100.0, n_views=2)
    params = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
              (sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb)]
    P = sum(v.width * v.height for v in sc.views)
    g = torch.Generator(device="cuda").manual_seed(0)
    d_out = (torch.randn(3 * P, device="cuda", generator=g), torch.randn(P, device="cuda", generator=g), None, None)
    path = str(tmp_path / "tune.json")
    import os
    os.environ["SPLAT2D_AUTOTUNE_CACHE"] = path
    try:
        best, ms = autotune.tune(sc.views, sc.n, autotune.cuda_runner(sc.views, params, d_out), path=path)
        assert best in [autotune._candidate(c) for c in autotune.CANDIDATES]
        assert len(ms) == len(autotune.CANDIDATES) and all(math.isfinite(v) and v > 0 for v in ms.values())
        rast = Rasterizer(sc.views, sc.n)  # no config: the cached choice
        assert (rast.config.tile_w, rast.config.tile_h, rast.config.chunk, rast.config.bwd_chunk) == best
        ref = Rasterizer(sc.views, sc.n, RasterConfig()).forward(*params)
        for c in autotune.CANDIDATES:
            c = autotune._candidate(c)
            im = Rasterizer(sc.views, sc.n, RasterConfig(tile_w=c[0], tile_h=c[1], chunk=c[2], bwd_chunk=c[3])).forward(*params)
            for a, b in zip(im, ref):
                assert float((a - b).abs().max()) <= 1e-5, c
    finally:
        del os.environ["SPLAT2D_AUTOTUNE_CACHE"]


test_tune_on_the_gpu = __import__("pytest").mark.gpu(test_tune_on_the_gpu)
