"""Parity at the full benchmark size: the 32-keyframe submap (6,291,456
surfels, 32 views at 512x384) in the launch configuration the benchmark
times (the shipped GB300 launch shape of its bucket), checked against the
oracle on sampled pixels -- the forward outputs pixel by pixel, and the
gradients of an upstream gradient that is nonzero only at the sampled
pixels of one view (so the oracle's sampled reverse pass is the whole
gradient)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_utils import FWD_ATOL, GRAD_REL_L2, oracle_cfg, rel_l2, to_dev, view_stack
from paper_2604_03092_gb300 import autotune, scenes
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def submap():
    sc = scenes.submap_scene(seed=2001, n_keyframes=32)
    assert sc.n == 6_291_456 and len(sc.views) == 32
    tw, th, ch, bch = autotune.SHIPPED[autotune.bucket_key(sc.views, sc.n)]
    cfg = RasterConfig(tile_w=tw, tile_h=th, chunk=ch, bwd_chunk=bch)
    params = to_dev(sc)
    rast = Rasterizer(sc.views, sc.n, cfg)
    im = rast.forward(*params)
    torch.cuda.synchronize()
    return sc, cfg, params, rast, im


@pytest.mark.parametrize("v", [0, 17, 31])
def test_forward_sampled_pixels_full_size(submap, v):
    sc, cfg, params, rast, im = submap
    H, W = sc.views[v].height, sc.views[v].width
    pix = np.sort(np.random.default_rng(v).choice(H * W, size=384, replace=False)).astype(np.int64)
    p = oracle.preprocess_scene_view(sc, v, oracle_cfg(cfg))
    ref, _, _, pf = oracle.render_pixels(p, pix)
    gpu = view_stack(rast, im, v).reshape(8, -1)[:, pix]
    ok = (pf & oracle.PF_FORWARD) == 0
    assert ok.mean() > 0.98
    err = np.abs(gpu - ref)[:, ok]
    assert err.max() <= FWD_ATOL, err.max(axis=1)
    assert (ref[7, ok] > 0.5).mean() > 0.5  # mostly covered pixels


def test_backward_sampled_pixels_full_size(submap):
    sc, cfg, params, rast, _ = submap
    v = 5
    H, W = sc.views[v].height, sc.views[v].width
    rng = np.random.default_rng(99)
    p = oracle.preprocess_scene_view(sc, v, oracle_cfg(cfg))
    # pixels whose blend decisions are clear of rounding (alpha near its
    # bounds, T near the stop, a tie in the low-pass max) carry the gradient
    cand = np.sort(rng.choice(H * W, size=400, replace=False)).astype(np.int64)
    _, _, _, pf = oracle.render_pixels(p, cand)
    flags = oracle.PF_FORWARD | oracle.PF_ALPHA_MAX | oracle.PF_BRANCH
    pix = cand[(pf & flags) == 0][:256]
    assert pix.size == 256
    g8 = np.zeros((8, H * W))
    g8[:, pix] = rng.normal(size=(8, pix.size))
    # the library's upstream gradients: zero everywhere but these pixels of view v
    P = rast.n_pixels
    o = int(rast._cviews[v].pixel_offset)
    d = [np.zeros(3 * P, np.float32), np.zeros(P, np.float32), np.zeros(3 * P, np.float32), np.zeros(P, np.float32)]
    for c in range(3):
        d[0][3 * o + c * H * W:3 * o + (c + 1) * H * W] = g8[c]
        d[2][3 * o + c * H * W:3 * o + (c + 1) * H * W] = g8[4 + c]
    d[1][o:o + H * W] = g8[3]
    d[3][o:o + H * W] = g8[7]
    grads = rast.backward(*params, [torch.from_numpy(x).cuda() for x in d])
    torch.cuda.synchronize()
    ref = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8.reshape(8, H, W), pix=pix)
    out = {name: rel_l2(getattr(grads, name).cpu().numpy(), getattr(ref, name))
           for name in ("means", "scales", "quats", "opacity", "rgb")}
    out["pose"] = rel_l2(grads.pose.cpu().numpy()[v], ref.pose)
    for k, e in out.items():
        assert e <= GRAD_REL_L2, (k, out)
    assert np.count_nonzero(ref.opacity) > 100
