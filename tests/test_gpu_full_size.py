"""Parity at the full benchmark size: the 32-keyframe submap (6,291,456
surfels, 32 views at 512x384) in the launch configuration the benchmark
times (the shipped GB300 launch shape of its bucket), checked against the
oracle on sampled pixels -- the forward outputs pixel by pixel (pixels whose
decisions the oracle flags as within rounding against either outcome of
those decisions), and the gradients of an upstream gradient that is nonzero
only at the sampled pixels of one view (so the oracle's sampled reverse pass
is the whole gradient)."""
import pytest
import torch

from gpu_utils import GRAD_REL_L2, MAX_UNRESOLVED, sampled_backward, sampled_forward, to_dev
from paper_2604_03092_gb300 import autotune, scenes
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

# flagged fraction measured with the oracle on 2,000 sampled pixels of
# views 0 and 17 of this submap: 5e-4 and 1.5e-3
MAX_FLAGGED = 3e-3


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
    yield sc, cfg, params, rast, im
    del rast, im, params
    torch.cuda.empty_cache()


def test_forward_sampled_pixels_full_size(submap):
    sc, cfg, params, rast, im = submap
    flagged = unresolved = total = 0
    for v in (0, 17, 31):
        f, u, n, covered = sampled_forward(sc, rast, im, cfg, v, 2000, seed=v)
        flagged, unresolved, total = flagged + f, unresolved + u, total + n
        assert covered > 0.5  # mostly covered pixels
    print(f"flagged {flagged}/{total} = {flagged / total:.2e} of sampled pixels; unresolved {unresolved}")
    assert flagged <= MAX_FLAGGED * total, (flagged, total)
    assert unresolved <= MAX_UNRESOLVED * total, (unresolved, flagged, total)


def test_backward_sampled_pixels_full_size(submap):
    sc, cfg, params, rast, _ = submap
    out = sampled_backward(sc, rast, params, cfg, 5, 256, seed=99)
    print(out)
    for k, e in out.items():
        assert e <= GRAD_REL_L2, (k, out)
