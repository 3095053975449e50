"""The backward's per-entry gradient sums accumulate in fixed point with
per-tile power-of-two scales (a tile's first chunk in float, terms outside
a chunk's range added exactly in global memory).  These tests pin what
that design must keep: the gradients of a scene whose tiles run many chunks
agree with the FP64 oracle far inside the parity bar, per parameter and per
surfel, and the scales follow the magnitude of the upstream gradient, so
scaling it by 2^k scales every gradient by 2^k."""
import numpy as np
import pytest
import torch

import oracle
from gpu_utils import oracle_cfg, rel_l2, to_dev
from paper_2604_03092_gb300 import scenes
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

pytestmark = pytest.mark.gpu

NAMES = ("means", "scales", "quats", "opacity", "rgb")


@pytest.fixture(scope="module")
def dense():
    # 60,000 small surfels over one 96x72 view: about 1,200 instances per
    # 8x8 tile, so each tile runs about 20 chunks of 64 entries
    sc = scenes.random_scene(n=60000, width=96, height=72, f=70.0, seed=5, n_views=1, scale_range=(0.01, 0.05))
    params = to_dev(sc)
    rast = Rasterizer(sc.views, sc.n, RasterConfig())
    rast.forward(*params)
    rng = np.random.default_rng(1)
    P = rast.n_pixels
    d = [rng.normal(size=n).astype(np.float32) for n in (3 * P, P, 3 * P, P)]
    return sc, params, rast, d


def _grads(rast, params, d, scale=1.0):
    g = rast.backward(*params, [torch.from_numpy(x * np.float32(scale)).cuda() for x in d])
    torch.cuda.synchronize()
    return {k: getattr(g, k).cpu().numpy().astype(np.float64) for k in NAMES + ("pose",)}


def test_dense_tiles_run_many_chunks(dense):
    sc, params, rast, d = dense
    _grads(rast, params, d)
    st = rast.stats()
    assert st["n_instances"] / rast.layout.n_tiles > 15 * 64
    # terms outside their chunk's range are a small share of all terms
    assert 0 < st["bwd_terms_outside"] < 0.05 * 14 * st["bwd_pairs_blended"]


def test_dense_gradients_match_oracle_per_surfel(dense):
    sc, params, rast, d = dense
    g = _grads(rast, params, d)
    view = sc.views[0]
    H, W = view.height, view.width
    g8 = np.concatenate([d[0].reshape(3, H, W), d[1].reshape(1, H, W), d[2].reshape(3, H, W),
                         d[3].reshape(1, H, W)]).astype(np.float64)
    ref = oracle.render_bwd(sc.means, sc.scales, sc.quats, oracle.preprocess_scene_view(sc, 0, oracle_cfg(RasterConfig())),
                            g8)
    for k in NAMES:
        r = getattr(ref, k).reshape(g[k].shape)
        assert rel_l2(g[k], r) <= 1e-4, k
        gn = np.linalg.norm(r.reshape(len(r), -1), axis=1)
        en = np.linalg.norm((g[k] - r).reshape(len(r), -1), axis=1)
        sel = gn > 1e-3 * gn.max()
        pe = en[sel] / gn[sel]
        assert np.median(pe) <= 1e-5 and np.quantile(pe, 0.99) <= 5e-4, (k, np.median(pe), np.quantile(pe, 0.99))


@pytest.mark.parametrize("k", [-60, 60])
def test_gradients_scale_with_the_upstream_gradient(dense, k):
    sc, params, rast, d = dense
    base = _grads(rast, params, d)
    s = 2.0 ** k
    scaled = _grads(rast, params, d, s)
    for name, v in base.items():
        assert rel_l2(scaled[name] / s, v) <= 1e-5, name
