"""Map-fusion consumers of the forward (Sec. 4.3, "Map Fusion"), through the
C ABI, against the oracle: the per-surfel error attribution that pruning
reads, and the accumulation gate that decides where new primitives go."""
import numpy as np
import pytest
import torch

import oracle
from gpu_utils import gpu_forward, oracle_cfg
from paper_2604_03092_gb300 import scenes
from paper_2604_03092_gb300.rasterizer import RasterConfig, accum_gate

pytestmark = pytest.mark.gpu


def _errors_and_reference(sc, rast, cfg, seed):
    """Seeded per-pixel errors (zero where a pixel's blend decisions are
    within rounding, so both sides see the same blended pairs) and the
    oracle's attribution, raised over all views."""
    rng = np.random.default_rng(seed)
    ocfg = oracle_cfg(cfg)
    ref = np.zeros(sc.n)
    errs = []
    for v, vw in enumerate(sc.views):
        p = oracle.preprocess_scene_view(sc, v, ocfg)
        im = oracle.render(p)
        e = rng.uniform(0.05, 1.0, (vw.height, vw.width)).astype(np.float32)
        e[(im.pflags & oracle.PF_FORWARD) != 0] = 0.0
        e[rng.uniform(size=e.shape) < 0.1] = 0.0  # pixels without error
        off, cnt = sc.view_ranges()[v]
        part = oracle.max_error(p, e.astype(np.float64))
        ref[off:off + cnt] = np.maximum(ref[off:off + cnt], part)
        errs.append(e.reshape(-1))
    return torch.from_numpy(np.concatenate(errs)).cuda(), ref


@pytest.mark.parametrize("tile", [(8, 8), (16, 16)])
def test_max_error_matches_oracle(tile):
    sc = scenes.random_scene(n=4096, seed=3, n_views=2)
    cfg = RasterConfig(tile_w=tile[0], tile_h=tile[1])
    rast, params, _ = gpu_forward(sc, cfg)
    err, ref = _errors_and_reference(sc, rast, cfg, seed=1)
    got = rast.max_error(err).cpu().numpy().astype(np.float64)
    assert (ref > 0).sum() > 500
    # a maximum of given values: exact
    np.testing.assert_array_equal(got, ref)
    # raising an existing array only ever increases it
    start = torch.full((sc.n,), 0.5, device="cuda")
    got2 = rast.max_error(err, start).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got2, np.maximum(ref, np.float32(0.5)))


def test_max_error_with_surfel_ranges():
    # views rendering different surfel ranges of one buffer (submaps)
    sc = scenes.random_scene(n=3000, width=64, height=48, f=50.0, seed=9, n_views=3)
    for v, (o, c) in enumerate(((0, 2000), (1000, 2000), (500, 1500))):
        sc.views[v].surfel_offset, sc.views[v].surfel_count = o, c
    cfg = RasterConfig()
    rast, params, _ = gpu_forward(sc, cfg)
    err, ref = _errors_and_reference(sc, rast, cfg, seed=2)
    got = rast.max_error(err).cpu().numpy().astype(np.float64)
    assert (ref > 0).sum() > 200
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("n", [0, 1, 1023, 1024, 100_003])
def test_accum_gate_is_an_ordered_compaction(n):
    rng = np.random.default_rng(n)
    a = rng.uniform(0, 1, n).astype(np.float32)
    tau = np.float32(0.4)
    if n > 10:
        a[::7] = tau                 # equal to the threshold: not kept
        a[3::11] = np.float32("nan")  # never kept
    keep, n_keep = accum_gate(torch.from_numpy(a).cuda(), float(tau))
    k = int(n_keep.item())
    expect = oracle.accum_gate(a, tau)
    assert k == expect.size
    np.testing.assert_array_equal(keep[:k].cpu().numpy().astype(np.int64), expect)
