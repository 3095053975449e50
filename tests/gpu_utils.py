"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

import oracle
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

# tolerances (the library's published parity bar)
FWD_ATOL = 1e-5        # rendered RGB / depth / alpha (and normal), absolute
GRAD_REL_L2 = 1e-3     # gradients, relative L2 per parameter group
# Pixels whose discrete decisions the oracle reports as within rounding are
# not dropped: each is checked against the oracle's outcomes of those
# decisions taken either way (oracle.render_pixels_either_side).  At most
# this fraction of the checked pixels may match none of them.
MAX_UNRESOLVED = 1e-4


def unresolved_flagged(gpu8, prep, pix, mode=1):
    """How many of the flagged pixels `pix` (flat indices of the view) have
    GPU outputs `gpu8` (8, len(pix)) that match, within FWD_ATOL on every
    channel, no outcome of their near-tie decisions."""
    pix = np.asarray(pix, np.int64)
    if pix.size == 0:
        return 0
    alts = oracle.render_pixels_either_side(prep, pix, mode)  # (k, 8, m)
    err = np.abs(alts - np.asarray(gpu8, np.float64)[None]).max(axis=1)
    return int((err.min(axis=0) > FWD_ATOL).sum())


def oracle_cfg(cfg: RasterConfig) -> oracle.Config:
    return oracle.Config(alpha_min=cfg.alpha_min, alpha_max=cfg.alpha_max, t_min=cfg.t_min,
                         sigma_lp=cfg.lowpass_sigma, z_near=cfg.z_near, bg=tuple(cfg.bg),
                         tile_w=cfg.tile_w, tile_h=cfg.tile_h, depth_ray=bool(cfg.depth_ray))


def to_dev(sc, dev="cuda"):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in
            (sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb)]


def gpu_forward(sc, cfg: RasterConfig, capacity=None):
    params = to_dev(sc)
    rast = Rasterizer(sc.views, sc.n, cfg, capacity=capacity)
    im = rast.forward(*params)
    torch.cuda.synchronize()
    return rast, params, im


def view_stack(rast, im, v):
    """(8, H, W) float64: r g b depth nx ny nz alpha of view v."""
    r = rast.view_images(im, v)
    return np.concatenate([r.rgb.cpu().numpy(), r.depth[None].cpu().numpy(), r.normal.cpu().numpy(),
                           r.alpha[None].cpu().numpy()]).astype(np.float64)


def upstream(rast, seed):
    """Seeded upstream gradients for every view, packed like the outputs;
    returns (torch tuple for the library, list of (8,H,W) arrays per view)."""
    rng = np.random.default_rng(seed)
    per_view = [rng.normal(size=(8, h, w)) for (h, w) in rast.sizes]
    rgb = np.concatenate([g[0:3].reshape(-1) for g in per_view])
    depth = np.concatenate([g[3].reshape(-1) for g in per_view])
    normal = np.concatenate([g[4:7].reshape(-1) for g in per_view])
    alpha = np.concatenate([g[7].reshape(-1) for g in per_view])
    dev = [torch.from_numpy(x.astype(np.float32)).cuda() for x in (rgb, depth, normal, alpha)]
    return dev, per_view


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def sampled_forward(sc, rast, im, cfg, v, n_pix, seed):
    """Forward outputs of view v at n_pix sampled pixels against the oracle
    (binned mode): unflagged pixels within FWD_ATOL (asserted here), flagged
    ones checked against either outcome of their decisions.  Returns
    (flagged, unresolved, checked, fraction of sampled pixels with alpha > 1/2)."""
    H, W = sc.views[v].height, sc.views[v].width
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(H * W, size=min(n_pix, H * W), replace=False)).astype(np.int64)
    p = oracle.preprocess_scene_view(sc, v, oracle_cfg(cfg))
    ref, _, _, pf = oracle.render_pixels(p, pix)
    gpu = view_stack(rast, im, v).reshape(8, -1)[:, pix]
    ok = (pf & oracle.PF_FORWARD) == 0
    err = np.abs(gpu - ref)[:, ok]
    assert err.max() <= FWD_ATOL, (v, err.max(axis=1))
    near = ~ok
    unresolved = unresolved_flagged(gpu[:, near], p, pix[near])
    return int(near.sum()), unresolved, int(pix.size), float((ref[7] > 0.5).mean())


def sampled_backward(sc, rast, params, cfg, v, n_pix, seed):
    """Gradients of an upstream gradient that is nonzero only at n_pix
    sampled pixels of view v whose blend decisions are clear of rounding (so
    the oracle's reverse pass over those pixels is the whole gradient),
    through the batched rasterizer `rast`.  Returns the relative L2 error per
    parameter group over the view's surfel range, the pose error of view v,
    and checks that nothing outside the range or on another view's pose
    received a gradient."""
    H, W = sc.views[v].height, sc.views[v].width
    off, cnt = sc.view_ranges()[v]
    sl = slice(off, off + cnt)
    rng = np.random.default_rng(seed)
    p = oracle.preprocess_scene_view(sc, v, oracle_cfg(cfg))
    cand = np.sort(rng.choice(H * W, size=min(H * W, int(n_pix * 1.6)), replace=False)).astype(np.int64)
    _, _, _, pf = oracle.render_pixels(p, cand)
    flags = oracle.PF_FORWARD | oracle.PF_ALPHA_MAX | oracle.PF_BRANCH
    pix = cand[(pf & flags) == 0][:n_pix]
    assert pix.size == n_pix
    g8 = np.zeros((8, H * W))
    g8[:, pix] = rng.normal(size=(8, pix.size))
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
    ref = oracle.render_bwd(sc.means[sl], sc.scales[sl], sc.quats[sl], p, g8.reshape(8, H, W), pix=pix)
    out = {}
    for name in ("means", "scales", "quats", "opacity", "rgb"):
        g = getattr(grads, name)
        out[name] = rel_l2(g[sl].cpu().numpy(), getattr(ref, name))
        assert int(torch.count_nonzero(g[:off])) == 0 and int(torch.count_nonzero(g[off + cnt:])) == 0, name
    gp = grads.pose.cpu().numpy()
    out["pose"] = rel_l2(gp[v], ref.pose)
    assert not np.any(np.delete(gp, v, axis=0)), "pose gradient on a view with no upstream gradient"
    assert np.count_nonzero(ref.opacity) > 100
    return out
