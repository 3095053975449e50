"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

import oracle
from paper_2604_03092_gb300.rasterizer import RasterConfig, Rasterizer

# tolerances (the library's published parity bar)
FWD_ATOL = 1e-5        # rendered RGB / depth / alpha (and normal), absolute
GRAD_REL_L2 = 1e-3     # gradients, relative L2 per parameter group


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
