"""Map maintenance kernels (adaptive voxelization, Sim(3) transforms)
through the C ABI, against the oracle's NumPy statements."""
import numpy as np
import pytest
import torch

from oracle import fusion
from paper_2604_03092_gb300 import mapping

pytestmark = pytest.mark.gpu


def _map(W, H, seed, tau_d):
    """A per-pixel map whose 2x2 blocks have a depth range either well
    below or well above tau_d (no block within rounding of the gate)."""
    rng = np.random.default_rng(seed)
    n = W * H
    yy, xx = np.divmod(np.arange(n), W)
    block = (yy // 2) * ((W + 1) // 2) + xx // 2
    rough = rng.uniform(size=block.max() + 1) < 0.3
    z = 0.5 + rng.uniform(0, 7.5, block.max() + 1)[block]
    z = z + np.where(rough[block], rng.uniform(0, 6 * tau_d, n) * (np.arange(n) % 2 + 1),
                     rng.uniform(0, 0.2 * tau_d, n))
    means = np.stack([rng.uniform(-3, 3, n), rng.uniform(-2, 2, n), z], 1)
    quats = rng.normal(size=(n, 4))
    scales = rng.uniform(0.002, 0.02, (n, 2))
    opacity = rng.uniform(0.5, 1.0, n)
    rgb = rng.uniform(0, 1, (n, 3))
    arrs = [a.astype(np.float32) for a in (means, quats, scales, opacity, rgb)]
    # keep every block clear of the gate: flatten blocks whose range ended up
    # near tau_d
    z32 = arrs[0][:, 2].astype(np.float64)
    nb = block.max() + 1
    lo, hi = np.full(nb, np.inf), np.full(nb, -np.inf)
    np.minimum.at(lo, block, z32)
    np.maximum.at(hi, block, z32)
    near = np.abs(hi - lo - tau_d) < 1e-3
    _, first = np.unique(block, return_index=True)
    flat = near[block]
    arrs[0][flat, 2] = arrs[0][first[block[flat]], 2]
    return arrs


@pytest.mark.parametrize("W,H", [(64, 48), (37, 23), (512, 384), (1, 1)])
def test_voxelize_matches_oracle(W, H):
    tau = 0.1
    m, q, s, o, c = _map(W, H, W * 7 + H, tau)
    dev = [torch.from_numpy(a).cuda() for a in (m, q, s, o, c)]
    (gm, gq, gs, go, gc), gb, n_out = mapping.voxelize(*dev, W, H, tau)
    k = int(n_out.item())
    (rm, rq, rs, ro, rc), rb = fusion.voxelize(m, q, s, o, c, W, H, tau)
    assert k == rb.size
    np.testing.assert_array_equal(gb[:k].cpu().numpy(), rb)
    for g, r, tol in ((gm, rm, 1e-6), (gq, rq, 2e-6), (gs, rs, 1e-6), (go, ro, 1e-6), (gc, rc, 1e-6)):
        g = g[:k].cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(g, r.reshape(g.shape), rtol=tol, atol=1e-7)
    if W * H > 4:
        assert (np.bincount(rb) > 1).any() and (np.bincount(rb) == 1).any()  # both kinds of block


@pytest.mark.parametrize("n,k,indexed", [(10_000, 5, True), (257, 1, False), (0, 1, False)])
def test_sim3_matches_oracle(n, k, indexed):
    rng = np.random.default_rng(n + k)
    means = rng.uniform(-5, 5, (n, 3)).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    scales = rng.uniform(0.01, 0.1, (n, 2)).astype(np.float32)
    sim3 = np.concatenate([rng.normal(size=(k, 4)), rng.normal(size=(k, 3)), rng.uniform(0.5, 2.0, (k, 1))],
                          1).astype(np.float32)
    index = rng.integers(0, k, n).astype(np.int32) if indexed else None
    dm, dq, ds = (torch.from_numpy(a.copy()).cuda() for a in (means, quats, scales))
    mapping.sim3_apply(dm, dq, ds, torch.from_numpy(sim3).cuda(),
                       None if index is None else torch.from_numpy(index).cuda())
    rm, rq, rs = fusion.sim3_apply(means, quats, scales, sim3.astype(np.float64), index)
    np.testing.assert_allclose(dm.cpu().numpy(), rm, rtol=2e-6, atol=2e-5)
    np.testing.assert_allclose(dq.cpu().numpy(), rq.reshape(-1, 4), rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(ds.cpu().numpy(), rs.reshape(-1, 2), rtol=2e-6, atol=1e-9)
