"""Pins for the oracle's map-maintenance statements (oracle/fusion.py):
closed forms of the 2x2 voxelization, quaternion alignment, the depth
gate, and Sim(3) transforms checked against rotation matrices and against
the image model (a similarity applied to map and camera leaves the image
unchanged, depth scaled).  CPU only."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from oracle import fusion
from paper_2604_03092_gb300 import scenes


def _map(W, H, seed, z0=2.0, dz=0.01):
    rng = np.random.default_rng(seed)
    n = W * H
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), z0 + rng.uniform(0, dz, n)], 1)
    quats = rng.normal(size=(n, 4))
    scales = rng.uniform(0.01, 0.05, (n, 2))
    opacity = rng.uniform(0.5, 1.0, n)
    rgb = rng.uniform(0, 1, (n, 3))
    return [a.astype(np.float32) for a in (means, quats, scales, opacity, rgb)]


def test_identical_block_merges_to_itself():
    m, q, s, o, c = _map(2, 2, 0)
    for a in (m, q, s, o, c):
        a[1:] = a[0]
    (m2, q2, s2, o2, c2), blk = fusion.voxelize(m, q, s, o, c, 2, 2, tau_d=0.1)
    assert len(blk) == 1
    np.testing.assert_allclose(m2[0], m[0], rtol=1e-7)
    np.testing.assert_allclose(q2[0], q[0] / np.linalg.norm(q[0]), rtol=1e-7)
    np.testing.assert_allclose(s2[0], s[0], rtol=1e-7)
    assert o2[0] == pytest.approx(o[0]) and np.allclose(c2[0], c[0])


def test_quaternion_alignment_and_means():
    """q and -q are one rotation: after alignment to the block's first
    quaternion their average is that rotation; the other attributes are
    plain means (written out by hand here)."""
    m, q, s, o, c = _map(2, 2, 1)
    q[:] = q[0]
    q[1] *= -1
    q[3] *= -1
    (m2, q2, s2, o2, c2), _ = fusion.voxelize(m, q, s, o, c, 2, 2, tau_d=0.1)
    np.testing.assert_allclose(q2[0], q[0] / np.linalg.norm(q[0]), rtol=1e-6)
    np.testing.assert_allclose(m2[0], (m[0].astype(float) + m[1] + m[2] + m[3]) / 4, rtol=1e-7)
    assert o2[0] == pytest.approx((float(o[0]) + o[1] + o[2] + o[3]) / 4)
    np.testing.assert_allclose(s2[0], (s[0].astype(float) + s[1] + s[2] + s[3]) / 4, rtol=1e-7)
    # the merged rotation is the normalised sum of the aligned rotations: for
    # two distinct rotations it bisects them (equal angle to each)
    q = np.array([[1, 0, 0, 0], [np.cos(0.3), np.sin(0.3), 0, 0], [1, 0, 0, 0], [np.cos(0.3), np.sin(0.3), 0, 0]],
                 np.float32)
    q[1] *= -1
    (_, q3, _, _, _), _ = fusion.voxelize(m, q, s, o, c, 2, 2, tau_d=0.1)
    ang = Rotation.from_quat([q3[0][1], q3[0][2], q3[0][3], q3[0][0]]).as_rotvec()
    assert ang[0] == pytest.approx(0.3, rel=1e-5) and abs(ang[1]) < 1e-9 and abs(ang[2]) < 1e-9


def test_depth_gate_keeps_blocks_and_order():
    W, H = 6, 4
    m, q, s, o, c = _map(W, H, 2)
    m[2 * W + 3, 2] += 0.5  # pixel (3, 2): block (1, 1) varies by more than tau_d
    (m2, q2, s2, o2, c2), blk = fusion.voxelize(m, q, s, o, c, W, H, tau_d=0.1)
    nb = (W // 2) * (H // 2)
    assert len(blk) == nb - 1 + 4
    assert list(blk) == sorted(blk)
    kept = np.nonzero(blk == 1 * (W // 2) + 1)[0]
    np.testing.assert_array_equal(m2[kept], m[[2 * W + 2, 2 * W + 3, 3 * W + 2, 3 * W + 3]].astype(np.float64))


def test_ragged_edges():
    W, H = 5, 3
    m, q, s, o, c = _map(W, H, 3)
    (m2, _, _, o2, _), blk = fusion.voxelize(m, q, s, o, c, W, H, tau_d=1.0)
    assert len(blk) == 3 * 2
    # block (2, 1) holds only pixel (4, 2)
    np.testing.assert_allclose(m2[-1], m[2 * W + 4], rtol=1e-7)
    # block (2, 0) holds pixels (4, 0) and (4, 1)
    assert o2[2] == pytest.approx((float(o[4]) + o[W + 4]) / 2)


def test_sim3_against_rotation_matrices():
    rng = np.random.default_rng(4)
    m, q, s, _, _ = _map(3, 3, 4)
    T = np.concatenate([rng.normal(size=4), rng.normal(size=3), [1.7]])
    m2, q2, s2 = fusion.sim3_apply(m, q, s, T)
    R = Rotation.from_quat([T[1], T[2], T[3], T[0]]).as_matrix()
    for i in range(len(m)):
        np.testing.assert_allclose(m2[i], 1.7 * R @ m[i].astype(float) + T[4:7], rtol=1e-10, atol=1e-12)
        Ri = Rotation.from_quat([q[i][1], q[i][2], q[i][3], q[i][0]]).as_matrix()
        R2 = Rotation.from_quat([q2[i][1], q2[i][2], q2[i][3], q2[i][0]]).as_matrix()
        np.testing.assert_allclose(R2, R @ Ri, atol=1e-12)
        np.testing.assert_allclose(s2[i], 1.7 * s[i].astype(float), rtol=1e-12)
    # composition and inverse
    U = np.concatenate([rng.normal(size=4), rng.normal(size=3), [0.6]])
    a = fusion.sim3_apply(*fusion.sim3_apply(m, q, s, T), U)
    b = fusion.sim3_apply(m, q, s, fusion.sim3_compose(T, U))
    for x, y in zip(a, b):
        np.testing.assert_allclose(np.abs(x) if x.shape[1] == 4 else x, np.abs(y) if y.shape[1] == 4 else y,
                                   rtol=1e-10, atol=1e-12)
    back = fusion.sim3_apply(*fusion.sim3_apply(m, q, s, T), fusion.sim3_inverse(T))
    np.testing.assert_allclose(back[0], m, atol=1e-6)
    np.testing.assert_allclose(back[2], s, rtol=1e-6)


@pytest.mark.parametrize("scale", [1.0, 1.6])
def test_sim3_leaves_the_image_unchanged(scale):
    """A similarity applied to the map and to the camera (x_cam' = s x_cam)
    leaves colour and alpha unchanged and scales depth by s: the image
    model pins how centers, rotations and scales are transformed."""
    sc = scenes.random_scene(n=300, width=40, height=30, f=35.0, seed=5, scale_range=(0.02, 0.1))
    rng = np.random.default_rng(6)
    T = np.concatenate([Rotation.from_rotvec(rng.normal(size=3) * 0.3).as_quat()[[3, 0, 1, 2]],
                        rng.normal(size=3) * 0.2, [scale]])
    m2, q2, s2 = fusion.sim3_apply(sc.means, sc.quats, sc.scales, T)
    R = fusion.quat_to_rot(T[:4])
    Rc, tc = sc.views[0].Rt[:, :3].astype(np.float64), sc.views[0].Rt[:, 3].astype(np.float64)
    R1 = Rc @ R.T
    t1 = scale * tc - R1 @ T[4:7]
    v1 = scenes.View(40, 30, 35.0, 35.0, 20.0, 15.0, np.concatenate([R1, t1[:, None]], 1).astype(np.float32))
    cfg = oracle.Config()
    im0 = oracle.render(oracle.preprocess(sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb, sc.views[0], cfg))
    im1 = oracle.render(oracle.preprocess(m2.astype(np.float32), s2.astype(np.float32), q2.astype(np.float32),
                                          sc.opacity, sc.rgb, v1, cfg))
    ok = ((im0.pflags | im1.pflags) & oracle.PF_FORWARD) == 0
    assert ok.mean() > 0.95 and (im0.alpha > 0).mean() > 0.3
    np.testing.assert_allclose(im1.rgb[:, ok], im0.rgb[:, ok], atol=2e-5)
    np.testing.assert_allclose(im1.alpha[ok], im0.alpha[ok], atol=2e-5)
    np.testing.assert_allclose(im1.depth[ok], scale * im0.depth[ok], atol=2e-4)
