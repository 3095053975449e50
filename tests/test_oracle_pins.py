"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a closed form, Eq. 1 in its screen-space-covariance form, an
independent ray-plane intersection, an invariant of the model, or FP64
central differences of its own forward (the definition of the derivative).
CPU only."""
import copy

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2604_03092_gb300 import scenes

EYE = np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32)


def _view(W=32, H=24, f=40.0, Rt=EYE, fy=None):
    return scenes.View(W, H, f, f if fy is None else fy, W / 2.0, H / 2.0, np.asarray(Rt, np.float32))


def _render(means, scales, quats, op, rgb, view, cfg, mode=1):
    p = oracle.preprocess(np.asarray(means, np.float32).reshape(-1, 3), np.asarray(scales, np.float32).reshape(-1, 2),
                          np.asarray(quats, np.float32).reshape(-1, 4), np.asarray(op, np.float32).reshape(-1),
                          np.asarray(rgb, np.float32).reshape(-1, 3), view, cfg)
    return oracle.render(p, mode), p


def _rot(q_wxyz):
    q = np.asarray(q_wxyz, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_single_surfel_at_pixel_center():
    """P1: a surfel whose center projects onto a pixel center has rho = 0
    there, so alpha = sigma, C = sigma c, D = sigma z, N = sigma n_c with n_c
    the surfel normal turned towards the camera (Eq. 1 with one term)."""
    cfg = oracle.Config()
    view = _view()
    z = 3.0
    for seed in range(5):
        rng = np.random.default_rng(seed)
        ix, iy = 11, 9
        mu = [(ix + 0.5 - view.cx) * z / view.fx, (iy + 0.5 - view.cy) * z / view.fy, z]
        q = rng.normal(size=4)
        # keep the surfel clearly off edge-on
        n = _rot(q)[:, 2]
        if abs(n[2]) < 0.3:
            q = np.array([1.0, 0.1, -0.2, 0.05])
        sigma, col = 0.7, rng.uniform(0, 1, 3)
        im, p = _render(mu, [0.05, 0.08], q, sigma, col, view, cfg)
        mu32 = np.asarray(mu, np.float32).astype(np.float64)
        sigma = float(np.float32(sigma))
        # the float32 center sits within ~1e-6 px of the pixel center
        assert im.alpha[iy, ix] == pytest.approx(sigma, abs=1e-9)
        np.testing.assert_allclose(im.rgb[:, iy, ix], sigma * col.astype(np.float32), atol=1e-9)
        assert im.depth[iy, ix] == pytest.approx(sigma * mu32[2], abs=1e-9)
        q32 = np.asarray(q, np.float32).astype(np.float64)
        nrm = _rot(q32)[:, 2]
        if nrm @ mu32 > 0:
            nrm = -nrm
        np.testing.assert_allclose(im.normal[:, iy, ix], sigma * nrm, atol=1e-9)


def test_edge_on_surfel():
    """P2: the camera center lies in the surfel plane.  With the low-pass
    term off the surfel is invisible; with it on, the image is exactly the
    screen-space blob sigma*exp(-|x-c|^2/(2 sigma_lp^2)) around the center."""
    view = _view(W=24, H=20, f=30.0)
    mu = [0.13, -0.07, 2.5]
    # plane spanned by the viewing ray through mu and the y axis -> contains the origin
    ray = np.array(mu) / np.linalg.norm(mu)
    tu = ray
    nvec = np.cross(ray, [0.0, 1.0, 0.0]); nvec /= np.linalg.norm(nvec)
    tv = np.cross(nvec, tu)
    q = Rotation.from_matrix(np.stack([tu, tv, nvec], 1)).as_quat()
    q = np.array([q[3], q[0], q[1], q[2]])
    sigma = float(np.float32(0.8))
    im, _ = _render(mu, [0.2, 0.2], q, sigma, [1, 1, 1], view, oracle.Config(sigma_lp=0.0))
    assert np.abs(im.out).max() == 0.0
    slp = 0.70710678118654752
    cfg = oracle.Config(sigma_lp=slp)
    im, p = _render(mu, [0.2, 0.2], q, sigma, [1, 1, 1], view, cfg)
    mu32 = np.asarray(mu, np.float32).astype(np.float64)
    cx, cy = view.fx * mu32[0] / mu32[2] + view.cx, view.fy * mu32[1] / mu32[2] + view.cy
    jj, ii = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
    d2 = (ii + 0.5 - cx) ** 2 + (jj + 0.5 - cy) ** 2
    a = np.minimum(cfg.alpha_max, sigma * np.exp(-d2 / (2 * np.float32(slp) ** 2)))
    a = np.where(a >= np.float32(cfg.alpha_min), a, 0.0)
    np.testing.assert_allclose(im.alpha, a, atol=1e-9)
    assert im.alpha.max() > 0.5


@pytest.mark.parametrize("theta,fy", [(0.0, 40.0), (0.7, 40.0), (2.1, 55.0)])
def test_fronto_parallel_is_eq1(theta, fy):
    """P3: for a surfel parallel to the image plane the 2DGS intersection is
    exactly Eq. 1: w = sigma exp(-1/2 d^T Sigma^-1 d) with the screen-space
    covariance Sigma = J R2 diag(s_u^2, s_v^2) R2^T J, J = diag(fx, fy)/z."""
    view = _view(W=40, H=30, f=40.0, fy=fy)
    cfg = oracle.Config(sigma_lp=0.0)
    mu = [0.11, -0.06, 2.0]
    su, sv, sigma = 0.09, 0.04, 0.6
    q = [np.cos(theta / 2), 0.0, 0.0, np.sin(theta / 2)]
    im, _ = _render(mu, [su, sv], q, sigma, [1, 1, 1], view, cfg)
    m = np.asarray(mu, np.float32).astype(np.float64)
    s = np.asarray([su, sv], np.float32).astype(np.float64)
    qq = np.asarray(q, np.float32).astype(np.float64)
    th = 2 * np.arctan2(qq[3], qq[0])
    R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    J = np.diag([np.float32(view.fx), np.float32(view.fy)]) / m[2]
    Sig = J @ R2 @ np.diag(s ** 2) @ R2.T @ J
    c = np.array([view.fx * m[0] / m[2] + view.cx, view.fy * m[1] / m[2] + view.cy])
    jj, ii = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
    d = np.stack([ii + 0.5 - c[0], jj + 0.5 - c[1]], -1)
    q2 = np.einsum("hwi,ij,hwj->hw", d, np.linalg.inv(Sig), d)
    w = np.float32(sigma) * np.exp(-0.5 * q2)
    w = np.where(w >= np.float32(cfg.alpha_min), np.minimum(w, np.float32(cfg.alpha_max)), 0.0)
    np.testing.assert_allclose(im.alpha, w, atol=1e-12)
    assert (im.alpha > 0).sum() > 20


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_tilted_surfel_matches_ray_plane_intersection(seed):
    """P3b: for a tilted surfel under a general pose, alpha at each pixel is
    sigma*exp(-(u^2+v^2)/2) with (u, v) the local coordinates of the point
    where the pixel's ray meets the surfel plane, found by a textbook
    ray-plane intersection (independent of the homography/adjugate)."""
    rng = np.random.default_rng(100 + seed)
    Rc = Rotation.from_rotvec(rng.normal(size=3) * 0.2).as_matrix()
    tc = rng.normal(size=3) * 0.3
    Rt = np.concatenate([Rc, tc[:, None]], 1).astype(np.float32)
    view = _view(W=36, H=28, f=35.0, Rt=Rt)
    cfg = oracle.Config(sigma_lp=0.0)
    Rc32, tc32 = Rt[:, :3].astype(np.float64), Rt[:, 3].astype(np.float64)
    # place the center 2.5 m in front of the camera near the optical axis
    mc = np.array([0.1, -0.05, 2.5]) + rng.normal(size=3) * 0.05
    mu = Rc32.T @ (mc - tc32)
    q = rng.normal(size=4)
    su, sv, sigma = 0.15, 0.08, 0.75
    im, p = _render(mu, [su, sv], q, sigma, [1, 1, 1], view, cfg)
    m = np.asarray(mu, np.float32).astype(np.float64)
    Rs = _rot(np.asarray(q, np.float32).astype(np.float64))
    s = np.asarray([su, sv], np.float32).astype(np.float64)
    mcam = Rc32 @ m + tc32
    U = Rc32 @ Rs[:, 0] * s[0]
    V = Rc32 @ Rs[:, 1] * s[1]
    n = np.cross(U, V)
    jj, ii = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
    dirs = np.stack([(ii + 0.5 - view.cx) / view.fx, (jj + 0.5 - view.cy) / view.fy, np.ones_like(ii, float)], -1)
    lam = (n @ mcam) / (dirs @ n)
    X = dirs * lam[..., None]
    # X - mu_c = u U + v V (U, V need not be exactly orthogonal: FP32 camera)
    G = np.array([[U @ U, U @ V], [U @ V, V @ V]])
    rhs = np.stack([(X - mcam) @ U, (X - mcam) @ V], -1)
    uv = rhs @ np.linalg.inv(G).T
    u, v = uv[..., 0], uv[..., 1]
    a = np.float32(sigma) * np.exp(-0.5 * (u * u + v * v))
    a = np.where((a >= np.float32(cfg.alpha_min)) & (lam > 0), np.minimum(a, np.float32(cfg.alpha_max)), 0.0)
    np.testing.assert_allclose(im.alpha, a, atol=1e-10)
    assert (im.alpha > 0).sum() >= 3


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ray_depth_matches_ray_plane_intersection(seed):
    """f1: with the per-pixel depth option, a single tilted surfel's depth
    output divided by its alpha is, at every pixel it covers, the depth of
    the point where the pixel's ray meets the surfel plane -- found here by
    the plane equation n . X = n . mu_c (independent of the adjugate and of
    det(M)); without the option it is the center's depth everywhere."""
    rng = np.random.default_rng(300 + seed)
    Rc = Rotation.from_rotvec(rng.normal(size=3) * 0.2).as_matrix()
    tc = rng.normal(size=3) * 0.3
    Rt = np.concatenate([Rc, tc[:, None]], 1).astype(np.float32)
    view = _view(W=36, H=28, f=35.0, Rt=Rt)
    Rc32, tc32 = Rt[:, :3].astype(np.float64), Rt[:, 3].astype(np.float64)
    mc = np.array([0.05, -0.05, 2.0]) + rng.normal(size=3) * 0.05
    mu = Rc32.T @ (mc - tc32)
    q = rng.normal(size=4)
    su, sv, sigma = 0.3, 0.02, 0.8  # thin: the screen-space term wins across it near the center
    m = np.asarray(mu, np.float32).astype(np.float64)
    Rs = _rot(np.asarray(q, np.float32).astype(np.float64))
    mcam = Rc32 @ m + tc32
    s32 = np.asarray([su, sv], np.float32).astype(np.float64)
    U, V = Rc32 @ Rs[:, 0] * s32[0], Rc32 @ Rs[:, 1] * s32[1]
    n = np.cross(U, V)
    jj, ii = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
    dirs = np.stack([(ii + 0.5 - view.cx) / view.fx, (jj + 0.5 - view.cy) / view.fy, np.ones_like(ii, float)], -1)
    zplane = (n @ mcam) / (dirs @ n)
    # which term of the low-pass max decides at each pixel (u, v from the plane point)
    X = dirs * zplane[..., None]
    Gm = np.array([[U @ U, U @ V], [U @ V, V @ V]])
    uv = np.stack([(X - mcam) @ U, (X - mcam) @ V], -1) @ np.linalg.inv(Gm).T
    rho_obj = (uv ** 2).sum(-1)
    cx, cy = view.fx * mcam[0] / mcam[2] + view.cx, view.fy * mcam[1] / mcam[2] + view.cy
    rho_lp = ((ii + 0.5 - cx) ** 2 + (jj + 0.5 - cy) ** 2) / 0.5
    for ray, lp in ((True, 0.0), (False, 0.0), (True, 0.70710678118654752)):
        cfg = oracle.Config(sigma_lp=lp, depth_ray=ray)
        im, p = _render(mu, [su, sv], q, sigma, [1, 1, 1], view, cfg)
        cov = im.alpha > 0
        assert cov.sum() > 10
        z = im.depth[cov] / im.alpha[cov]
        if not ray:
            np.testing.assert_allclose(z, mcam[2], rtol=1e-12)
        elif lp == 0.0:
            np.testing.assert_allclose(z, zplane[cov], rtol=1e-10)
        else:
            # with the low-pass max, pixels where the screen-space term wins
            # take the center's depth (pixels with the two terms within 1e-6
            # of a tie are not checked)
            obj = (rho_obj <= rho_lp)[cov]
            clear = (np.abs(rho_obj - rho_lp) > 1e-6 * (1 + rho_lp))[cov]
            np.testing.assert_allclose(z[obj & clear], zplane[cov][obj & clear], rtol=1e-10)
            np.testing.assert_allclose(z[~obj & clear], mcam[2], rtol=1e-12)
            assert (obj & clear).sum() > 5 and (~obj & clear).sum() > 0


def test_ray_depth_fronto_parallel_is_center_depth():
    """f1: a surfel parallel to the image plane meets every ray at its
    center's depth, so both depth readings give the same image."""
    view = _view(W=30, H=24, f=30.0)
    mu, q = [0.05, -0.02, 2.5], [1.0, 0.0, 0.0, 0.0]
    ims = [_render(mu, [0.2, 0.12], q, 0.7, [0.2, 0.5, 0.9], view, oracle.Config(depth_ray=r))[0] for r in (0, 1)]
    np.testing.assert_allclose(ims[1].out, ims[0].out, rtol=1e-12, atol=1e-15)
    assert (ims[0].alpha > 0).sum() > 20


def test_two_surfels_blend_front_to_back():
    """P4: two surfels centred on the same pixel at depths z1 < z2:
    C = c1 s1 + c2 s2 (1 - s1), D = z1 s1 + z2 s2 (1 - s1), regardless of
    their order in the arrays."""
    view = _view()
    cfg = oracle.Config()
    ix, iy = 7, 13
    zs = [2.0, 3.0]
    mus = [[(ix + 0.5 - view.cx) * z / view.fx, (iy + 0.5 - view.cy) * z / view.fy, z] for z in zs]
    cols = np.array([[1.0, 0.2, 0.1], [0.1, 0.9, 0.3]], np.float32)
    sig = np.array([0.6, 0.5], np.float32).astype(np.float64)
    q = [[1, 0.05, 0.02, 0], [1, -0.03, 0.04, 0.1]]
    for order in ([0, 1], [1, 0]):
        im, _ = _render(np.array(mus)[order], [[0.05, 0.05]] * 2, np.array(q)[order], sig[order], cols[order],
                        view, cfg)
        c = cols[0] * sig[0] + cols[1] * sig[1] * (1 - sig[0])
        np.testing.assert_allclose(im.rgb[:, iy, ix], c, atol=1e-8)
        z32 = np.asarray(mus, np.float32)[:, 2].astype(np.float64)
        assert im.depth[iy, ix] == pytest.approx(z32[0] * sig[0] + z32[1] * sig[1] * (1 - sig[0]), abs=1e-8)


def test_transmittance_stop_rule():
    """P5: a stack of identical surfels with alpha = 1/2 at one pixel blends
    exactly the 13 that keep T >= 1e-4 (0.5^13 >= 1e-4 > 0.5^14) and stops."""
    view = _view()
    cfg = oracle.Config()
    ix, iy = 5, 5
    zs = 2.0 + 0.01 * np.arange(20)
    mus = np.array([[(ix + 0.5 - view.cx) * z / view.fx, (iy + 0.5 - view.cy) * z / view.fy, z] for z in zs])
    k = len(zs)
    im, _ = _render(mus, [[0.05, 0.05]] * k, [[1, 0, 0, 0]] * k, [0.5] * k, [[1, 1, 1]] * k, view, cfg)
    assert im.nblend[iy, ix] == 13
    assert im.alpha[iy, ix] == pytest.approx(1 - 0.5 ** 13, abs=1e-12)
    assert im.tfinal[iy, ix] == pytest.approx(0.5 ** 13, abs=1e-15)


def test_near_plane_cull():
    """A surfel whose opacity-aware disk reaches z <= z_near contributes
    nothing; moved slightly back so that the disk clears the plane, it does."""
    view = _view()
    cfg = oracle.Config(z_near=0.5)
    q = Rotation.from_rotvec([0.0, 1.2, 0.0]).as_quat()
    q = [q[3], q[0], q[1], q[2]]  # tilted so the disk spans depth
    s = 0.1
    k = np.sqrt(2 * np.log(0.9 / np.float32(cfg.alpha_min)))
    sin_t = np.sin(1.2)
    zmin_off = k * s * sin_t
    im, p = _render([0, 0, 0.5 + 0.5 * zmin_off], [s, s], q, 0.9, [1, 1, 1], view, cfg)
    assert p.status[0] == oracle.ST_NEAR and im.alpha.max() == 0
    im, p = _render([0, 0, 0.5 + 1.5 * zmin_off], [s, s], q, 0.9, [1, 1, 1], view, cfg)
    assert p.status[0] == oracle.ST_VISIBLE and im.alpha.max() > 0.5


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _dyadic_scene(seed, n=200):
    """Values on dyadic grids so that exact rigid motions stay exact in FP32."""
    rng = np.random.default_rng(seed)
    m = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n), rng.uniform(1.5, 3.0, n)], 1)
    m = np.round(m * 4096) / 4096
    s = np.round(np.exp(rng.uniform(np.log(0.02), np.log(0.12), (n, 2))) * 4096) / 4096
    q = np.round(rng.uniform(-1, 1, (n, 4)) * 256) / 256
    q[np.abs(q).sum(1) == 0, 0] = 1
    op = np.round(rng.uniform(0.05, 1.0, n) * 256) / 256
    col = rng.uniform(0, 1, (n, 3))
    return [a.astype(np.float32) for a in (m, s, q, op, col)]


def _qmul(a, b):
    w1, v1 = a[..., 0], a[..., 1:]
    w2, v2 = b[..., 0], b[..., 1:]
    w = w1 * w2 - np.sum(v1 * v2, -1)
    v = w1[..., None] * v2 + w2[..., None] * v1 + np.cross(v1, v2)
    return np.concatenate([w[..., None], v], -1)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_rigid_motion_invariance(axis):
    """P5: moving every surfel and the camera by the same rigid motion g
    (90 degrees about a coordinate axis plus an integer shift, exact in FP32)
    leaves RGB, depth, normal and alpha unchanged."""
    m, s, q, op, col = _dyadic_scene(7 + axis)
    cfg = oracle.Config()
    W, H, f = 48, 36, 40.0
    base = oracle.render(oracle.preprocess(m, s, q, op, col, _view(W, H, f), cfg))
    Rg = np.round(Rotation.from_rotvec(np.eye(3)[axis] * np.pi / 2).as_matrix())
    tg = np.array([3.0, -2.0, 5.0])
    qg = np.zeros(4); qg[0] = 1.0; qg[1 + axis] = 1.0  # unnormalised: the rasterizer normalises
    m2 = (m.astype(np.float64) @ Rg.T + tg).astype(np.float32)
    q2 = _qmul(np.broadcast_to(qg, q.shape), q.astype(np.float64)).astype(np.float32)
    Rt2 = np.concatenate([Rg.T, (-Rg.T @ tg)[:, None]], 1).astype(np.float32)
    moved = oracle.render(oracle.preprocess(m2, s, q2, op, col, _view(W, H, f, Rt=Rt2), cfg))
    assert np.array_equal(base.nblend, moved.nblend)
    np.testing.assert_allclose(moved.out, base.out, atol=1e-11)
    assert base.alpha.max() > 0.9


def test_similarity_scale():
    """P5 (Sim(3), as in the map fusion transform mu_w = s R mu_c + t):
    scaling means, tangent scales and the camera translation by 2 leaves
    RGB/normal/alpha unchanged and doubles the depth."""
    m, s, q, op, col = _dyadic_scene(3)
    cfg = oracle.Config()
    Rt = EYE.copy(); Rt[:, 3] = [0.25, -0.125, 0.5]
    a = oracle.render(oracle.preprocess(m, s, q, op, col, _view(48, 36, 40.0, Rt=Rt), cfg))
    Rt2 = Rt.copy(); Rt2[:, 3] *= 2
    b = oracle.render(oracle.preprocess(2 * m, 2 * s, q, op, col, _view(48, 36, 40.0, Rt=Rt2), cfg))
    for c in (0, 1, 2, 4, 5, 6, 7):
        np.testing.assert_allclose(b.out[c], a.out[c], atol=1e-11)
    np.testing.assert_allclose(b.depth, 2 * a.depth, atol=1e-11)


def test_weights_and_permutation():
    """P5: A = 1 - T_final in [0, 1 - t_min]; T_final >= t_min by the stop
    rule; permuting surfel indices (distinct depths) gives identical bits."""
    sc = scenes.random_scene(n=512, width=48, height=40, f=40.0, seed=11)
    cfg = oracle.Config()
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    im = oracle.render(p)
    assert np.all(im.alpha >= 0) and np.all(im.alpha <= 1 - cfg.t_min + 1e-15)
    np.testing.assert_allclose(im.alpha, 1 - im.tfinal, atol=0)
    assert np.all(im.tfinal >= np.float32(cfg.t_min))
    perm = np.random.default_rng(0).permutation(sc.n)
    p2 = oracle.preprocess(sc.means[perm], sc.scales[perm], sc.quats[perm], sc.opacity[perm], sc.rgb[perm],
                           sc.views[0], cfg)
    im2 = oracle.render(p2)
    assert np.array_equal(im.out, im2.out)


# --------------------------------------------------------------------------
# the screen extent is the bounding box of the alpha >= alpha_min region,
# no wider: pinned against a closed form and against the projected disk
# --------------------------------------------------------------------------

def _pix_interval(lo, hi, lim):
    """Pixel centers (index + 1/2) inside [lo, hi], clipped to [0, lim]."""
    a, b = int(np.ceil(lo - 0.5)), int(np.floor(hi - 0.5))
    return max(a, 0), min(b, lim)


def _edge_clear(lo, hi, margin=1e-6):
    """Neither edge of [lo, hi] is within `margin` of a pixel-center boundary."""
    return all(abs(e - 0.5 - np.round(e - 0.5)) > margin for e in (lo, hi))


@pytest.mark.parametrize("fy", [52.0, 71.0])
def test_extent_fronto_parallel_closed_form(fy):
    """C5 for a surfel parallel to the image plane: the support of alpha >=
    alpha_min is the ellipse of Eq. 1's screen-space covariance
    Sigma = J R2 diag(s^2) R2^T J (J = diag(fx, fy)/z) at Mahalanobis radius
    k = sqrt(2 ln(sigma/alpha_min)), united with the low-pass disk of radius
    sigma_lp k around the projected center c; its bounding box is
    c +- k sqrt(Sigma_ii) and c +- sigma_lp k, and the pixel rect is the
    pixel centers inside it, clipped to the image -- exactly, so an extent
    that is wider than the support (a spare margin, a wider low-pass square)
    fails here as surely as one that is too small."""
    W, H, fx = 64, 48, 52.0
    view = _view(W=W, H=H, f=fx, fy=fy)
    cfg = oracle.Config()
    rng = np.random.default_rng(int(fy))
    n = 400
    z = rng.uniform(1.5, 4.0, n)
    mu = np.stack([rng.uniform(-1.2, 1.2, n) * z / 2.0, rng.uniform(-0.9, 0.9, n) * z / 2.0, z], 1)
    th = rng.uniform(0, 2 * np.pi, n)
    q = np.stack([np.cos(th / 2), np.zeros(n), np.zeros(n), np.sin(th / 2)], 1)
    # small surfels (the low-pass disk decides) to large ones (the ellipse decides)
    sc_ = np.exp(rng.uniform(np.log(0.003), np.log(0.15), (n, 2)))
    op = rng.uniform(0.02, 1.0, n)
    p = oracle.preprocess(mu.astype(np.float32), sc_.astype(np.float32), q.astype(np.float32),
                          op.astype(np.float32), np.ones((n, 3), np.float32), view, cfg)
    m32, s32 = mu.astype(np.float32).astype(np.float64), sc_.astype(np.float32).astype(np.float64)
    q32, o32 = q.astype(np.float32).astype(np.float64), op.astype(np.float32).astype(np.float64)
    a_min, slp = float(np.float32(cfg.alpha_min)), float(np.float32(cfg.sigma_lp))
    fxx, fyy, cxx, cyy = (float(np.float32(x)) for x in (view.fx, view.fy, view.cx, view.cy))
    checked = lowpass_decides = 0
    for i in range(n):
        R2 = _rot(q32[i])[:2, :2]
        J = np.diag([fxx, fyy]) / m32[i, 2]
        Sig = J @ R2 @ np.diag(s32[i] ** 2) @ R2.T @ J
        k = np.sqrt(2.0 * np.log(o32[i] / a_min))
        c = np.array([fxx * m32[i, 0] / m32[i, 2] + cxx, fyy * m32[i, 1] / m32[i, 2] + cyy])
        half = np.maximum(k * np.sqrt(np.diag(Sig)), slp * k)
        lo, hi = c - half, c + half
        if not (_edge_clear(lo[0], hi[0]) and _edge_clear(lo[1], hi[1])):
            continue
        x0, x1 = _pix_interval(lo[0], hi[0], W - 1)
        y0, y1 = _pix_interval(lo[1], hi[1], H - 1)
        if x0 > x1 or y0 > y1:
            assert p.status[i] == oracle.ST_EMPTY, i
            continue
        assert p.status[i] == oracle.ST_VISIBLE, i
        assert list(p.pixrect[i]) == [x0, y0, x1, y1], (i, list(p.pixrect[i]), [x0, y0, x1, y1])
        checked += 1
        lowpass_decides += int(np.any(k * np.sqrt(np.diag(Sig)) < slp * k))
    assert checked > 250 and lowpass_decides > 20, (checked, lowpass_decides)


def _disk_extent(mc, U, V, k, f, cc, axis, sign, samples=4096):
    """max over the boundary circle u^2 + v^2 = k^2 of sign * (projected
    coordinate along `axis`): P(phi) = mu_c + k (cos phi U + sin phi V),
    x(phi) = f P_axis / P_z + c; dense sampling, then a bounded scalar
    refinement around the best sample."""
    from scipy.optimize import minimize_scalar

    def x(ph):
        P = mc[:, None] + k * (np.cos(ph) * U[:, None] + np.sin(ph) * V[:, None])
        return sign * (f * P[axis] / P[2] + cc)
    ph = np.linspace(0, 2 * np.pi, samples, endpoint=False)
    j = int(np.argmax(x(ph)))
    h = 2 * np.pi / samples
    r = minimize_scalar(lambda t: -float(x(np.array([t]))[0]), bounds=(ph[j] - h, ph[j] + h), method="bounded",
                        options={"xatol": 1e-13})
    return sign * max(-r.fun, float(x(ph[j:j + 1])[0]))


@pytest.mark.parametrize("seed", [0, 1])
def test_extent_is_bounding_box_of_alpha_support(seed):
    """C5 for tilted surfels under a general pose: the oracle's extent (a
    dual conic) equals the bounding box of the set where sigma G >= alpha_min
    -- the perspective image of the disk u^2 + v^2 <= k^2 on the surfel
    plane, whose extreme coordinates lie on its boundary circle (found here
    by maximising the projected circle directly), united with the low-pass
    disk |x - c| <= sigma_lp k -- and the pixel rect is the pixel centers in
    it, clipped to the image: no pixel center is in the rect that no point of
    the support reaches in that row or column."""
    rng = np.random.default_rng(300 + seed)
    Rc = Rotation.from_rotvec(rng.normal(size=3) * 0.3).as_matrix()
    tc = rng.normal(size=3) * 0.3
    Rt = np.concatenate([Rc, tc[:, None]], 1).astype(np.float32)
    W, H = 80, 60
    view = _view(W=W, H=H, f=60.0, Rt=Rt, fy=66.0)
    cfg = oracle.Config()
    n = 300
    R32, t32 = Rt[:, :3].astype(np.float64), Rt[:, 3].astype(np.float64)
    mc = np.stack([rng.uniform(-1.0, 1.0, n), rng.uniform(-0.8, 0.8, n), rng.uniform(1.5, 4.0, n)], 1)
    mc[:, :2] *= mc[:, 2:3] / 2.0
    mu = (mc - t32) @ R32  # world centers: R^T (mc - t)
    q = rng.normal(size=(n, 4))
    sc_ = np.exp(rng.uniform(np.log(0.004), np.log(0.2), (n, 2)))
    op = rng.uniform(0.02, 1.0, n)
    p = oracle.preprocess(mu.astype(np.float32), sc_.astype(np.float32), q.astype(np.float32),
                          op.astype(np.float32), np.ones((n, 3), np.float32), view, cfg)
    m32, s32 = mu.astype(np.float32).astype(np.float64), sc_.astype(np.float32).astype(np.float64)
    q32, o32 = q.astype(np.float32).astype(np.float64), op.astype(np.float32).astype(np.float64)
    a_min, slp = float(np.float32(cfg.alpha_min)), float(np.float32(cfg.sigma_lp))
    fxx, fyy, cxx, cyy = (float(np.float32(x)) for x in (view.fx, view.fy, view.cx, view.cy))
    checked = 0
    for i in range(n):
        if p.status[i] not in (oracle.ST_VISIBLE, oracle.ST_EMPTY) or p.sflags[i]:
            continue
        Rs = _rot(q32[i])
        mcam = R32 @ m32[i] + t32
        U = R32 @ Rs[:, 0] * s32[i, 0]
        V = R32 @ Rs[:, 1] * s32[i, 1]
        k = np.sqrt(2.0 * np.log(o32[i] / a_min))
        c = np.array([fxx * mcam[0] / mcam[2] + cxx, fyy * mcam[1] / mcam[2] + cyy])
        lo, hi = np.zeros(2), np.zeros(2)
        for ax, (f_, cc) in enumerate(((fxx, cxx), (fyy, cyy))):
            hi[ax] = max(_disk_extent(mcam, U, V, k, f_, cc, ax, 1.0), c[ax] + slp * k)
            lo[ax] = min(_disk_extent(mcam, U, V, k, f_, cc, ax, -1.0), c[ax] - slp * k)
        if not (_edge_clear(lo[0], hi[0], 1e-5) and _edge_clear(lo[1], hi[1], 1e-5)):
            continue
        x0, x1 = _pix_interval(lo[0], hi[0], W - 1)
        y0, y1 = _pix_interval(lo[1], hi[1], H - 1)
        if x0 > x1 or y0 > y1:
            assert p.status[i] == oracle.ST_EMPTY, i
            continue
        assert p.status[i] == oracle.ST_VISIBLE, i
        assert list(p.pixrect[i]) == [x0, y0, x1, y1], (i, list(p.pixrect[i]), [x0, y0, x1, y1], lo, hi)
        checked += 1
    assert checked > 150, checked


@pytest.mark.parametrize("seed,tile", [(0, (16, 16)), (1, (8, 8)), (2, (32, 8))])
def test_binned_equals_definition(seed, tile):
    """P6: restricting each surfel to the pixels of its opacity-aware rect
    (the tiled renderer's semantics) changes no pixel, except those the
    oracle itself reports as decided within rounding."""
    sc = scenes.random_scene(n=1024, width=64, height=48, f=50.0, seed=seed)
    cfg = oracle.Config(tile_w=tile[0], tile_h=tile[1])
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    a = oracle.render(p, 1)
    b = oracle.render(p, 0)
    ok = ((a.pflags | b.pflags) & oracle.PF_FORWARD) == 0
    assert ok.mean() > 0.995
    np.testing.assert_allclose(a.out[:, ok], b.out[:, ok], atol=1e-12)


def test_binned_equals_definition_keyframe_crop():
    """P6 on the per-pixel keyframe workload (crop of a 512x384 keyframe)."""
    sc = scenes.keyframe_scene(seed=1001, width=96, height=72, f=75.0, n_views=2)
    cfg = oracle.Config()
    for v in range(2):
        p = oracle.preprocess_scene_view(sc, v, cfg)
        a = oracle.render(p, 1)
        b = oracle.render(p, 0)
        ok = ((a.pflags | b.pflags) & oracle.PF_FORWARD) == 0
        assert ok.mean() > 0.99
        np.testing.assert_allclose(a.out[:, ok], b.out[:, ok], atol=1e-12)
        assert a.alpha.mean() > 0.5


def test_bin_sort_is_a_stable_sort_of_the_rect_instances():
    """P9: the instance list holds exactly one (tile, surfel) pair per tile of
    each visible surfel's tile rect (enumerated here independently), keys
    are non-decreasing and equal keys keep ascending surfel index."""
    sc = scenes.random_scene(n=300, width=64, height=48, f=50.0, seed=5, n_views=3)
    cfg = oracle.Config(tile_w=8, tile_h=8)
    preps = [oracle.preprocess_scene_view(sc, v, cfg) for v in range(3)]
    tx, ty = 8, 6
    keys, vals = oracle.bin_sort(preps, [0, tx * ty, 2 * tx * ty], [tx] * 3, [0, 0, 0])
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])
    expect = set()
    for v, p in enumerate(preps):
        for s in np.nonzero(p.status == 0)[0]:
            x0, y0, x1, y1 = p.tilerect[s]
            for yy in range(y0, y1 + 1):
                for xx in range(x0, x1 + 1):
                    expect.add((v * tx * ty + yy * tx + xx, int(s)))
    got = {(int(k >> np.uint64(32)), int(vv)) for k, vv in zip(keys, vals)}
    assert got == expect and len(got) == len(keys)
    # the low 32 bits are the FP32 depth of the surfel, rounded as specified
    for k, vv in zip(keys[:50], vals[:50]):
        v = int(k >> np.uint64(32)) // (tx * ty)
        z = np.uint32(k & np.uint64(0xFFFFFFFF)).view(np.float32)
        assert z == pytest.approx(float(preps[v].rec[vv, 11]), rel=1e-6)


# --------------------------------------------------------------------------
# error attribution for pruning (Sec. 4.3, Map Fusion)
# --------------------------------------------------------------------------

def test_max_error_single_surfel_is_max_over_its_footprint():
    """One surfel: the pixels that blend it are exactly those where the
    image's alpha is nonzero, so its attributed error is the maximum of the
    error map there."""
    rng = np.random.default_rng(5)
    view = _view(W=30, H=22, f=28.0)
    cfg = oracle.Config()
    im, p = _render([0.02, 0.01, 2.0], [0.15, 0.09], rng.normal(size=4), 0.8, [0.3, 0.6, 0.9], view, cfg)
    err = rng.uniform(0, 1, (view.height, view.width))
    got = oracle.max_error(p, err)
    cov = im.alpha > 0
    assert cov.sum() > 10
    assert got[0] == err[cov].max()
    assert oracle.max_error(p, np.where(cov, 0.0, err))[0] == 0.0


def test_max_error_respects_occlusion_stop():
    """Two surfels on the optical axis, the nearer one in front; with
    t_min = 0.2 a pixel stops before the back surfel wherever the front one
    has taken T to 1 - a1 and (1 - a1)(1 - a2) < 0.2 (composited here from
    each surfel's own alpha map), so the back surfel is charged only the
    error of pixels where it is actually blended."""
    view = _view(W=24, H=24, f=30.0)
    cfg = oracle.Config(t_min=0.2, sigma_lp=0.0)
    q = [1.0, 0.0, 0.0, 0.0]
    front = ([0.0, 0.0, 2.0], [0.12, 0.12], q, 0.7)
    back = ([0.0, 0.0, 3.0], [0.25, 0.25], q, 0.7)
    a = [_render(m, s_, q_, o, [1, 1, 1], view, oracle.Config(t_min=1e-4, sigma_lp=0.0))[0].alpha
         for m, s_, q_, o in (front, back)]
    blend_f = (a[0] > 0) & ((1 - a[0]) >= cfg.t_min)
    t_after = np.where(blend_f, 1 - a[0], 1.0)
    blend_b = (a[1] > 0) & (t_after * (1 - a[1]) >= cfg.t_min)
    assert (a[1] > 0).sum() > blend_b.sum() > 0  # the stop hides part of the back surfel
    err = np.random.default_rng(6).uniform(0, 1, (24, 24))
    err[12, 12] = 5.0  # under both surfels, where the back one is never blended
    assert not blend_b[12, 12] and blend_f[12, 12]
    _, p = _render(np.array([front[0], back[0]]), np.array([front[1], back[1]]), np.array([q, q]),
                   [0.7, 0.7], np.ones((2, 3)), view, cfg)
    got = oracle.max_error(p, err)
    assert got[0] == err[blend_f].max() == 5.0
    assert got[1] == err[blend_b].max() < 5.0


def test_accum_gate_brute_force():
    """The insertion gate keeps exactly the pixels below the threshold, in
    order (a pixel-by-pixel loop)."""
    rng = np.random.default_rng(8)
    a = rng.uniform(0, 1, 200)
    a[::9] = 0.3
    a[5::13] = np.nan
    expect = [i for i in range(a.size) if a[i] == a[i] and a[i] < 0.3]
    assert list(oracle.accum_gate(a, 0.3)) == expect
    assert oracle.accum_gate(np.zeros(0), 0.5).size == 0


# --------------------------------------------------------------------------
# gradients: FP64 central differences and rigid-motion identities
# --------------------------------------------------------------------------

def _loss_setup(seed, n=48, W=28, H=22, f=26.0, depth_ray=False):
    sc = scenes.random_scene(n=n, width=W, height=H, f=f, seed=seed)
    Rc = Rotation.from_rotvec(np.random.default_rng(seed).normal(size=3) * 0.05).as_matrix()
    sc.views[0].Rt = np.concatenate([Rc, np.array([[0.02], [-0.03], [0.1]])], 1).astype(np.float32)
    cfg = oracle.Config(bg=(0.1, 0.2, 0.3), depth_ray=depth_ray)
    g8 = np.random.default_rng(seed + 99).normal(size=(8, H, W))
    return sc, cfg, g8


def _loss(sc, cfg, g8, cam=None):
    p = oracle.preprocess(sc.means, sc.scales, sc.quats, sc.opacity, sc.rgb, sc.views[0], cfg, cam=cam)
    im = oracle.render(p)
    return float((g8 * im.out).sum()), im.phash


@pytest.mark.parametrize("seed,depth_ray", [(0, False), (1, False), (2, True), (3, True)])
def test_gradient_matches_central_differences(seed, depth_ray):
    """P7: analytic gradient of L = sum(g . outputs) w.r.t. every parameter
    vs FP64 central differences; parameters whose +-h step changes any
    discrete decision (decision hash) are skipped.  Also with the per-pixel
    ray-splat intersection depth."""
    sc, cfg, g8 = _loss_setup(seed, depth_ray=depth_ray)
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    g = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8)
    checked = 0
    worst = 0.0
    for name in ("means", "scales", "quats", "opacity", "rgb"):
        arr = getattr(sc, name)
        an = getattr(g, name).reshape(-1)
        for i in range(arr.size):
            v0 = float(arr.reshape(-1)[i])
            h = 1e-4 * max(1.0, abs(v0))
            res = []
            for sgn in (1, -1):
                s2 = copy.copy(sc)
                a2 = arr.copy()
                a2.reshape(-1)[i] = np.float32(v0 + sgn * h)
                setattr(s2, name, a2)
                L, ph = _loss(s2, cfg, g8)
                res.append((L, float(a2.reshape(-1)[i]), ph))
            if not np.array_equal(res[0][2], res[1][2]):
                continue
            fd = (res[0][0] - res[1][0]) / (res[0][1] - res[1][1])
            err = abs(fd - an[i]) / (abs(an[i]) + 1e-2)
            worst = max(worst, err)
            checked += 1
            assert abs(fd - an[i]) <= 2e-4 * abs(an[i]) + 2e-4, (name, i, an[i], fd)
    assert checked > 300


@pytest.mark.parametrize("seed,depth_ray", [(0, False), (1, False), (2, True)])
def test_pose_gradient_matches_central_differences(seed, depth_ray):
    """P7 for the camera: d L / d xi at xi = 0 for T_cw <- Exp(xi) T_cw,
    xi = (rho, phi); FD through rho -> t + rho and phi -> R(phi) [R | t]."""
    sc, cfg, g8 = _loss_setup(seed, depth_ray=depth_ray)
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    g = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8)
    cam0 = oracle.cam_array(sc.views[0])
    R0 = cam0[6:].reshape(3, 4)[:, :3]
    t0 = cam0[6:].reshape(3, 4)[:, 3]
    checked = 0
    for k in range(6):
        for h in (1e-6, 3e-7, 3e-6, 1e-7):
            Ls = []
            for sgn in (1, -1):
                xi = np.zeros(6); xi[k] = sgn * h
                Rx = Rotation.from_rotvec(xi[3:]).as_matrix()
                R1, t1 = Rx @ R0, Rx @ t0 + xi[:3]
                cam = cam0.copy()
                cam[6:] = np.concatenate([R1, t1[:, None]], 1).reshape(-1)
                Ls.append(_loss(sc, cfg, g8, cam=cam))
            if not np.array_equal(Ls[0][1], Ls[1][1]):
                continue  # a discrete decision flipped inside +-h: try another step
            fd = (Ls[0][0] - Ls[1][0]) / (2 * h)
            assert fd == pytest.approx(g.pose[k], rel=2e-4, abs=1e-3), (k, g.pose[k], fd)
            checked += 1
            break
    assert checked >= 5


def test_rigid_gradient_identities():
    """Because a rigid motion of surfels and camera leaves the image
    unchanged, the surfel gradients must balance the pose gradient:
      sum_s dL/dmu_s = R^T dL/drho,
      sum_s [mu_s x dL/dmu_s + 1/2 ((0,e_k) (x) q_s) . dL/dq_s]_k
          = [R^T (dL/dphi - t x dL/drho)]_k."""
    sc, cfg, g8 = _loss_setup(4, n=96)
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    g = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8)
    R = sc.views[0].Rt[:, :3].astype(np.float64)
    t = sc.views[0].Rt[:, 3].astype(np.float64)
    np.testing.assert_allclose(g.means.sum(0), R.T @ g.pose[:3], rtol=1e-9, atol=1e-9)
    m = sc.means.astype(np.float64)
    q = sc.quats.astype(np.float64)
    lhs = np.cross(m, g.means).sum(0)
    for k in range(3):
        e = np.zeros((sc.n, 4)); e[:, 1 + k] = 1
        lhs[k] += 0.5 * np.sum(_qmul(e, q) * g.quats)
    rhs = R.T @ (g.pose[3:] - np.cross(t, g.pose[:3]))
    # exact for an orthogonal R; the FP32 camera rotation is orthogonal to ~1e-7
    np.testing.assert_allclose(lhs, rhs, rtol=2e-7, atol=1e-8)


# --------------------------------------------------------------------------
# depth distortion (the 2DGS regulariser): closed forms, invariants, FD
# --------------------------------------------------------------------------

def test_distortion_closed_form_stacked_surfels():
    """Surfels parallel to the image plane whose centers project onto the
    same pixel center have alpha = sigma there, so the blended weights are
    w_1 = s_1, w_2 = s_2 (1 - s_1), w_3 = s_3 (1 - s_1)(1 - s_2) in depth
    order, and the distortion at that pixel is
    2 [w_2 w_1 (z_2 - z_1) + w_3 w_1 (z_3 - z_1) + w_3 w_2 (z_3 - z_2)]."""
    view = _view(W=24, H=20, f=30.0)
    ix, iy = 9, 7
    z = np.array([2.0, 2.6, 3.3])
    sig = np.array([0.5, 0.35, 0.8])
    mu = np.stack([(ix + 0.5 - view.cx) * z / view.fx, (iy + 0.5 - view.cy) * z / view.fy, z], 1)
    # listed out of depth order: the sort decides
    order = [2, 0, 1]
    p = oracle.preprocess(mu[order].astype(np.float32), np.full((3, 2), 0.05, np.float32),
                          np.tile(np.array([1.0, 0, 0, 0], np.float32), (3, 1)), sig[order].astype(np.float32),
                          np.ones((3, 3), np.float32), view, oracle.Config())
    d = oracle.render_dist(p)
    s32 = sig.astype(np.float32).astype(np.float64)
    z32 = mu[:, 2].astype(np.float32).astype(np.float64)
    w = np.array([s32[0], s32[1] * (1 - s32[0]), s32[2] * (1 - s32[0]) * (1 - s32[1])])
    want = 2 * (w[1] * w[0] * (z32[1] - z32[0]) + w[2] * w[0] * (z32[2] - z32[0]) + w[2] * w[1] * (z32[2] - z32[1]))
    assert d[iy, ix] == pytest.approx(want, rel=1e-9)
    # one surfel alone has no distortion anywhere
    p1 = oracle.preprocess(mu[:1].astype(np.float32), np.full((1, 2), 0.05, np.float32),
                           np.array([[1.0, 0, 0, 0]], np.float32), sig[:1].astype(np.float32),
                           np.ones((1, 3), np.float32), view, oracle.Config())
    assert np.abs(oracle.render_dist(p1)).max() == 0.0


def test_distortion_invariants():
    """A rigid motion of surfels and camera leaves the distortion unchanged
    (depth differences along the optical axis are preserved); a similarity
    scale s of surfels, their scales and the camera translation scales it by
    s; it is never negative with the center depth (the sort key)."""
    sc, cfg, _ = _loss_setup(5, n=64)
    cfg = oracle.Config()
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    d0 = oracle.render_dist(p)
    assert d0.max() > 1e-3 and d0.min() >= 0.0
    Rg = Rotation.from_rotvec([0.1, -0.2, 0.05]).as_matrix()
    tg = np.array([0.3, -0.1, 0.2])
    R, t = sc.views[0].Rt[:, :3].astype(np.float64), sc.views[0].Rt[:, 3].astype(np.float64)
    means2 = (sc.means.astype(np.float64) @ Rg.T + tg).astype(np.float32)
    qg = Rotation.from_matrix(Rg).as_quat()
    qg = np.array([qg[3], qg[0], qg[1], qg[2]])
    q = sc.quats.astype(np.float64)
    w0, v0 = qg[0], qg[1:]
    qw, qv = q[:, :1], q[:, 1:]
    quats2 = np.concatenate([w0 * qw - qv @ v0[:, None], w0 * qv + qw * v0 + np.cross(v0, qv)], 1).astype(np.float32)
    R2 = R @ Rg.T
    t2 = t - R2 @ tg
    v2 = copy.copy(sc.views[0])
    v2.Rt = np.concatenate([R2, t2[:, None]], 1).astype(np.float32)
    p2 = oracle.preprocess(means2, sc.scales, quats2, sc.opacity, sc.rgb, v2, cfg)
    d2 = oracle.render_dist(p2)
    ok = ((oracle.render(p).pflags | oracle.render(p2).pflags) & oracle.PF_FORWARD) == 0
    np.testing.assert_allclose(d2[ok], d0[ok], atol=1e-5)
    s = 1.7
    v3 = copy.copy(sc.views[0])
    v3.Rt = np.concatenate([R, (s * t)[:, None]], 1).astype(np.float32)
    p3 = oracle.preprocess((s * sc.means.astype(np.float64)).astype(np.float32),
                           (s * sc.scales.astype(np.float64)).astype(np.float32), sc.quats, sc.opacity, sc.rgb, v3, cfg)
    d3 = oracle.render_dist(p3)
    ok = ((oracle.render(p).pflags | oracle.render(p3).pflags) & oracle.PF_FORWARD) == 0
    np.testing.assert_allclose(d3[ok], s * d0[ok], rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("seed,depth_ray", [(0, False), (3, True)])
def test_distortion_gradient_matches_central_differences(seed, depth_ray):
    """Analytic gradient of L = sum(g . outputs) + sum(g_d . distortion)
    w.r.t. every parameter vs FP64 central differences (parameters whose
    step flips a discrete decision are skipped), with the center depth and
    with the per-pixel ray depth."""
    sc, cfg, g8 = _loss_setup(seed, depth_ray=depth_ray)
    gd = np.random.default_rng(seed + 7).normal(size=g8.shape[1:]) * 3.0
    p = oracle.preprocess_scene_view(sc, 0, cfg)
    g = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8, g_dist=gd)

    def loss(s2):
        q = oracle.preprocess(s2.means, s2.scales, s2.quats, s2.opacity, s2.rgb, s2.views[0], cfg)
        im = oracle.render(q)
        return float((g8 * im.out).sum() + (gd * oracle.render_dist(q)).sum()), im.phash
    checked = 0
    for name in ("means", "scales", "quats", "opacity", "rgb"):
        arr = getattr(sc, name)
        an = getattr(g, name).reshape(-1)
        for i in range(arr.size):
            v0 = float(arr.reshape(-1)[i])
            h = 2e-5 * max(1.0, abs(v0))  # the ray depth (1 / c) curves more: a smaller step
            res = []
            for sgn in (1, -1):
                s2 = copy.copy(sc)
                a2 = arr.copy()
                a2.reshape(-1)[i] = np.float32(v0 + sgn * h)
                setattr(s2, name, a2)
                L, ph = loss(s2)
                res.append((L, float(a2.reshape(-1)[i]), ph))
            if not np.array_equal(res[0][2], res[1][2]):
                continue
            fd = (res[0][0] - res[1][0]) / (res[0][1] - res[1][1])
            assert abs(fd - an[i]) <= 2e-4 * abs(an[i]) + 2e-4, (name, i, an[i], fd)
            checked += 1
    assert checked > 300
    # the distortion term is not negligible in this loss
    g0 = oracle.render_bwd(sc.means, sc.scales, sc.quats, p, g8)
    assert np.abs(g.means - g0.means).max() > 1e-2 * np.abs(g0.means).max()


def test_normal_consistency_identity_closed_form():
    """sum_i w_i (1 - n_i.N) = A - N_hat.N: the normal-consistency term of the
    2DGS geometry is a function of the rendered alpha and normal maps.  Three
    surfels of different tilts whose centers project onto one pixel center
    have alpha = sigma there whatever their tilt, so their weights (sigma_1,
    sigma_2 (1 - sigma_1), ...) and normals (turned to face the camera) are
    known in closed form."""
    view = _view(W=24, H=20, f=30.0)
    ix, iy = 9, 7
    z = np.array([2.0, 2.5, 3.1])
    sig = np.array([0.4, 0.55, 0.7], np.float32)
    mu = np.stack([(ix + 0.5 - view.cx) * z / view.fx, (iy + 0.5 - view.cy) * z / view.fy, z], 1).astype(np.float32)
    rots = [Rotation.from_rotvec(r) for r in ([0.3, 0.0, 0.1], [-0.2, 0.4, 0.0], [0.1, -0.1, 0.5])]
    q = np.array([[r.as_quat()[3], *r.as_quat()[:3]] for r in rots], np.float32)
    p = oracle.preprocess(mu, np.full((3, 2), 0.05, np.float32), q, sig, np.ones((3, 3), np.float32), view,
                          oracle.Config())
    o = oracle.render(p).out
    s = sig.astype(np.float64)
    w = np.array([s[0], s[1] * (1 - s[0]), s[2] * (1 - s[0]) * (1 - s[1])])
    n = []
    for qq, m in zip(q.astype(np.float64), mu.astype(np.float64)):
        nv = _rot(qq)[:, 2]
        n.append(-nv if nv @ m > 0 else nv)
    n = np.array(n)
    for N in (np.array([0.2, -0.3, -0.93]), np.array([0.0, 0.0, -1.0]), n[1]):
        N = N / np.linalg.norm(N)
        want = float((w * (1.0 - n @ N)).sum())
        assert o[7, iy, ix] - o[4:7, iy, ix] @ N == pytest.approx(want, abs=1e-9)
