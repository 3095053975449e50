"""Seeded synthetic surfel scenes shaped like the paper's workloads.

Flash-Mono's frontend predicts one 2D Gaussian surfel per pixel of each
keyframe, in camera coordinates, and the backend fuses them into a world map
that it renders from the latest keyframes' poses (Sec. 4.1, Eq. "problem
formulation"; Sec. 4.3).  The paper evaluates on ScanNet / BundleFusion indoor
sequences, which are not available here, so these generators stand in for
them: a ray-cast piecewise-planar room (axis-aligned walls plus boxes), one
surfel unprojected at every pixel center, normals from depth gradients,
scales from the pixel footprint, a procedural texture for colour.

This module produces inputs only.  It holds none of the rasterizer's
arithmetic and is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  Everything is drawn from numpy's PCG64 with explicit seeds.
"""
from __future__ import annotations

import dataclasses
import math
import os
from typing import List, Optional

import numpy as np

__all__ = [
    "View", "Scene", "random_scene", "keyframe_scene", "submap_scene",
    "uneven_batch_scene", "large_map_scene", "look_at", "perturb_pose",
]


@dataclasses.dataclass
class View:
    """One camera: pinhole intrinsics, world-to-camera pose and the surfel
    range [surfel_offset, surfel_offset + surfel_count) it renders."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    Rt: np.ndarray  # (3, 4) float32, world -> camera, row-major
    surfel_offset: int = 0
    surfel_count: int = -1  # -1: all surfels from surfel_offset on


@dataclasses.dataclass
class Scene:
    means: np.ndarray    # (N, 3) float32, world
    scales: np.ndarray   # (N, 2) float32, linear tangent scales
    quats: np.ndarray    # (N, 4) float32, (w, x, y, z), any nonzero norm
    opacity: np.ndarray  # (N,) float32 in (0, 1)
    rgb: np.ndarray      # (N, 3) float32 in [0, 1]
    views: List[View]
    target_rgb: Optional[np.ndarray] = None    # (V, 3, H, W) when all views share a size
    target_depth: Optional[np.ndarray] = None  # (V, H, W)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def view_ranges(self):
        out = []
        for v in self.views:
            cnt = self.n - v.surfel_offset if v.surfel_count < 0 else v.surfel_count
            out.append((v.surfel_offset, cnt))
        return out


# --------------------------------------------------------------------------
# small geometry helpers (scene synthesis only)
# --------------------------------------------------------------------------

def _rot_axis_angle(axis: np.ndarray, ang: float) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    x, y, z = axis
    c, s = math.cos(ang), math.sin(ang)
    C = 1 - c
    return np.array([[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
                     [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
                     [z * x * C - y * s, z * y * C + x * s, c + z * z * C]])


def look_at(eye, target, up=(0.0, -1.0, 0.0)) -> np.ndarray:
    """World-to-camera [R|t] (OpenCV axes: x right, y down, z forward)."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([1.0, 0.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    Rcw = np.stack([r, d, f], axis=0)
    return np.concatenate([Rcw, (-Rcw @ eye)[:, None]], axis=1)


def perturb_pose(Rt: np.ndarray, rng: np.random.Generator, max_deg: float, max_trans: float) -> np.ndarray:
    """Rotate the camera by an angle U[0, max_deg] about a uniform axis and
    move its center by a uniform direction times U[0, max_trans]."""
    R = np.asarray(Rt[:, :3], np.float64)
    t = np.asarray(Rt[:, 3], np.float64)
    C = -R.T @ t
    axis = rng.normal(size=3)
    dR = _rot_axis_angle(axis, math.radians(rng.uniform(0, max_deg)))
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    C2 = C + d * rng.uniform(0, max_trans)
    R2 = dR @ R
    return np.concatenate([R2, (-R2 @ C2)[:, None]], axis=1)


def _rotmat_to_quat(R: np.ndarray) -> np.ndarray:
    """(..., 3, 3) rotation matrices -> (..., 4) unit quaternions (w, x, y, z)."""
    R = np.asarray(R, np.float64)
    m00, m01, m02 = R[..., 0, 0], R[..., 0, 1], R[..., 0, 2]
    m10, m11, m12 = R[..., 1, 0], R[..., 1, 1], R[..., 1, 2]
    m20, m21, m22 = R[..., 2, 0], R[..., 2, 1], R[..., 2, 2]
    tr = m00 + m11 + m22
    q = np.zeros(R.shape[:-2] + (4,))
    c0 = tr > 0
    s = np.sqrt(np.maximum(tr + 1.0, 1e-12)) * 2
    q[c0] = np.stack([0.25 * s, (m21 - m12) / s, (m02 - m20) / s, (m10 - m01) / s], -1)[c0]
    c1 = ~c0 & (m00 > m11) & (m00 > m22)
    s = np.sqrt(np.maximum(1.0 + m00 - m11 - m22, 1e-12)) * 2
    q[c1] = np.stack([(m21 - m12) / s, 0.25 * s, (m01 + m10) / s, (m02 + m20) / s], -1)[c1]
    c2 = ~c0 & ~c1 & (m11 > m22)
    s = np.sqrt(np.maximum(1.0 + m11 - m00 - m22, 1e-12)) * 2
    q[c2] = np.stack([(m02 - m20) / s, (m01 + m10) / s, 0.25 * s, (m12 + m21) / s], -1)[c2]
    c3 = ~c0 & ~c1 & ~c2
    s = np.sqrt(np.maximum(1.0 + m22 - m00 - m11, 1e-12)) * 2
    q[c3] = np.stack([(m10 - m01) / s, (m02 + m20) / s, (m12 + m21) / s, 0.25 * s], -1)[c3]
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


# --------------------------------------------------------------------------
# config 0: random surfels in a box in front of one camera
# --------------------------------------------------------------------------

def random_scene(n: int = 4096, width: int = 128, height: int = 96, f: float = 100.0,
                 seed: int = 0, depth_range=(2.0, 4.0), xy_range=1.0,
                 scale_range=(0.01, 0.1), n_views: int = 1, with_target: bool = True) -> Scene:
    """Centers uniform in [-r,r]^2 x [z0,z1] before an identity-pose pinhole
    camera, log-uniform tangent scales, uniform unit quaternions,
    opacity = sigmoid(N(0,1)), RGB uniform [0,1]; a seeded random target."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-xy_range, xy_range, n), rng.uniform(-xy_range, xy_range, n),
                      rng.uniform(depth_range[0], depth_range[1], n)], 1)
    lo, hi = np.log(scale_range[0]), np.log(scale_range[1])
    scales = np.exp(rng.uniform(lo, hi, (n, 2)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(size=n)))
    rgb = rng.uniform(0, 1, (n, 3))
    views = []
    for v in range(n_views):
        Rt = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
        if v > 0:
            Rt = perturb_pose(Rt, rng, 5.0, 0.1)
        views.append(View(width, height, f, f, width / 2.0, height / 2.0, Rt.astype(np.float32)))
    sc = Scene(means.astype(np.float32), scales.astype(np.float32), q.astype(np.float32),
               opacity.astype(np.float32), rgb.astype(np.float32), views, name=f"random{n}")
    if with_target:
        sc.target_rgb = rng.uniform(0, 1, (n_views, 3, height, width)).astype(np.float32)
        sc.target_depth = rng.uniform(depth_range[0], depth_range[1], (n_views, height, width)).astype(np.float32)
    return sc


# --------------------------------------------------------------------------
# rooms: axis-aligned wall rectangles + boxes, ray cast
# --------------------------------------------------------------------------

@dataclasses.dataclass
class _Layout:
    # wall rectangles: axis index, plane coordinate, bounds on the other two axes
    q_axis: np.ndarray
    q_pos: np.ndarray
    q_lo: np.ndarray   # (Q, 2) bounds on the two other axes (in increasing axis order)
    q_hi: np.ndarray
    q_room: np.ndarray
    b_min: np.ndarray  # (B, 3)
    b_max: np.ndarray
    b_room: np.ndarray
    room_gain: np.ndarray  # (R,) colour gain per room
    room_lo: np.ndarray    # (R, 3)
    room_hi: np.ndarray
    tex: dict


def _layout(n_rooms: int, rng: np.random.Generator, boxes_per_room: int = 10,
            gains=None, room_w=5.0, room_d=6.0, room_h=2.8) -> _Layout:
    """Rooms side by side along x, sharing walls that have a doorway."""
    qa, qp, ql, qh, qr = [], [], [], [], []

    def rect(axis, pos, lo, hi, room):
        qa.append(axis); qp.append(pos); ql.append(lo); qh.append(hi); qr.append(room)

    door_w, door_h = 1.0, 2.1
    for r in range(n_rooms):
        x0, x1 = r * room_w, (r + 1) * room_w
        # floor (y=0), ceiling (y=h): axis 1, bounds on (x, z)
        rect(1, 0.0, (x0, 0.0), (x1, room_d), r)
        rect(1, room_h, (x0, 0.0), (x1, room_d), r)
        # front/back walls z=0, z=d: axis 2, bounds on (x, y)
        rect(2, 0.0, (x0, 0.0), (x1, room_h), r)
        rect(2, room_d, (x0, 0.0), (x1, room_h), r)
        # side walls x = x0 (only the first room) and x = x1, with a doorway when shared
        for xw, shared in ((x0, r > 0), (x1, r < n_rooms - 1)):
            if xw == x0 and r > 0:
                continue  # already emitted by the previous room
            if not shared:
                rect(0, xw, (0.0, 0.0), (room_h, room_d), r)
            else:
                zc = room_d * 0.5
                rect(0, xw, (0.0, 0.0), (room_h, zc - door_w / 2), r)
                rect(0, xw, (0.0, zc + door_w / 2), (room_h, room_d), r)
                rect(0, xw, (door_h, zc - door_w / 2), (room_h, zc + door_w / 2), r)
    bmin, bmax, broom = [], [], []
    for r in range(n_rooms):
        x0 = r * room_w
        for _ in range(boxes_per_room):
            sx, sy, sz = rng.uniform(0.2, 1.0), rng.uniform(0.2, 1.4), rng.uniform(0.2, 1.0)
            cx = rng.uniform(x0 + 0.3 + sx / 2, x0 + room_w - 0.3 - sx / 2)
            cz = rng.uniform(0.3 + sz / 2, room_d - 0.3 - sz / 2)
            lo = np.array([cx - sx / 2, 0.0, cz - sz / 2])
            if rng.uniform() < 0.3:  # some boxes float (shelves)
                lo[1] = rng.uniform(0.5, room_h - sy - 0.1) if room_h - sy - 0.1 > 0.5 else 0.0
            bmin.append(lo)
            bmax.append(lo + np.array([sx, sy, sz]))
            broom.append(r)
    if gains is None:
        gains = np.ones(n_rooms)
    tex = dict(freq=rng.uniform(0.8, 4.0, (3, 3, 3)) * rng.choice([-1, 1], (3, 3, 3)),
               phase=rng.uniform(0, 2 * np.pi, (3, 3)), amp=rng.uniform(0.1, 0.25, (3, 3)),
               base=rng.uniform(0.3, 0.7, (max(n_rooms, 1) * (boxes_per_room + 1) + 8, 3)),
               checker=rng.uniform(0.25, 0.6))
    return _Layout(np.array(qa), np.array(qp, np.float64), np.array(ql, np.float64),
                   np.array(qh, np.float64), np.array(qr), np.array(bmin).reshape(-1, 3),
                   np.array(bmax).reshape(-1, 3), np.array(broom, dtype=np.int64),
                   np.asarray(gains, np.float64),
                   np.array([[r * room_w, 0, 0] for r in range(n_rooms)], np.float64),
                   np.array([[(r + 1) * room_w, room_h, room_d] for r in range(n_rooms)], np.float64),
                   tex)


def _raycast(L: _Layout, origin: np.ndarray, dirs: np.ndarray):
    """Nearest hit along each ray: t, hit id (walls first, then boxes + Q)."""
    P = dirs.shape[0]
    tbest = np.full(P, np.inf)
    hid = np.full(P, -1, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        for q in range(L.q_axis.shape[0]):
            a = int(L.q_axis[q])
            o1, o2 = [k for k in range(3) if k != a]
            t = (L.q_pos[q] - origin[a]) / dirs[:, a]
            p1 = origin[o1] + t * dirs[:, o1]
            p2 = origin[o2] + t * dirs[:, o2]
            ok = (t > 1e-6) & (t < tbest) & (p1 >= L.q_lo[q, 0]) & (p1 <= L.q_hi[q, 0]) & \
                 (p2 >= L.q_lo[q, 1]) & (p2 <= L.q_hi[q, 1])
            tbest = np.where(ok, t, tbest)
            hid = np.where(ok, q, hid)
        inv = 1.0 / dirs
        Q = L.q_axis.shape[0]
        for b in range(L.b_min.shape[0]):
            t0 = (L.b_min[b] - origin) * inv
            t1 = (L.b_max[b] - origin) * inv
            tn = np.max(np.minimum(t0, t1), axis=1)
            tf = np.min(np.maximum(t0, t1), axis=1)
            ok = (tf >= tn) & (tn > 1e-6) & (tn < tbest)
            tbest = np.where(ok, tn, tbest)
            hid = np.where(ok, Q + b, hid)
    return tbest, hid


def _texture(L: _Layout, X: np.ndarray, hid: np.ndarray) -> np.ndarray:
    """Sum of three world-space sinusoids per channel plus a checker, with a
    per-object base colour and the room's colour gain."""
    T = L.tex
    Q = L.q_axis.shape[0]
    obj = np.where(hid >= Q, 1 + (hid - Q), 0)
    obj = np.clip(obj, 0, T["base"].shape[0] - 1)
    col = T["base"][obj].copy()
    for ch in range(3):
        for k in range(3):
            col[:, ch] += T["amp"][ch, k] * np.sin(X @ T["freq"][ch, k] + T["phase"][ch, k])
    chk = (np.floor(X[:, 0] * 2) + np.floor(X[:, 1] * 2) + np.floor(X[:, 2] * 2)) % 2
    col *= (1.0 - T["checker"] * 0.5) + T["checker"] * chk[:, None]
    room = np.where(hid >= Q, L.b_room[np.clip(hid - Q, 0, max(L.b_room.shape[0] - 1, 0))] if L.b_room.size else 0,
                    L.q_room[np.clip(hid, 0, Q - 1)])
    col *= L.room_gain[room][:, None]
    return np.clip(col, 0.0, 1.0)


def _render_keyframe(L: _Layout, Rt: np.ndarray, W: int, H: int, f: float):
    """Ray-cast depth (camera z), world hit points and colour per pixel."""
    R = Rt[:, :3].astype(np.float64)
    t = Rt[:, 3].astype(np.float64)
    C = -R.T @ t
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    dc = np.stack([(ii + 0.5 - W / 2) / f, (jj + 0.5 - H / 2) / f, np.ones_like(ii, dtype=np.float64)], -1)
    dw = dc.reshape(-1, 3) @ R  # camera -> world directions (rows times R = R^T d)
    tt, hid = _raycast(L, C, dw)
    depth = np.clip(np.where(np.isfinite(tt), tt, 8.0), 0.5, 8.0)
    X = C + dw * depth[:, None]
    col = _texture(L, X, hid)
    return depth.reshape(H, W), X.reshape(H, W, 3), col.reshape(H, W, 3), dc


def _render_keyframes(L: _Layout, poses, W: int, H: int, f: float):
    """_render_keyframe of every pose, in order; the ray casts run on a
    thread pool (they draw no random numbers, so the results are those of a
    sequential loop)."""
    import concurrent.futures
    workers = max(1, min(len(poses), os.cpu_count() or 1, 16))
    if workers == 1:
        return [_render_keyframe(L, P, W, H, f) for P in poses]
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        return list(ex.map(lambda P: _render_keyframe(L, P, W, H, f), poses))


def _surfels_from_keyframe(L: _Layout, Rt: np.ndarray, W: int, H: int, f: float,
                           rng: np.random.Generator, rendered=None):
    """One surfel per pixel: unprojected center, normal from depth gradients,
    tangent u = camera x projected on the plane, scales = pixel footprint x
    U[0.8, 1.5] per axis, procedural colour, opacity U[0.5, 1].  `rendered`
    is this pose's _render_keyframe result, if already computed."""
    depth, Xw, col, dc = rendered if rendered is not None else _render_keyframe(L, Rt, W, H, f)
    Pc = dc.reshape(H, W, 3) * depth[..., None]
    gx = np.gradient(Pc, axis=1)
    gy = np.gradient(Pc, axis=0)
    n = np.cross(gx, gy)
    nn = np.linalg.norm(n, axis=-1, keepdims=True)
    bad = nn[..., 0] < 1e-12
    n = np.where(bad[..., None], np.array([0.0, 0.0, -1.0]), n / np.maximum(nn, 1e-12))
    flip = np.sum(n * Pc, axis=-1) > 0
    n[flip] *= -1
    ex = np.array([1.0, 0.0, 0.0])
    tu = ex - np.sum(n * ex, -1, keepdims=True) * n
    tn = np.linalg.norm(tu, axis=-1, keepdims=True)
    alt = np.array([0.0, 1.0, 0.0])
    tu2 = alt - np.sum(n * alt, -1, keepdims=True) * n
    tu = np.where(tn > 1e-6, tu / np.maximum(tn, 1e-12), tu2 / np.maximum(np.linalg.norm(tu2, axis=-1, keepdims=True), 1e-12))
    tv = np.cross(n, tu)
    Rcam = np.stack([tu, tv, n], axis=-1)  # columns
    Rwc = Rt[:, :3].astype(np.float64).T
    Rw = np.einsum("ij,hwjk->hwik", Rwc, Rcam)
    q = _rotmat_to_quat(Rw.reshape(-1, 3, 3))
    foot = (depth / f).reshape(-1)
    scales = foot[:, None] * rng.uniform(0.8, 1.5, (H * W, 2))
    opacity = rng.uniform(0.5, 1.0, H * W)
    return (Xw.reshape(-1, 3), scales, q, opacity, col.reshape(-1, 3), depth,
            col.transpose(2, 0, 1))


def _room_camera(L: _Layout, rng: np.random.Generator, room: int = 0) -> np.ndarray:
    lo, hi = L.room_lo[room], L.room_hi[room]
    eye = np.array([rng.uniform(lo[0] + 1.0, hi[0] - 1.0), rng.uniform(1.2, 1.7), rng.uniform(1.0, 2.0)])
    tgt = np.array([rng.uniform(lo[0] + 0.5, hi[0] - 0.5), rng.uniform(0.8, 1.4), hi[2]])
    return look_at(eye, tgt)


def _pack(parts, views, name, targets=None) -> Scene:
    means = np.concatenate([p[0] for p in parts]).astype(np.float32)
    scales = np.concatenate([p[1] for p in parts]).astype(np.float32)
    quats = np.concatenate([p[2] for p in parts]).astype(np.float32)
    opacity = np.concatenate([p[3] for p in parts]).astype(np.float32)
    rgb = np.concatenate([p[4] for p in parts]).astype(np.float32)
    sc = Scene(means, scales, quats, opacity, rgb, views, name=name)
    if targets is not None:
        sc.target_depth = np.stack([t[0] for t in targets]).astype(np.float32)
        sc.target_rgb = np.stack([t[1] for t in targets]).astype(np.float32)
    return sc


# --------------------------------------------------------------------------
# config 1: one keyframe of per-pixel surfels, 8 perturbed views
# --------------------------------------------------------------------------

def keyframe_scene(seed: int = 1001, width: int = 512, height: int = 384, f: float = 400.0,
                   n_views: int = 8, max_deg: float = 5.0, max_trans: float = 0.2) -> Scene:
    """A 5-plane room with 10 boxes, one surfel per pixel of one keyframe,
    rendered from n_views poses perturbed by <= max_deg and <= max_trans."""
    rng = np.random.default_rng(seed)
    L = _layout(1, rng, boxes_per_room=10)
    Rt = _room_camera(L, rng, 0)
    part = _surfels_from_keyframe(L, Rt, width, height, f, rng)
    views, targets = [], []
    for _ in range(n_views):
        Rv = perturb_pose(Rt, rng, max_deg, max_trans)
        views.append(View(width, height, f, f, width / 2.0, height / 2.0, Rv.astype(np.float32)))
        d, _, c, _ = _render_keyframe(L, Rv, width, height, f)
        targets.append((d, c.transpose(2, 0, 1)))
    return _pack([part], views, f"keyframe{width}x{height}", targets)


# --------------------------------------------------------------------------
# config 2: a submap of K keyframes along a smooth trajectory, 3 rooms
# --------------------------------------------------------------------------

def _trajectory(L: _Layout, rng: np.random.Generator, n: int, step: float, deg: float):
    eye = np.array([rng.uniform(1.5, 3.5), rng.uniform(1.3, 1.6), rng.uniform(1.0, 2.0)])
    yaw = rng.uniform(-0.3, 0.3)
    turn = math.radians(deg) * rng.choice([-1.0, 1.0])
    poses = []
    for k in range(n):
        fwd = np.array([math.sin(yaw), 0.0, math.cos(yaw)])
        pitch = 0.08 * math.sin(0.3 * k)
        tgt = eye + fwd + np.array([0.0, pitch, 0.0])
        poses.append(look_at(eye, tgt))
        nxt = eye + step * fwd
        lo, hi = L.room_lo.min(0) + 0.6, L.room_hi.max(0) - 0.6
        if np.any(nxt[[0, 2]] < lo[[0, 2]]) or np.any(nxt[[0, 2]] > hi[[0, 2]]):
            turn = -turn if rng.uniform() < 0.5 else turn
            yaw += 6 * turn
            nxt = eye
        eye = nxt
        yaw += turn
    return poses


def submap_scene(seed: int = 2001, n_keyframes: int = 32, width: int = 512, height: int = 384,
                 f: float = 400.0, n_rooms: int = 3, step: float = 0.05, deg: float = 2.0,
                 gains=None, view_width: Optional[int] = None, view_height: Optional[int] = None,
                 view_f: Optional[float] = None, n_views: Optional[int] = None,
                 with_targets: bool = True) -> Scene:
    """K keyframes x (W*H) per-pixel surfels along a seeded smooth trajectory
    (step metres and deg degrees per frame) through an n_rooms layout.  By
    default every keyframe pose is also a view that renders all surfels."""
    rng = np.random.default_rng(seed)
    L = _layout(n_rooms, rng, boxes_per_room=10, gains=gains)
    poses = _trajectory(L, rng, n_keyframes, step, deg)
    parts = []
    for b in range(0, len(poses), 16):  # ray casts in parallel, 16 keyframes at a time
        batch = poses[b:b + 16]
        for P, r in zip(batch, _render_keyframes(L, batch, width, height, f)):
            parts.append(_surfels_from_keyframe(L, P, width, height, f, rng, rendered=r))
    vw, vh, vf = view_width or width, view_height or height, view_f or f
    vidx = list(range(n_keyframes)) if n_views is None else \
        [int(round(i * (n_keyframes - 1) / max(n_views - 1, 1))) for i in range(n_views)]
    views, targets = [], []
    for k in vidx:
        views.append(View(vw, vh, vf, vf, vw / 2.0, vh / 2.0, poses[k].astype(np.float32)))
        if with_targets:
            if (vw, vh, vf) == (width, height, f):
                targets.append((parts[k][5], parts[k][6]))
            else:
                d, _, c, _ = _render_keyframe(L, poses[k], vw, vh, vf)
                targets.append((d, c.transpose(2, 0, 1)))
    return _pack(parts, views, f"submap{n_keyframes}x{width}x{height}", targets if with_targets else None)


# --------------------------------------------------------------------------
# config 3: many independent submaps of uneven size and image size
# --------------------------------------------------------------------------

IMAGE_SIZES = ((320, 240), (512, 384), (640, 480))


def uneven_batch_scene(seed: int = 3001, n_submaps: int = 64, n_min: int = 50_000,
                       n_max: int = 2_000_000, views_per_submap: int = 4,
                       sizes=IMAGE_SIZES) -> Scene:
    """n_submaps independent submaps, surfel counts log-uniform in
    [n_min, n_max] (subsampled without replacement from per-pixel keyframes
    of that submap's own room), image sizes drawn from `sizes` with the focal
    length scaled to the width (f = 400 * W / 512), views_per_submap views
    each rendering only its own submap's surfel range."""
    rng = np.random.default_rng(seed)
    parts, views = [], []
    off = 0
    for m in range(n_submaps):
        n_m = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        W, H = sizes[int(rng.integers(len(sizes)))]
        f = 400.0 * W / 512.0
        L = _layout(1, rng, boxes_per_room=6)
        base = _room_camera(L, rng, 0)
        pool, got = [], 0
        while got < n_m:
            Pk = perturb_pose(base, rng, 10.0, 0.3)
            p = _surfels_from_keyframe(L, Pk, W, H, f, rng)
            pool.append(p)
            got += p[0].shape[0]
        cat = [np.concatenate([p[i] for p in pool]) for i in range(5)]
        pick = np.sort(rng.choice(cat[0].shape[0], n_m, replace=False))
        parts.append(tuple(c[pick] for c in cat))
        for _ in range(views_per_submap):
            Rv = perturb_pose(base, rng, 5.0, 0.2)
            views.append(View(W, H, f, f, W / 2.0, H / 2.0, Rv.astype(np.float32), off, n_m))
        off += n_m
    return _pack(parts, views, f"uneven{n_submaps}")


# --------------------------------------------------------------------------
# config 4: a large multi-room map
# --------------------------------------------------------------------------

def large_map_scene(seed: int = 4001, n_keyframes: int = 150, n_rooms: int = 6, n_views: int = 16,
                    width: int = 512, height: int = 384, f: float = 400.0,
                    view_width: int = 640, view_height: int = 480, view_f: float = 500.0) -> Scene:
    """n_keyframes x (W*H) surfels over an n_rooms layout with two
    illumination levels (colour gain x0.4 or x1.0 per room), rendered from
    n_views keyframe poses at view_width x view_height."""
    rng = np.random.default_rng(seed)
    gains = rng.choice([0.4, 1.0], n_rooms)
    return submap_scene(seed=seed + 1, n_keyframes=n_keyframes, width=width, height=height, f=f,
                        n_rooms=n_rooms, step=0.12, deg=2.5, gains=gains, view_width=view_width,
                        view_height=view_height, view_f=view_f, n_views=n_views, with_targets=False)

