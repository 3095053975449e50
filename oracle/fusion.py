"""TEST INFRASTRUCTURE ONLY -- plain NumPy statements of the per-surfel map
maintenance steps of Flash-Mono's backend (Sec. 4.3, "2DGS Map
Optimization"), for checking the CUDA kernels.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may use this module.

* Adaptive voxelization ("Adaptive Voxelization", the attribute averages
  printed there): a keyframe's per-pixel map is cut into 2x2 blocks of
  primitives; the primitives of a block are replaced by one whose center,
  opacity, colour and scales are the means over the block and whose rotation
  is the normalised sum of the block's quaternions, each first turned to
  the hemisphere of the block's first one (align).  A block whose depth
  variation (largest minus smallest camera-frame depth of its primitives)
  exceeds tau_d keeps its primitives.  Output order: blocks in row-major
  order, each contributing its merged primitive or its own primitives in
  row-major order.
* Sim(3) transforms ("Map Fusion" and "Loop Correction of Gaussian Map"):
  mu' = s R mu + t, r' = q (x) r (Hamilton product, q the quaternion of R),
  and the tangent scales times s (a similarity scales the disk with the
  map; the paper writes the center and rotation only).  A loop correction
  applies, per keyframe, Delta T = T_new T_old^-1 to the primitives bound to
  that keyframe.

Loops are per block / per primitive, for clarity, not speed.
"""
from __future__ import annotations

import numpy as np


def quat_mul(a, b):
    """Hamilton product of (w, x, y, z) quaternions."""
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def quat_to_rot(q):
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def voxelize(means, quats, scales, opacity, rgb, width: int, height: int, tau_d: float):
    """2x2 block merge of a per-pixel map (arrays indexed y * width + x,
    means in the keyframe's camera frame).  Returns the merged map as
    (means, quats, scales, opacity, rgb) in FP64, and for each output
    primitive the index of its block."""
    out = {k: [] for k in ("means", "quats", "scales", "opacity", "rgb", "block")}
    bw, bh = (width + 1) // 2, (height + 1) // 2
    for by in range(bh):
        for bx in range(bw):
            idx = [y * width + x for y in (2 * by, 2 * by + 1) for x in (2 * bx, 2 * bx + 1)
                   if x < width and y < height]
            z = [float(means[i][2]) for i in idx]
            b = by * bw + bx
            if max(z) - min(z) > tau_d:
                for i in idx:
                    out["means"].append(np.asarray(means[i], np.float64))
                    out["quats"].append(np.asarray(quats[i], np.float64))
                    out["scales"].append(np.asarray(scales[i], np.float64))
                    out["opacity"].append(float(opacity[i]))
                    out["rgb"].append(np.asarray(rgb[i], np.float64))
                    out["block"].append(b)
                continue
            n = len(idx)
            q1 = np.asarray(quats[idx[0]], np.float64)
            acc = np.zeros(4)
            for i in idx:
                q = np.asarray(quats[i], np.float64)
                acc += q if np.dot(q, q1) >= 0 else -q
            out["means"].append(sum(np.asarray(means[i], np.float64) for i in idx) / n)
            out["quats"].append(acc / np.linalg.norm(acc))
            out["scales"].append(sum(np.asarray(scales[i], np.float64) for i in idx) / n)
            out["opacity"].append(sum(float(opacity[i]) for i in idx) / n)
            out["rgb"].append(sum(np.asarray(rgb[i], np.float64) for i in idx) / n)
            out["block"].append(b)
    shapes = {"means": (0, 3), "quats": (0, 4), "scales": (0, 2), "rgb": (0, 3)}
    res = []
    for k in ("means", "quats", "scales", "opacity", "rgb"):
        a = np.array(out[k], np.float64)
        res.append(a.reshape(shapes.get(k, (0,))) if a.size == 0 else a)
    return tuple(res), np.array(out["block"], np.int64)


def sim3_apply(means, quats, scales, sim3, index=None):
    """Apply per primitive the similarity sim3[index[i]] (or sim3[0]):
    rows (qw, qx, qy, qz, tx, ty, tz, s).  Returns FP64 copies."""
    sim3 = np.atleast_2d(np.asarray(sim3, np.float64))
    n = len(means)
    m2, q2, s2 = np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 2))
    for i in range(n):
        T = sim3[0 if index is None else int(index[i])]
        q, t, s = T[:4], T[4:7], T[7]
        R = quat_to_rot(q)
        m2[i] = s * (R @ np.asarray(means[i], np.float64)) + t
        q2[i] = quat_mul(q / np.linalg.norm(q), np.asarray(quats[i], np.float64))
        s2[i] = s * np.asarray(scales[i], np.float64)
    return m2, q2, s2


def sim3_compose(a, b):
    """a then b: the row of x -> b(a(x))."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    qa, ta, sa = a[:4] / np.linalg.norm(a[:4]), a[4:7], a[7]
    qb, tb, sb = b[:4] / np.linalg.norm(b[:4]), b[4:7], b[7]
    q = quat_mul(qb, qa)
    t = sb * (quat_to_rot(qb) @ ta) + tb
    return np.concatenate([q, t, [sa * sb]])


def sim3_inverse(a):
    a = np.asarray(a, np.float64)
    q, t, s = a[:4] / np.linalg.norm(a[:4]), a[4:7], a[7]
    qi = np.array([q[0], -q[1], -q[2], -q[3]])
    ti = -(quat_to_rot(qi) @ t) / s
    return np.concatenate([qi, ti, [1.0 / s]])
