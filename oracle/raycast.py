"""FP64 oracle of batched depth rendering by ray casting.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper renders depth images in parallel with MJX's ray-cast pipeline
(Results, Computation Performance: 64x64 rays across 1024 environments;
Materials and Methods, Visualization and Collision Checking).  The reading adopted
here: each drone carries a pinhole depth camera at its centre looking along
body +x (image columns run from body +y to -y, rows from body +z to -z); pixel
(row i, column j) of an H x W image casts the ray
    d_body = normalise(1, -tan(hfov/2) (2 (j + 0.5) / W - 1),
                          -tan(vfov/2) (2 (i + 0.5) / H - 1))
rotated to the world by R(q); the depth is the distance to the first hit among
spheres (centre, radius), axis-aligned boxes (min corner, max corner) and the
ground plane z = 0, or max_range when nothing is hit closer.

Parity status: a reading (the paper's camera model and scene are MJX's);
pinned in tests/test_oracle_raycast.py by closed forms: a downward camera over
the ground (range h / cos of the ray angle), a sphere and a box straight
ahead, a miss, and the camera inside a sphere.
"""
from __future__ import annotations

import numpy as np

from .rotation import quat_to_rot
import torch


def ray_directions(H: int, W: int, hfov: float, vfov: float) -> np.ndarray:
    """Body-frame unit ray directions [H, W, 3]."""
    j = (np.arange(W) + 0.5) / W * 2.0 - 1.0
    i = (np.arange(H) + 0.5) / H * 2.0 - 1.0
    d = np.stack(np.broadcast_arrays(np.ones((H, W)), -np.tan(hfov / 2) * j[None, :],
                                     -np.tan(vfov / 2) * i[:, None]), axis=-1)
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def hit_sphere(o, d, c, r):
    """Nearest t >= 0 of |o + t d - c| = r (|d| = 1), inf if none."""
    oc = o - c
    b = (oc * d).sum(-1)
    cc = (oc * oc).sum(-1) - r * r
    disc = b * b - cc
    s = np.sqrt(np.maximum(disc, 0.0))
    t0, t1 = -b - s, -b + s
    t = np.where(t0 >= 0, t0, t1)
    return np.where((disc >= 0) & (t >= 0), t, np.inf)


def hit_box(o, d, lo, hi):
    """Slab test: entry distance of the ray into [lo, hi] (0 if inside), inf if none."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta = (lo - o) * inv
        tb = (hi - o) * inv
    tmin = np.nanmax(np.minimum(ta, tb), axis=-1)
    tmax = np.nanmin(np.maximum(ta, tb), axis=-1)
    t = np.maximum(tmin, 0.0)
    return np.where(tmax >= t, t, np.inf)


def hit_ground(o, d):
    with np.errstate(divide="ignore", invalid="ignore"):
        t = -o[..., 2] / d[..., 2]
    return np.where((d[..., 2] < 0) & (t >= 0), t, np.inf)


def render(poses, spheres, boxes, H: int, W: int, hfov: float, vfov: float, max_range: float):
    """Depth images [n, H, W] for drone poses [n, 7] = (p, q scalar-last)."""
    poses = np.asarray(poses, dtype=np.float64)
    R = quat_to_rot(torch.tensor(poses[:, 3:7])).numpy()
    db = ray_directions(H, W, hfov, vfov)
    out = np.empty((len(poses), H, W))
    for e in range(len(poses)):
        d = db @ R[e].T
        o = np.broadcast_to(poses[e, 0:3], d.shape)
        t = hit_ground(o, d)
        for s in np.asarray(spheres).reshape(-1, 4):
            t = np.minimum(t, hit_sphere(o, d, s[0:3], s[3]))
        for b in np.asarray(boxes).reshape(-1, 6):
            t = np.minimum(t, hit_box(o, d, b[0:3], b[3:6]))
        out[e] = np.minimum(t, max_range)
    return out
