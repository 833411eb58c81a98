"""Rotations used by the oracle (float64, batched over the leading dimension).

TEST INFRASTRUCTURE ONLY (see the package header).

Quaternions are scalar-last, q = [x, y, z, w], as the paper fixes for the
first-principles model (Materials and Methods, First Principles Modeling,
after Eqs. 1-4).  The product is the Hamilton product.  R(q) maps body-frame
vectors to the world frame.  Euler angles Psi = (roll, pitch, yaw) of the
abstracted model (Abstracted Physics Modeling, Eqs. 7-10) use
R = Rz(yaw) Ry(pitch) Rx(roll) (the paper does not state the convention; the oracle
and the CUDA kernels both read it this way).

Pinned by tests/test_oracle_rotation.py against scipy.spatial.transform
(an independent library implementation of the same conventions).
"""
from __future__ import annotations

import torch


def quat_mul(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Hamilton product a (x) b of scalar-last quaternions [..., 4]."""
    ax, ay, az, aw = a.unbind(-1)
    bx, by, bz, bw = b.unbind(-1)
    x = aw * bx + ax * bw + ay * bz - az * by
    y = aw * by - ax * bz + ay * bw + az * bx
    z = aw * bz + ax * by - ay * bx + az * bw
    w = aw * bw - ax * bx - ay * by - az * bz
    return torch.stack([x, y, z, w], dim=-1)


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix [..., 3, 3] (body -> world) of a scalar-last quaternion.

    The unit-quaternion formula R = (w^2 - |v|^2) I + 2 v v^T + 2 w [v]x is
    applied to q as given; the stepper renormalises q once per step, so RK4
    stage states (|q| = 1 + O(dt^5)) also use it as stored."""
    x, y, z, w = q.unbind(-1)
    r00 = w * w + x * x - y * y - z * z
    r11 = w * w - x * x + y * y - z * z
    r22 = w * w - x * x - y * y + z * z
    r01 = 2 * (x * y - w * z)
    r10 = 2 * (x * y + w * z)
    r02 = 2 * (x * z + w * y)
    r20 = 2 * (x * z - w * y)
    r12 = 2 * (y * z - w * x)
    r21 = 2 * (y * z + w * x)
    return torch.stack([torch.stack([r00, r01, r02], -1),
                        torch.stack([r10, r11, r12], -1),
                        torch.stack([r20, r21, r22], -1)], dim=-2)


def rot_x(a: torch.Tensor) -> torch.Tensor:
    c, s = torch.cos(a), torch.sin(a)
    o, z = torch.ones_like(a), torch.zeros_like(a)
    return torch.stack([torch.stack([o, z, z], -1), torch.stack([z, c, -s], -1),
                        torch.stack([z, s, c], -1)], -2)


def rot_y(a: torch.Tensor) -> torch.Tensor:
    c, s = torch.cos(a), torch.sin(a)
    o, z = torch.ones_like(a), torch.zeros_like(a)
    return torch.stack([torch.stack([c, z, s], -1), torch.stack([z, o, z], -1),
                        torch.stack([-s, z, c], -1)], -2)


def rot_z(a: torch.Tensor) -> torch.Tensor:
    c, s = torch.cos(a), torch.sin(a)
    o, z = torch.ones_like(a), torch.zeros_like(a)
    return torch.stack([torch.stack([c, -s, z], -1), torch.stack([s, c, z], -1),
                        torch.stack([z, z, o], -1)], -2)


def euler_to_rot(psi: torch.Tensor) -> torch.Tensor:
    """R = Rz(yaw) @ Ry(pitch) @ Rx(roll) for psi = [..., (roll, pitch, yaw)]."""
    return rot_z(psi[..., 2]) @ rot_y(psi[..., 1]) @ rot_x(psi[..., 0])


def vee(S: torch.Tensor) -> torch.Tensor:
    """Vector of a skew-symmetric matrix: vee([w]x) = w."""
    return torch.stack([S[..., 2, 1], S[..., 0, 2], S[..., 1, 0]], dim=-1)
