"""The step kernels' attitude interface works on quaternions: the command as
qd = qz(yaw) (x) qy(pitch) (x) qx(roll) from half angles, scaled by 2, and the
geometric controller's 2 e_R = vee(Rd^T R - R^T Rd) as w v of qd* (x) q.  These
checks pin that restatement to the oracle's matrix definitions (euler_to_rot,
quat_to_rot, attitude_torque's vee form), including quaternions that are not of
unit norm, as between renormalisations."""
import math

import numpy as np
import torch

from oracle.rotation import euler_to_rot, quat_to_rot, vee


def _half_angle_command(ang):
    """Twice the desired quaternion (x, y, z, w), as the kernels form it."""
    hr, hp, hy = 0.5 * ang[:, 0], 0.5 * ang[:, 1], 0.5 * ang[:, 2]
    sr, cr, sp, cp, sy, cy = (torch.sin(hr), torch.cos(hr), torch.sin(hp), torch.cos(hp),
                              torch.sin(hy), torch.cos(hy))
    a, b, c, d = 2 * cp * cy, 2 * sp * sy, 2 * sp * cy, 2 * cp * sy
    return torch.stack([sr * a - cr * b, cr * c + sr * d, cr * d - sr * c, cr * a + sr * b], -1)


def _error2_q(q, qd2):
    qx, qy, qz, qw = q.unbind(-1)
    dx, dy, dz, dw = qd2.unbind(-1)
    vx = dw * qx - qw * dx - dy * qz + dz * qy
    vy = dw * qy - qw * dy - dz * qx + dx * qz
    vz = dw * qz - qw * dz - dx * qy + dy * qx
    w = dw * qw + dx * qx + dy * qy + dz * qz
    return torch.stack([w * vx, w * vy, w * vz], -1)


def _cases(n=2000, seed=0):
    g = torch.Generator().manual_seed(seed)
    ang = (torch.rand(n, 3, generator=g, dtype=torch.float64) * 2 - 1) * math.pi
    ang[: n // 2] *= math.pi / 6 / math.pi  # the action range, and beyond it
    q = torch.randn(n, 4, generator=g, dtype=torch.float64)
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    q = q * (1 + 1e-3 * torch.randn(n, 1, generator=g, dtype=torch.float64))  # off unit norm
    return ang, q


def test_half_angle_quaternion_is_the_euler_rotation():
    ang, _ = _cases()
    qd2 = _half_angle_command(ang)
    np.testing.assert_allclose(torch.linalg.vector_norm(qd2, dim=-1).numpy(), 2.0, atol=1e-12)
    # quat_to_rot's quadratic form scales with |q|^2 = 4
    np.testing.assert_allclose((quat_to_rot(qd2) / 4).numpy(), euler_to_rot(ang).numpy(), atol=1e-12)


def test_quaternion_error_equals_the_matrix_vee():
    ang, q = _cases(seed=1)
    Rd, R = euler_to_rot(ang), quat_to_rot(q)
    ref = vee(Rd.transpose(-1, -2) @ R - R.transpose(-1, -2) @ Rd)
    got = _error2_q(q, _half_angle_command(ang))
    np.testing.assert_allclose(got.numpy(), ref.numpy(), atol=1e-12)
    assert ref.abs().max() > 0.5  # large errors, not only near the set point


def test_sign_and_axis_of_the_error():
    """Drone rolled by +0.1 rad against a level command: e_R points along +x
    (vee(Rd^T R - R^T Rd) = 2 sin(0.1) e_x); a mistaken conjugate would flip it."""
    ang = torch.zeros(1, 3, dtype=torch.float64)
    q = torch.tensor([[math.sin(0.05), 0.0, 0.0, math.cos(0.05)]], dtype=torch.float64)
    got = _error2_q(q, _half_angle_command(ang))[0].numpy()
    np.testing.assert_allclose(got, [2 * math.sin(0.1), 0.0, 0.0], atol=1e-15)
