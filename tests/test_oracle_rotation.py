"""Pins of oracle/rotation.py against scipy.spatial.transform (an independent
library implementation of scalar-last quaternions and intrinsic Euler angles)."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import rotation as rot

F64 = torch.float64


def _rand_quats(n, seed):
    return Rotation.random(n, random_state=seed).as_quat()  # scalar-last


def test_quat_to_rot_matches_scipy():
    q = _rand_quats(64, 1)
    R = rot.quat_to_rot(torch.tensor(q, dtype=F64)).numpy()
    np.testing.assert_allclose(R, Rotation.from_quat(q).as_matrix(), atol=1e-14)


def test_quat_mul_is_composition():
    a, b = _rand_quats(32, 2), _rand_quats(32, 3)
    ab = rot.quat_mul(torch.tensor(a, dtype=F64), torch.tensor(b, dtype=F64)).numpy()
    ref = (Rotation.from_quat(a) * Rotation.from_quat(b)).as_matrix()
    np.testing.assert_allclose(Rotation.from_quat(ab).as_matrix(), ref, atol=1e-14)
    # and the product of unit quaternions stays unit
    np.testing.assert_allclose(np.linalg.norm(ab, axis=1), 1.0, atol=1e-15)


def test_quat_mul_identity_and_pure_vector():
    q = torch.tensor(_rand_quats(8, 4), dtype=F64)
    e = torch.tensor([[0.0, 0.0, 0.0, 1.0]], dtype=F64).expand(8, 4)
    assert torch.allclose(rot.quat_mul(q, e), q, atol=0)
    assert torch.allclose(rot.quat_mul(e, q), q, atol=0)
    # q (x) [v, 0] (x) q* rotates v by R(q)
    v = torch.randn(8, 3, dtype=F64)
    qc = q * torch.tensor([-1.0, -1.0, -1.0, 1.0], dtype=F64)
    vq = torch.cat([v, torch.zeros(8, 1, dtype=F64)], -1)
    rv = rot.quat_mul(rot.quat_mul(q, vq), qc)[:, :3]
    Rv = (rot.quat_to_rot(q) @ v[..., None])[..., 0]
    assert torch.allclose(rv, Rv, atol=1e-14)


@pytest.mark.parametrize("seed", [5, 6])
def test_euler_to_rot_matches_scipy_zyx(seed):
    rng = np.random.default_rng(seed)
    rpy = rng.uniform(-1.2, 1.2, (40, 3))
    R = rot.euler_to_rot(torch.tensor(rpy, dtype=F64)).numpy()
    ref = Rotation.from_euler("ZYX", rpy[:, ::-1]).as_matrix()
    np.testing.assert_allclose(R, ref, atol=1e-14)


def test_vee_inverts_hat():
    w = torch.randn(10, 3, dtype=F64)
    z = torch.zeros(10, dtype=F64)
    hat = torch.stack([torch.stack([z, -w[:, 2], w[:, 1]], -1),
                       torch.stack([w[:, 2], z, -w[:, 0]], -1),
                       torch.stack([-w[:, 1], w[:, 0], z], -1)], -2)
    assert torch.equal(rot.vee(hat), w)
    # hat(w) v == w x v
    v = torch.randn(10, 3, dtype=F64)
    assert torch.allclose((hat @ v[..., None])[..., 0], torch.linalg.cross(w, v, dim=-1))
