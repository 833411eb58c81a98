"""Pins of the depth ray-cast oracle by closed forms."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import raycast as rc


def _pose(p, rpy_deg=(0, 0, 0)):
    q = Rotation.from_euler("ZYX", [rpy_deg[2], rpy_deg[1], rpy_deg[0]], degrees=True).as_quat()
    return np.concatenate([p, q])


def test_ray_directions_are_unit_and_symmetric():
    d = rc.ray_directions(8, 12, math.radians(90), math.radians(60))
    np.testing.assert_allclose(np.linalg.norm(d, axis=-1), 1.0, rtol=1e-15)
    np.testing.assert_allclose(d[:, ::-1, 1], -d[:, :, 1], atol=1e-15)
    np.testing.assert_allclose(d[::-1, :, 2], -d[:, :, 2], atol=1e-15)
    # the corner ray leaves at the half field of view in each image direction
    # column 0 looks towards body +y (left), row 0 towards +z (up)
    assert abs(d[0, 0, 1] / d[0, 0, 0] - math.tan(math.radians(45)) * (1 - 1 / 12)) < 1e-15
    assert abs(d[0, 0, 2] / d[0, 0, 0] - math.tan(math.radians(30)) * (1 - 1 / 8)) < 1e-15


def test_downward_camera_over_ground():
    """Pitched 90 deg down at height h: the range to z = 0 is h / cos(angle
    between the ray and the vertical)."""
    h = 2.5
    img = rc.render([_pose([0.3, -0.2, h], (0, 90, 0))], [], [], 16, 16, math.radians(60),
                    math.radians(60), 100.0)[0]
    d = rc.ray_directions(16, 16, math.radians(60), math.radians(60))
    np.testing.assert_allclose(img, h / d[..., 0], rtol=1e-13)


def test_sphere_and_box_straight_ahead_and_miss():
    """Odd image sizes put a ray exactly on the optical axis."""
    pose = _pose([0.0, 0.0, 1.0])
    img = rc.render([pose], [[3.0, 0.0, 1.0, 0.5]], [], 9, 9, math.radians(40), math.radians(40),
                    20.0)[0]
    assert abs(img[4, 4] - 2.5) < 1e-14
    img = rc.render([pose], [], [[4.0, -1.0, 0.5, 5.0, 1.0, 1.5]], 9, 9, math.radians(40),
                    math.radians(40), 20.0)[0]
    assert abs(img[4, 4] - 4.0) < 1e-14
    # looking up at the sky: nothing but max range
    img = rc.render([_pose([0, 0, 1.0], (0, -80, 0))], [], [], 5, 5, math.radians(20),
                    math.radians(20), 7.0)[0]
    assert np.all(img == 7.0)


def test_camera_inside_a_sphere_sees_its_shell():
    img = rc.render([_pose([1.0, 1.0, 5.0], (10, 20, 30))], [[1.0, 1.0, 5.0, 0.7]], [], 6, 6,
                    math.radians(90), math.radians(90), 50.0)[0]
    np.testing.assert_allclose(img, 0.7, rtol=1e-14)
