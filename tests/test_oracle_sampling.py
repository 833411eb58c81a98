"""Pins of the sampling oracle: Philox4x32-10 against its published
known-answer vectors, the Box-Muller map, and the rollout cost against a
closed form and a scalar brute-force evaluation."""
import math
import os

import numpy as np
import torch

import workloads as W
from oracle import physics as ph
from oracle import sampling as sa

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = sa.philox4x32_10(np.array(v[0:4], dtype=np.uint64), np.array(v[4:6], dtype=np.uint64))
        assert [int(o) for o in out] == v[6:10]


def test_philox_vectorised_matches_scalar_calls():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, (50, 4), dtype=np.uint64)
    key = rng.integers(0, 2**32, (50, 2), dtype=np.uint64)
    batch = sa.philox4x32_10(ctr, key)
    for i in range(50):
        assert np.array_equal(batch[i], sa.philox4x32_10(ctr[i], key[i]))


def test_uniform24_is_exact_and_open_interval():
    w = np.array([0, 0x1FF, 0x200, 0xFFFFFFFF], dtype=np.uint32)
    u = sa.uniform24(w)
    assert u[0] == 2.0 ** -24 and u[1] == u[0]
    assert u[2] == 3 * 2.0 ** -24
    assert u[3] == 1.0 - 2.0 ** -24
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)


def test_normals_moments_and_determinism():
    ids = np.arange(200_000, dtype=np.uint64) * np.uint64(977) + np.uint64(2**40)
    z = sa.normals(1234567890123, ids, 3)
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    # the four columns are uncorrelated
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(4)).max() < 4 / math.sqrt(len(ids))
    assert np.array_equal(sa.normals(1234567890123, ids[:10], 3), z[:10])
    assert not np.array_equal(sa.normals(1234567890123, ids[:10], 4), z[:10])


def _tiny():
    P = W.crazyflie_params()
    x0 = np.zeros((3, 20))
    x0[:, 0:3] = [[0.0, 0.0, 1.0], [0.5, -0.5, 2.0], [1.0, 1.0, 1.5]]
    x0[:, 6] = 1.0
    x0[:, 13:17] = W.hover_rpm(P)
    goals = np.array([[1.0, 0.0, 1.0], [0.0, 0.0, 3.0]])
    world = np.array([0, 0, 1])
    obs = np.array([[0.0, 0.1, 1.0, 0.3], [0.5, -0.5, 2.2, 0.25], [3.0, 3.0, 3.0, 0.2]])
    return P, x0, goals, world, obs


def test_zero_noise_hover_cost_closed_form():
    """sigma = 0 and a zero nominal: the drones hover in place, so the cost is
    H (|p0 - g| + w_obs sum_o max(0, r_o - |p0 - c_o|))."""
    P, x0, goals, world, obs = _tiny()
    H, S = 20, 4
    drones = np.repeat(np.arange(3), S)
    samples = np.tile(np.arange(S), 3)
    c = sa.rollout_cost(x0, goals, obs, P, S, H, 1 / 500, 0.0, 99, 1000.0, drones, samples, world)
    p0 = x0[drones, 0:3]
    g = goals[world[drones]]
    pen = np.clip(obs[None, :, 3] - np.linalg.norm(p0[:, None] - obs[None, :, 0:3], axis=-1), 0, None)
    expect = H * (np.linalg.norm(p0 - g, axis=-1) + 1000.0 * pen.sum(-1))
    np.testing.assert_allclose(c, expect, rtol=1e-11)
    assert pen.sum() > 0  # the instance does exercise the obstacle hinge


def test_cost_matches_scalar_brute_force():
    """A scalar re-evaluation: one (drone, sample) pair stepped one drone at a
    time with explicit loops over the four Box-Muller outputs and the
    obstacles."""
    P, x0, goals, world, obs = _tiny()
    H, S, seed, sigma = 8, 5, 2**33 + 17, 0.3
    d, s = 1, 3
    c = sa.rollout_cost(x0, goals, obs, P, S, H, 1 / 500, sigma, seed, 1000.0, [d], [s], world)[0]
    sid = d * S + s
    key = (seed & 0xFFFFFFFF, seed >> 32)
    x = torch.tensor(x0[d:d + 1], dtype=torch.float64)
    Pb = ph.param_batch([P], [0])
    total = 0.0
    for k in range(H):
        w = sa.philox4x32_10(np.array([sid & 0xFFFFFFFF, sid >> 32, k, 0], dtype=np.uint64),
                             np.array(key, dtype=np.uint64))
        u = [((int(wi) >> 9) + 0.5) / 2**23 for wi in w]
        z = []
        for u1, u2 in ((u[0], u[1]), (u[2], u[3])):
            r = math.sqrt(-2 * math.log(u1))
            z += [r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)]
        a = torch.tensor([[min(1.0, max(-1.0, sigma * zi)) for zi in z]], dtype=torch.float64)
        x = ph.step(x, a, Pb, 1 / 500, ph.RK4, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        p = x[0, 0:3].numpy()
        total += math.dist(p, goals[world[d]])
        for o in obs:
            total += 1000.0 * max(0.0, o[3] - math.dist(p, o[0:3]))
    assert abs(total - c) < 1e-12 * max(1.0, abs(c))
