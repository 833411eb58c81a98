"""Pins of the MPPI / iCEM update oracle: a single elite reproduces the best
sample exactly, infinite temperature gives the plain elite mean, the warm start
is a one-step shift, the AR(1) noise has the stated statistics, and repeated
iterations lower the best cost."""
import numpy as np

import workloads as W
from oracle import mppi as mp
from oracle import sampling as sa


def _setup(n=2, S=60, H=12, n_ctrl=3, seed=3):
    rng = np.random.default_rng(seed)
    P = W.crazyflie_params()
    x0 = np.zeros((n, 20))
    x0[:, 0:3] = rng.uniform(-1, 1, (n, 3)) + [0, 0, 1.5]
    x0[:, 6] = 1.0
    x0[:, 13:17] = W.hover_rpm(P)
    goals = x0[:, 0:3] + rng.uniform(-0.5, 0.5, (n, 3))
    mean = rng.uniform(-0.3, 0.3, (n, n_ctrl, H, 4))
    obs = np.array([[x0[0, 0] + 0.2, x0[0, 1], x0[0, 2], 0.15]])
    return P, x0, goals, mean, obs


def test_single_elite_is_the_best_sample():
    P, x0, goals, mean, obs = _setup()
    S, H, C, seed, sig, rho = 60, 12, 3, 77, 0.3, 0.4
    costs = mp.sample_costs(x0, goals, obs, P, S, H, C, 0.02, sig, rho, seed, 1000.0, mean,
                            np.arange(2), np.arange(2))
    nxt, plan, best = mp.update(costs, mean, seed, S, H, C, sig, rho, 1e-6, 0.1, np.arange(2))
    S_c = S // C
    for i in range(2):
        s = int(np.argmin(costs[i]))  # overall best sample (lowest index on ties)
        c = s // S_c
        assert best[i] == costs[i, s]
        a = sa.sampled_actions(seed, [np.uint64(i * S + s)], H, mean[i, c][None], sig, rho)[0]
        np.testing.assert_array_equal(plan[i], a)
        # warm start: the best controller's next mean is the plan shifted by one step
        np.testing.assert_array_equal(nxt[i, c, :-1], plan[i, 1:])
        np.testing.assert_array_equal(nxt[i, c, -1], plan[i, -1])


def test_infinite_temperature_is_the_elite_mean():
    P, x0, goals, mean, obs = _setup(n=1, H=8, n_ctrl=2)
    S, H, C, seed, sig, rho = 40, 8, 2, 5, 0.2, 0.0
    costs = mp.sample_costs(x0, goals, obs, P, S, H, C, 0.02, sig, rho, seed, 1000.0, mean, [0], [0])
    frac = 0.25
    _, plan, _ = mp.update(costs, mean, seed, S, H, C, sig, rho, frac, 1e30, [0])
    S_c = S // C
    n_e = mp.n_elites(S_c, frac)
    jmins = [np.sort(costs[0, c * S_c:(c + 1) * S_c])[0] for c in range(C)]
    c = int(np.argmin(jmins))
    el = np.argsort(costs[0, c * S_c:(c + 1) * S_c], kind="stable")[:n_e] + c * S_c
    acts = sa.sampled_actions(seed, el.astype(np.uint64), H, np.broadcast_to(mean[0, c], (n_e, H, 4)),
                              sig, rho)
    np.testing.assert_allclose(plan[0], acts.mean(0), rtol=0, atol=1e-15)


def test_ar1_noise_statistics():
    ids = np.arange(100_000, dtype=np.uint64) + np.uint64(12345)
    sig, rho = 1e-3, 0.7  # small sigma: no clipping, eps = a / sigma
    a = sa.sampled_actions(99, ids, 6, None, sig, rho) / sig
    for k in range(6):
        assert abs(a[:, k].var() - 1.0) < 0.02
    c = np.mean([np.corrcoef(a[:, k, j], a[:, k + 1, j])[0, 1] for k in range(5) for j in range(4)])
    assert abs(c - rho) < 0.01


def test_iterations_lower_the_best_cost():
    P, x0, goals, mean, obs = _setup(n=1, H=15, n_ctrl=2)
    mean[:] = 0.0
    S, H, C = 100, 15, 2
    bests = []
    for it in range(6):
        costs = mp.sample_costs(x0, goals, obs[:0], P, S, H, C, 0.02, 0.3, 0.5, 1000 + it, 0.0, mean,
                                [0], [0])
        mean_next, plan, best = mp.update(costs, mean, 1000 + it, S, H, C, 0.3, 0.5, 0.05, 0.5, [0])
        bests.append(best[0])
        mean = mean_next  # warm start (the drone is re-planned from the same state)
    assert bests[-1] < bests[0]
