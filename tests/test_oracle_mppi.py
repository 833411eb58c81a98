"""Pins of the MPPI / iCEM update oracle: a single elite reproduces the best
sample exactly; finite-temperature weights on hand-picked costs give the plan
in closed form; infinite temperature gives the plain mean of brute-force elite
sets (also beyond 32 elites, with ties); the paper's "top 1 %" elite counts;
the warm start is a one-step shift; ties between controllers go to the lower
one; the AR(1) noise has the stated statistics; and repeated iterations lower
the best cost."""
import math

import numpy as np
import pytest

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
    nxt, plan, best = mp.update(costs, mean, seed, S, H, C, sig, rho, 1, 0.1, np.arange(2))
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
    S_c = S // C
    n_e = mp.n_elites(S_c, 0.25)
    assert n_e == 5
    _, plan, _ = mp.update(costs, mean, seed, S, H, C, sig, rho, n_e, 1e30, [0])
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
        mean_next, plan, best = mp.update(costs, mean, 1000 + it, S, H, C, 0.3, 0.5,
                                          mp.n_elites(S // C, 0.05), 0.5, [0])
        bests.append(best[0])
        mean = mean_next  # warm start (the drone is re-planned from the same state)
    assert bests[-1] < bests[0]


def _acts(seed, ids, H, mean_c, sig, rho):
    """Actions of the listed samples (controller mean mean_c [H, 4])."""
    ids = np.asarray(ids, dtype=np.uint64)
    return sa.sampled_actions(seed, ids, H, np.broadcast_to(mean_c, (len(ids), H, 4)), sig, rho)


@pytest.mark.parametrize("swap", [False, True])
def test_two_elites_at_finite_temperature(swap):
    """Costs J1 and J1 + lam ln 3: weights 1 and 1/3, so the plan is exactly
    (3 a1 + a2) / 4 -- a sign error, a missing 1/lam or a wrong normaliser
    gives another value.  Swapping the costs swaps the weights."""
    S, H, seed, sig, rho, lam = 12, 6, 21, 0.4, 0.3, 0.37
    mean = np.random.default_rng(2).uniform(-0.2, 0.2, (1, 1, H, 4))
    costs = np.full((1, S), 50.0)
    lo_s, hi_s = (3, 7) if not swap else (7, 3)
    costs[0, lo_s] = 2.0
    costs[0, hi_s] = 2.0 + lam * math.log(3.0)
    nxt, plan, best = mp.update(costs, mean, seed, S, H, 1, sig, rho, 2, lam, [0])
    a = _acts(seed, [lo_s, hi_s], H, mean[0, 0], sig, rho)
    np.testing.assert_allclose(plan[0], (3 * a[0] + a[1]) / 4, rtol=0, atol=1e-14)
    assert best[0] == 2.0
    np.testing.assert_allclose(nxt[0, 0, :-1], plan[0, 1:], rtol=0, atol=0)


def test_three_elites_at_finite_temperature():
    """Gaps lam ln 2 and lam ln 4 over the best: weights 1, 1/2, 1/4 and the
    normaliser 7/4, so the plan is (4 a1 + 2 a2 + a3) / 7."""
    S, H, seed, sig, rho, lam = 20, 5, 8, 0.3, 0.6, 0.05
    mean = np.random.default_rng(3).uniform(-0.3, 0.3, (1, 1, H, 4))
    costs = np.full((1, S), 9.0)
    costs[0, 5] = 1.0
    costs[0, 1] = 1.0 + lam * math.log(2.0)
    costs[0, 8] = 1.0 + lam * math.log(4.0)
    _, plan, best = mp.update(costs, mean, seed, S, H, 1, sig, rho, 3, lam, [0])
    a = _acts(seed, [5, 1, 8], H, mean[0, 0], sig, rho)
    np.testing.assert_allclose(plan[0], (4 * a[0] + 2 * a[1] + a[2]) / 7, rtol=0, atol=1e-14)


@pytest.mark.parametrize("S_c,n_e", [(5000, 50), (3300, 33), (200, 200)])
def test_elite_sets_beyond_a_warp_match_brute_force(S_c, n_e):
    """Infinite temperature: the plan is the plain mean of the n_e samples that
    come first in (cost, index) order -- costs drawn from few values, so many
    ties sit at the threshold."""
    H, seed, sig, rho = 3, 40, 0.5, 0.2
    rng = np.random.default_rng(S_c)
    costs = np.round(rng.uniform(0, 20, (1, 2 * S_c)), 0)
    mean = rng.uniform(-0.3, 0.3, (1, 2, H, 4))
    _, plan, best = mp.update(costs, mean, seed, 2 * S_c, H, 2, sig, rho, n_e, 1e30, [0])
    jmins = [costs[0, c * S_c:(c + 1) * S_c].min() for c in range(2)]
    c = 0 if jmins[0] <= jmins[1] else 1
    row = costs[0, c * S_c:(c + 1) * S_c]
    el = sorted(range(S_c), key=lambda s: (row[s], s))[:n_e]
    a = _acts(seed, np.asarray(el) + c * S_c, H, mean[0, c], sig, rho)
    np.testing.assert_allclose(plan[0], a.mean(0), rtol=0, atol=1e-14)
    assert best[0] == min(jmins)


def test_equal_best_costs_choose_the_lower_controller():
    S, H, seed = 30, 4, 5
    rng = np.random.default_rng(6)
    costs = rng.uniform(5, 10, (1, S))
    costs[0, 4] = costs[0, 25] = 1.0  # controllers 0 and 2 share the best cost
    mean = rng.uniform(-0.3, 0.3, (1, 3, H, 4))
    nxt, plan, best = mp.update(costs, mean, seed, S, H, 3, 0.3, 0.5, 1, 0.2, [0])
    a = _acts(seed, [4], H, mean[0, 0], 0.3, 0.5)[0]
    np.testing.assert_array_equal(plan[0], a)


def test_top_one_percent_elite_counts():
    """The paper keeps the top 1 % of each controller's samples: 1000 of each
    of five controllers' 100 000 (500k trajectories), 16 of 1600; at least one;
    fractions count as the decimals they are written as."""
    assert mp.n_elites(100_000, 0.01) == 1000
    assert mp.n_elites(1600, 0.01) == 16
    assert mp.n_elites(150, 0.01) == 2
    assert mp.n_elites(50, 0.01) == 1
    assert mp.n_elites(20, 0.1) == 2
    assert mp.n_elites(7, 1.0) == 7
    with pytest.raises(ValueError):
        mp.n_elites(10, 0.0)
    import workloads as W
    for S in (8000, 500_000):
        cfg = W.mppi_workload(n_drones=1, S=S).cfg
        assert cfg["n_elite"] == mp.n_elites(S // cfg["n_ctrl"], 0.01)
