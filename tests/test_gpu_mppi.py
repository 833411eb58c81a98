"""GPU parity of the MPPI / iCEM iteration: sampling costs against the FP64
oracle, and the update (elites, exponential weights, warm start, best
controller) against the oracle given the same costs -- the elite selection is
an integer decision, so both sides take it on identical inputs.  Both update
kernels are covered: the warp path (small controllers) and the cluster path
(more than 2048 samples or 32 elites per controller), the latter up to the
paper's size, 500k trajectories in five controllers of 100 000 with the top
1 % (1000) as elites."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mppi as mp
from oracle import sampling as sa
from paper_2606_01478_b300 import RK4, Sim

pytestmark = pytest.mark.gpu


def _seed(s):
    return torch.tensor([s], dtype=torch.int64, device="cuda")


def _setup(n_w, dt=1 / 50, seed=3):
    rng = np.random.default_rng(seed)
    P = W.crazyflie_params()
    n = int(sum(n_w))
    x0 = W.fp_state(rng.uniform([-1, -1, 1], [1, 1, 2], (n, 3)), np.zeros((n, 3)),
                    rng.uniform(-0.5, 0.5, (n, 3)), np.zeros((n, 3)), np.full((n, 4), W.hover_rpm(P)))
    goals = rng.uniform([-1, -1, 1], [1, 1, 2], (len(n_w), 3))
    obs = np.concatenate([x0[np.arange(3) % n, 0:3] + rng.uniform(-0.2, 0.2, (3, 3)),
                          np.full((3, 1), 0.15)], 1)
    sim = Sim.batched(np.asarray(n_w), np.zeros(len(n_w), np.int32), RK4, dt)
    sim.set_params(P)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    return P, x0, goals, obs, sim


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_mppi_iteration_parity_and_warm_start():
    n_w = [2, 5, 1]
    P, x0, goals, obs, sim = _setup(n_w)
    n = sum(n_w)
    world = np.repeat(np.arange(3), n_w)
    cfg = dict(S=60, H=12, n_ctrl=3, sigma=0.3, rho=0.5, n_elite=2, lam=0.5, w_obs=1000.0)
    mean0 = np.random.default_rng(4).uniform(-0.3, 0.3, (n, 3, 12, 4))
    mean = torch.tensor(mean0, dtype=torch.float32, device="cuda")
    g = torch.tensor(goals, dtype=torch.float32, device="cuda")
    mean_in = _f32(mean0)
    for it, seed in enumerate((11, 12)):  # two iterations: the second starts from the warm start
        plan, cost, best = sim.mppi_iteration(cfg, _seed(seed), g, obs, mean)
        c_gpu = cost.cpu().numpy().astype(np.float64)
        c_ref = mp.sample_costs(_f32(x0), _f32(goals), _f32(obs), P, 60, 12, 3, 1 / 50, 0.3, 0.5, seed,
                                1000.0, mean_in, world, np.arange(n))
        np.testing.assert_allclose(c_gpu, c_ref, rtol=1e-4, atol=1e-4)
        nxt, plan_ref, best_ref = mp.update(c_gpu, mean_in, seed, 60, 12, 3, 0.3, 0.5, 2, 0.5,
                                            np.arange(n))
        np.testing.assert_array_equal(best.cpu().numpy().astype(np.float64), best_ref)
        np.testing.assert_allclose(plan.cpu().numpy(), plan_ref, rtol=0, atol=2e-5)
        np.testing.assert_allclose(mean.cpu().numpy(), nxt, rtol=0, atol=2e-5)
        mean_in = mean.cpu().numpy().astype(np.float64)


def test_single_controller_white_noise_matches_sampling_entry_point():
    """n_ctrl = 1, rho = 0 and a per-drone mean equal to the world's nominal
    sequence: the MPPI sampling costs equal sim_sample_rollouts' costs."""
    n_w = [3, 4]
    P, x0, goals, obs, sim = _setup(n_w, seed=5)
    H, S = 10, 32
    nom = np.random.default_rng(1).uniform(-0.2, 0.2, (2, H, 4)).astype(np.float32)
    g = torch.tensor(goals, dtype=torch.float32, device="cuda")
    ref = sim.sample_rollouts(S, H, _seed(99), 0.25, g, obs, 1000.0,
                              nominal=torch.tensor(nom, device="cuda")).clone()
    mean = torch.tensor(np.repeat(nom, n_w, axis=0)[:, None], device="cuda").contiguous()
    cfg = dict(S=S, H=H, n_ctrl=1, sigma=0.25, rho=0.0, n_elite=2, lam=1.0, w_obs=1000.0)
    _, cost, best = sim.mppi_iteration(cfg, _seed(99), g, obs, mean)
    assert torch.equal(cost, ref)
    assert torch.equal(best, ref.min(dim=1).values)


def test_mppi_workload_runs_and_improves():
    """The paper-scale MPPI workload (64 drones x 8000 samples, 5 controllers):
    costs finite, and re-planning from the same states lowers the mean best cost."""
    wl = W.mppi_workload(n_drones=16, S=2000)
    sim = Sim.batched(wl.n_per_world, np.zeros(len(wl.n_per_world), np.int32), RK4, wl.dt)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
    c = wl.cfg
    mean = torch.zeros(16, c["n_ctrl"], c["H"], 4, device="cuda")
    g = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    bests = []
    for it in range(6):
        _, cost, best = sim.mppi_iteration(c, _seed(wl.seed + it), g, wl.obstacles, mean)
        assert torch.isfinite(cost).all()
        bests.append(best.mean().item())
    assert bests[-1] < bests[0]


def _cluster_case(n_w, S, C, n_e, H, seed_base, sample_costs=256, iters=2, lam=0.05):
    P, x0, goals, obs, sim = _setup(n_w, seed=seed_base)
    n = int(sum(n_w))
    world = np.repeat(np.arange(len(n_w)), n_w)
    cfg = dict(S=S, H=H, n_ctrl=C, sigma=0.3, rho=0.7, n_elite=n_e, lam=lam, w_obs=1000.0)
    rng = np.random.default_rng(seed_base + 1)
    mean0 = rng.uniform(-0.3, 0.3, (n, C, H, 4))
    mean = torch.tensor(mean0, dtype=torch.float32, device="cuda")
    g = torch.tensor(goals, dtype=torch.float32, device="cuda")
    mean_in = _f32(mean0)
    S_c = S // C
    for it in range(iters):  # the second iteration starts from the warm start
        seed = 100 + seed_base + it
        plan, cost, best = sim.mppi_iteration(cfg, _seed(seed), g, obs, mean)
        c_gpu = cost.cpu().numpy().astype(np.float64)
        # sampled costs against the oracle (every controller, first and last samples included)
        d = rng.integers(0, n, sample_costs)
        s = rng.integers(0, S, sample_costs)
        s[:2 * C] = np.concatenate([np.arange(C) * S_c, np.arange(1, C + 1) * S_c - 1])
        ids = d.astype(np.uint64) * np.uint64(S) + s.astype(np.uint64)
        acts = sa.sampled_actions(seed, ids, H, mean_in[d, s // S_c], 0.3, 0.7)
        ref = sa.cost_of_actions(_f32(x0)[d], _f32(goals)[world[d]], _f32(obs), P, acts, 1 / 50,
                                 1000.0, RK4)
        np.testing.assert_allclose(c_gpu[d, s], np.ravel(ref), rtol=1e-4, atol=1e-4)
        nxt, plan_ref, best_ref = mp.update(c_gpu, mean_in, seed, S, H, C, 0.3, 0.7, n_e, lam,
                                            np.arange(n))
        np.testing.assert_array_equal(best.cpu().numpy().astype(np.float64), best_ref)
        np.testing.assert_allclose(plan.cpu().numpy(), plan_ref, rtol=0, atol=2e-5)
        np.testing.assert_allclose(mean.cpu().numpy(), nxt, rtol=0, atol=2e-5)
        mean_in = mean.cpu().numpy().astype(np.float64)


def test_cluster_update_beyond_a_warp():
    """5 controllers of 6000 samples, the top 1 % (60 elites each), three drones
    in two worlds, two iterations."""
    _cluster_case([1, 2], S=30000, C=5, n_e=60, H=10, seed_base=7)


@pytest.mark.parametrize("C,S_c,n_e", [(1, 2049, 1), (2, 300, 33), (8, 4000, 4000), (3, 9000, 1500)])
def test_cluster_update_shapes(C, S_c, n_e):
    """Cluster sizes 1-8; a controller just past the warp path's costs; elites
    just past a warp; every sample an elite (n_e = S_c); more than 1024 elites
    (several elites per thread)."""
    _cluster_case([2], S=C * S_c, C=C, n_e=n_e, H=7, seed_base=C + S_c, sample_costs=64, iters=1,
                  lam=0.5)


def test_paper_scale_mppi_iteration():
    """The paper's MPPI: one drone, 500k trajectories in five controllers of
    100 000, the top 1 % (1000 elites each), a 25-step horizon at 50 Hz."""
    wl = W.mppi_workload(n_drones=1, S=500_000)
    assert wl.cfg["n_elite"] == 1000 and wl.cfg["n_ctrl"] == 5
    sim = Sim.batched(wl.n_per_world, np.zeros(1, np.int32), RK4, wl.dt)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
    c = wl.cfg
    S, H, C = c["S"], c["H"], c["n_ctrl"]
    mean0 = np.zeros((1, C, H, 4))
    mean = torch.zeros(1, C, H, 4, device="cuda")
    g = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    plan, cost, best = sim.mppi_iteration(c, _seed(wl.seed), g, wl.obstacles, mean)
    c_gpu = cost.cpu().numpy().astype(np.float64)
    assert np.isfinite(c_gpu).all()
    s = np.random.default_rng(3).integers(0, S, 64)
    acts = sa.sampled_actions(wl.seed, s.astype(np.uint64), H, np.zeros((64, H, 4)), c["sigma"], c["rho"])
    ref = sa.cost_of_actions(_f32(wl.x0)[np.zeros(64, int)], _f32(wl.goals)[np.zeros(64, int)],
                             _f32(wl.obstacles), wl.params, acts, wl.dt, c["w_obs"], RK4)
    np.testing.assert_allclose(c_gpu[0, s], np.ravel(ref), rtol=1e-4, atol=1e-4)
    nxt, plan_ref, best_ref = mp.update(c_gpu, mean0, wl.seed, S, H, C, c["sigma"], c["rho"],
                                        c["n_elite"], c["lam"], [0])
    np.testing.assert_array_equal(best.cpu().numpy().astype(np.float64), best_ref)
    np.testing.assert_allclose(plan.cpu().numpy(), plan_ref, rtol=0, atol=2e-5)
    np.testing.assert_allclose(mean.cpu().numpy(), nxt, rtol=0, atol=2e-5)


def test_cluster_update_is_deterministic():
    """Fixed-order sums: two runs of the same iteration give identical outputs."""
    P, x0, goals, obs, sim = _setup([2, 1], seed=12)
    cfg = dict(S=15000, H=9, n_ctrl=3, sigma=0.3, rho=0.5, n_elite=50, lam=0.1, w_obs=1000.0)
    g = torch.tensor(goals, dtype=torch.float32, device="cuda")
    mean0 = torch.tensor(np.random.default_rng(1).uniform(-0.2, 0.2, (3, 3, 9, 4)), dtype=torch.float32,
                         device="cuda")
    outs = []
    for _ in range(2):
        mean = mean0.clone()
        plan, cost, best = sim.mppi_iteration(cfg, _seed(77), g, obs, mean)
        outs.append((plan.clone(), cost.clone(), best.clone(), mean))
    for u, v in zip(*outs):
        assert torch.equal(u, v)


def test_cluster_path_limits_are_refused():
    """More than 8 controllers or a horizon beyond 1024 on the cluster path, an
    elite count above the controller's samples or SIM_MAX_ELITES: SIM_EINVAL,
    nothing launched."""
    from paper_2606_01478_b300 import SimError
    from paper_2606_01478_b300 import _lib as L
    P, x0, goals, obs, sim = _setup([1], seed=2)
    g = torch.tensor(goals, dtype=torch.float32, device="cuda")
    for S, C, n_e, H in ((9 * 3000, 9, 30, 4), (5000, 1, 50, 1025), (100, 1, 101, 4),
                         (10000, 1, L.MAX_ELITES + 1, 4), (100, 1, 0, 4)):
        cfg = dict(S=S, H=H, n_ctrl=C, sigma=0.3, rho=0.5, n_elite=n_e, lam=0.1, w_obs=1000.0)
        mean = torch.zeros(1, C, H, 4, device="cuda")
        with pytest.raises(SimError) as ei:
            sim.mppi_iteration(cfg, _seed(1), g, obs, mean)
        assert ei.value.code == L.SIM_EINVAL
    # the warp path takes more controllers
    cfg = dict(S=9 * 100, H=4, n_ctrl=9, sigma=0.3, rho=0.5, n_elite=1, lam=0.1, w_obs=1000.0)
    sim.mppi_iteration(cfg, _seed(1), g, obs, torch.zeros(1, 9, 4, 4, device="cuda"))
