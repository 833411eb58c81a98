"""GPU parity of the MPPI / iCEM iteration: sampling costs against the FP64
oracle, and the update (elites, exponential weights, warm start, best
controller) against the oracle given the same costs -- the elite selection is
an integer decision, so both sides take it on identical inputs."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mppi as mp
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
    obs = np.concatenate([x0[:3, 0:3] + rng.uniform(-0.2, 0.2, (3, 3)), np.full((3, 1), 0.15)], 1)
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
    cfg = dict(S=60, H=12, n_ctrl=3, sigma=0.3, rho=0.5, elite_frac=0.1, lam=0.5, w_obs=1000.0)
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
        nxt, plan_ref, best_ref = mp.update(c_gpu, mean_in, seed, 60, 12, 3, 0.3, 0.5, 0.1, 0.5,
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
    cfg = dict(S=S, H=H, n_ctrl=1, sigma=0.25, rho=0.0, elite_frac=0.05, lam=1.0, w_obs=1000.0)
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
