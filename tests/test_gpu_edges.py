"""Edge cases of the CUDA path: a batch of 2^27 drones checked on sampled
drones, free fall in closed form, the shortest rollout horizon, the extremes
of the MPPI elite count, the smallest sampling problem and a camera that sees
nothing."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import workloads as W
from gpu_util import assert_parity
from oracle import mppi as mp
from oracle import physics as ph
from oracle import policy as po
from oracle import sampling as sa
from paper_2606_01478_b300 import CTRL_ROTOR_SPEED, EULER, FIRST_PRINCIPLES, RK4, Sim
from paper_2606_01478_b300.rollout import PolicyRollout

pytestmark = pytest.mark.gpu


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def test_large_batch_sampled():
    """2^27 drones (one per world), RK4, attitude commands, 20 steps as two
    launches of K = 10; 64 sampled drones (first and last included) against the
    oracle.  Inputs come from torch's seeded device generator."""
    n = 1 << 27
    free, _ = torch.cuda.mem_get_info()
    if free < 64e9:
        pytest.skip("needs 64 GB of free device memory")
    g = torch.Generator(device="cuda")
    g.manual_seed(2027)
    P = W.crazyflie_params()
    x = torch.zeros(n, 20, device="cuda")
    x[:, 0:3] = torch.rand(n, 3, device="cuda", generator=g) * 2 - 1
    x[:, 2] += 1.0
    q = torch.cat([0.1 * torch.randn(n, 3, device="cuda", generator=g), torch.ones(n, 1, device="cuda")], 1)
    x[:, 3:7] = q / q.norm(dim=1, keepdim=True)
    x[:, 7:10] = torch.rand(n, 3, device="cuda", generator=g) * 2 - 1
    x[:, 10:13] = torch.rand(n, 3, device="cuda", generator=g) * 4 - 2
    x[:, 13:17] = float(W.hover_rpm(P))
    cmd = torch.rand(1, n, 4, device="cuda", generator=g) - 0.5
    pick = np.concatenate([[0, n - 1], np.random.default_rng(5).choice(n, 62, replace=False)])
    idx = torch.tensor(pick, device="cuda")
    x0_s = x[idx].cpu().numpy().astype(np.float64)
    cmd_s = cmd[:, idx].cpu().numpy().astype(np.float64)
    sim = Sim(n, 1, FIRST_PRINCIPLES, RK4, 1 / 500)
    sim.set_params(P)
    sim.set_state(x)
    sim.set_commands(cmd, 20)
    del x, cmd
    torch.cuda.empty_cache()
    sim.run(20, 10)
    assert sim.status() == 0
    out = sim.get_state()[idx].cpu().numpy()
    ref = ph.rollout(x0_s, cmd_s, 20, 20, [P], np.zeros(64, np.int64), np.zeros(64, np.int64), 1 / 500,
                     ph.RK4, ph.CTRL_ATTITUDE).numpy()
    assert_parity(out, ref, np.zeros(64, np.int64))


@pytest.mark.parametrize("integrator", [EULER, RK4])
def test_free_fall_closed_form(integrator):
    """Rotors stopped and commanded to zero: explicit Euler gives exactly
    p_n = p0 + n dt v0 - g dt^2 n (n - 1) / 2 e_z, RK4 the exact parabola; the
    attitude (zero body rate) stays put."""
    rng = np.random.default_rng(17)
    m, steps, dt = 37, 300, 1 / 500
    x0 = np.zeros((m, 20))
    x0[:, 0:3] = rng.uniform(-1, 1, (m, 3))
    x0[:, 3:7] = Rotation.random(m, random_state=3).as_quat()
    x0[:, 7:10] = rng.uniform(-2, 2, (m, 3))
    x0 = _f32(x0)
    sim = Sim(m, 1, FIRST_PRINCIPLES, integrator, dt, ctrl=CTRL_ROTOR_SPEED)
    sim.set_params(W.crazyflie_params())
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    sim.set_commands(torch.zeros(1, m, 4, device="cuda"), 1)
    sim.run(steps, 100)
    out = sim.get_state().cpu().numpy().astype(np.float64)
    g, dtf = 9.81, float(np.float32(dt))
    fall = g * dtf * dtf * steps * (steps - 1) / 2 if integrator == EULER else g * (steps * dtf) ** 2 / 2
    p = x0[:, 0:3] + steps * dtf * x0[:, 7:10]
    p[:, 2] -= fall
    v = x0[:, 7:10].copy()
    v[:, 2] -= steps * dtf * g
    # float32: 300 additions of ~1 ulp each (position ~2 m, velocity ~6 m/s)
    np.testing.assert_allclose(out[:, 0:3], p, atol=1e-4)
    np.testing.assert_allclose(out[:, 7:10], v, atol=1e-4)
    np.testing.assert_allclose(out[:, 3:7], x0[:, 3:7], atol=2e-5)  # renormalised every step
    assert np.all(out[:, 13:17] == 0)


@pytest.mark.parametrize("reward", [None, po.TRACKING_REWARD], ids=["squared", "reward"])
def test_rollout_single_step_horizon(reward):
    """H = C = 1 on 65 drones (one full CTA of 64 and a one-drone tail)."""
    rw = W.policy_bptt(seed=70, M=65, H=1, C=1)
    sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, reward=reward)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
    w = torch.tensor(po.pack(rw.weights), dtype=torch.float32, device="cuda").to(torch.bfloat16)
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
    loss, dW, dx0 = runner.grad(x0, w, p_ref)
    L, _, dW_ref, dx_ref = po.rollout_grad(_f32(rw.x0), rw.weights, _f32(rw.p_ref), rw.params, rw.dt,
                                           rw.H, rw.w_act, reward)
    assert abs(loss.item() - L) <= 1e-4 * abs(L)
    g = po.pack(dW_ref)
    assert np.linalg.norm(dW.cpu().numpy() - g) <= 1e-3 * np.linalg.norm(g)
    assert np.linalg.norm(dx0.cpu().numpy() - dx_ref) <= 1e-3 * np.linalg.norm(dx_ref)


@pytest.mark.parametrize("n_e", [100, 1, 32, 33])
def test_mppi_elite_count_extremes(n_e):
    """Every sample of a 100-sample controller an elite (cluster path), a single
    elite (whose plan is that sample's actions), and elite counts at and just
    past one warp."""
    rng = np.random.default_rng(9)
    P = W.crazyflie_params()
    n, S, H, C = 4, 200, 8, 2
    x0 = W.fp_state(rng.uniform([-1, -1, 1], [1, 1, 2], (n, 3)), np.zeros((n, 3)), np.zeros((n, 3)),
                    np.zeros((n, 3)), np.full((n, 4), W.hover_rpm(P)))
    goals = rng.uniform([-1, -1, 1], [1, 1, 2], (n, 3))
    sim = Sim.batched(np.ones(n, np.int64), np.zeros(n, np.int32), RK4, 1 / 50)
    sim.set_params(P)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    cfg = dict(S=S, H=H, n_ctrl=C, sigma=0.3, rho=0.6, n_elite=n_e, lam=0.3, w_obs=1000.0)
    mean0 = _f32(rng.uniform(-0.2, 0.2, (n, C, H, 4)))
    mean = torch.tensor(mean0, dtype=torch.float32, device="cuda")
    seed = torch.tensor([31], dtype=torch.int64, device="cuda")
    plan, cost, best = sim.mppi_iteration(cfg, seed, torch.tensor(goals, dtype=torch.float32, device="cuda"),
                                          np.zeros((0, 4)), mean)
    nxt, plan_ref, best_ref = mp.update(cost.cpu().numpy().astype(np.float64), mean0, 31, S, H, C, 0.3, 0.6,
                                        n_e, 0.3, np.arange(n))
    np.testing.assert_array_equal(best.cpu().numpy().astype(np.float64), best_ref)
    np.testing.assert_allclose(plan.cpu().numpy(), plan_ref, rtol=0, atol=2e-5)
    np.testing.assert_allclose(mean.cpu().numpy(), nxt, rtol=0, atol=2e-5)


def test_sampling_single_sample_single_step_no_obstacles():
    """S = 1, H = 1, no obstacles: the cost is the goal distance after one step."""
    rng = np.random.default_rng(23)
    P = W.crazyflie_params()
    n_w = np.array([1, 2, 1])
    n = int(n_w.sum())
    x0 = W.fp_state(rng.uniform(-1, 1, (n, 3)), np.zeros((n, 3)), rng.uniform(-1, 1, (n, 3)),
                    rng.uniform(-1, 1, (n, 3)), np.full((n, 4), W.hover_rpm(P)))
    goals = rng.uniform(-1, 1, (3, 3))
    sim = Sim.batched(n_w, np.zeros(3, np.int32), RK4, 1 / 500)
    sim.set_params(P)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    seed = torch.tensor([5], dtype=torch.int64, device="cuda")
    cost = sim.sample_rollouts(1, 1, seed, 0.2, torch.tensor(goals, dtype=torch.float32, device="cuda"),
                               np.zeros((0, 4)), 1000.0).cpu().numpy()
    world = np.repeat(np.arange(3), n_w)
    ref = sa.rollout_cost(_f32(x0), _f32(goals), np.zeros((0, 4)), P, 1, 1, 1 / 500, 0.2, 5, 1000.0,
                          np.arange(n), np.arange(1), world)
    np.testing.assert_allclose(cost[:, 0].astype(np.float64), np.ravel(ref), rtol=1e-5, atol=1e-6)


def test_camera_looking_up_sees_nothing():
    """Nose up (pitch -90 deg) with fields of view below 180 deg: every ray
    climbs, nothing is hit, every pixel reads max_range exactly."""
    n = 5
    P = W.crazyflie_params()
    x = np.zeros((n, 20))
    x[:, 0:3] = [[0, 0, 1], [1, 2, 0.5], [-3, 1, 2], [0, 0, 0.1], [5, 5, 3]]
    x[:, 3:7] = Rotation.from_euler("ZYX", np.stack([np.linspace(-3, 3, n), np.full(n, -np.pi / 2),
                                                     np.zeros(n)], 1)).as_quat()
    x[:, 13:17] = W.hover_rpm(P)
    sim = Sim(n, 1, FIRST_PRINCIPLES, RK4, 1 / 500)
    sim.set_params(P)
    sim.set_state(torch.tensor(x, dtype=torch.float32, device="cuda"))
    img = sim.render_depth(16, 24, math.radians(100), math.radians(80), 7.5,
                           spheres=[[0, 0, -2, 1.0]], boxes=[[-1, -1, -3, 1, 1, -2]])
    assert torch.all(img == 7.5)
