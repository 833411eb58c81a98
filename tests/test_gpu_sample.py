"""GPU parity of the batched sampling rollouts (Philox noise, RK4 rollouts,
goal + obstacle cost) against the FP64 oracle; Philox bit-exactness on 10^6
counters; CUDA-graph replay with a fresh device seed."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import sampling as sa
from paper_2606_01478_b300 import EULER, RK4, Sim
from paper_2606_01478_b300 import _lib as L

pytestmark = pytest.mark.gpu

RTOL = 1e-4  # cost: FP32 rollout of 50 steps vs FP64 (relative to the cost)


def _seed_tensor(seed):
    # the 64 bits of the key, reinterpreted as int64
    return torch.tensor([np.int64(np.uint64(seed).view(np.int64))], device="cuda")


def _sim_for(n_per_world, P, x0, integrator=RK4, dt=1 / 500):
    sim = Sim.batched(np.asarray(n_per_world), np.zeros(len(n_per_world), np.int32), integrator,
                      dt)
    sim.set_params(P)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    return sim


def _oracle(x0, goals, obs, P, S, H, sigma, seed, w_obs, n_per_world, drones, samples, nominal=None,
            dt=1 / 500, integrator=RK4):
    world = np.repeat(np.arange(len(n_per_world)), n_per_world)
    x0f = np.asarray(x0, np.float32).astype(np.float64)
    return sa.rollout_cost(x0f, np.asarray(goals, np.float32).astype(np.float64),
                           np.asarray(obs, np.float32).astype(np.float64), P, S, H, dt, sigma,
                           seed, w_obs, drones, samples, world,
                           None if nominal is None else np.asarray(nominal, np.float32).astype(np.float64),
                           sa.ph.RK4 if integrator == RK4 else sa.ph.EULER)


def _scene(seed, n_per_world, **kw):
    wl = W.uneven_sampling_rk4(seed=seed, M=len(n_per_world), **kw)
    n = int(np.sum(n_per_world))
    rng = np.random.default_rng(seed)
    x0 = wl.x0[:1].repeat(n, 0)
    x0[:, 0:3] = rng.uniform([-1.5, -1.5, 0.5], [1.5, 1.5, 3.5], (n, 3))
    return wl, x0


def test_philox_bit_exact_on_a_million_counters():
    seed = 0x9E3779B97F4A7C15
    sd = _seed_tensor(seed)
    n = 1 << 20
    first = 2**33 + 5
    words = torch.empty(n, 4, dtype=torch.int32, device="cuda")
    z = torch.empty(n, 4, dtype=torch.float32, device="cuda")
    lib = L.load()
    r = lib.sim_philox_normals(ctypes.c_void_p(sd.data_ptr()), first, n, 7,
                               ctypes.c_void_p(words.data_ptr()), ctypes.c_void_p(z.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == L.SIM_OK
    got = words.cpu().numpy().view(np.uint32)
    ids = np.arange(first, first + n, dtype=np.uint64)
    ctr = np.stack([ids & np.uint64(0xFFFFFFFF), ids >> np.uint64(32), np.full(n, 7, np.uint64),
                    np.zeros(n, np.uint64)], -1)
    key = np.broadcast_to(np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64), (n, 2))
    assert np.array_equal(got, sa.philox4x32_10(ctr, key))
    # every normal of the million counters; the radius takes a series where u1 lies
    # within 2^-8 of 1 and the hardware logarithm elsewhere: check both sides
    ref = sa.normals(seed, ids, 7)
    err = np.abs(z.cpu().numpy() - ref)
    assert err.max() < 2e-5
    u = sa.uniform24(got)
    for pair in (0, 2):
        near = u[:, pair] > 1.0 - 2.0 ** -8
        assert near.sum() > 1000 and (~near).sum() > 1000
        assert err[near][:, pair:pair + 2].max() < 2e-5
        edge = u[:, pair] > 1.0 - 2.0 ** -16  # radius below 1.3e-2
        assert edge.sum() > 0 and err[edge][:, pair:pair + 2].max() < 2e-6


@pytest.mark.parametrize("S", [1, 37])
def test_uneven_sampling_parity(S):
    n_w = [1, 5, 40, 3, 100, 2, 33]
    wl, x0 = _scene(71, n_w)
    sim = _sim_for(n_w, wl.params, x0)
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    cost = sim.sample_rollouts(S, 50, _seed_tensor(wl.seed), 0.2, goals, wl.obstacles, wl.w_obs)
    assert cost.shape == (sum(n_w), S)
    n = sum(n_w)
    drones = np.repeat(np.arange(n), S)
    samples = np.tile(np.arange(S), n)
    ref = _oracle(x0, wl.goals, wl.obstacles, wl.params, S, 50, 0.2, wl.seed, wl.w_obs, n_w,
                  drones, samples).reshape(n, S)
    got = cost.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-4)


@pytest.mark.parametrize("asym", [False, True])
def test_per_world_parameter_sets(asym):
    """Worlds on different parameter sets (mass, thrust coefficient, motor lag; with
    asym, one set with Jx != Jy, which keeps the yaw rate's gyroscopic term): each
    rollout reads its world's set; the oracle runs each set's drones with it."""
    n_w = [5, 7, 3, 9, 4]
    wl, x0 = _scene(75, n_w)
    x0[:, 10:13] = np.random.default_rng(3).uniform(-2.0, 2.0, (len(x0), 3))  # body rates
    third = dict(Jy=1.9e-5) if asym else {}
    sets = [W.crazyflie_params(), W.crazyflie_params(mass=0.031, kf=3.4e-10),
            W.crazyflie_params(mass=0.025, cv_up=1.0 / 0.045, cv_down=1.0 / 0.045, **third)]
    sow = np.array([1, 0, 2, 1, 2], np.int32)
    sim = Sim.batched(np.asarray(n_w), np.zeros(len(n_w), np.int32), RK4, 1 / 500)
    sim.set_params(sets, set_of_world=sow)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    S, H = 16, 50
    cost = sim.sample_rollouts(S, H, _seed_tensor(wl.seed), 0.2,
                               torch.tensor(wl.goals, dtype=torch.float32, device="cuda"),
                               wl.obstacles, wl.w_obs).cpu().numpy().astype(np.float64)
    world = np.repeat(np.arange(len(n_w)), n_w)
    for k, P in enumerate(sets):
        drones = np.flatnonzero(sow[world] == k)
        d = np.repeat(drones, S)
        smp = np.tile(np.arange(S), len(drones))
        ref = _oracle(x0, wl.goals, wl.obstacles, P, S, H, 0.2, wl.seed, wl.w_obs, n_w, d,
                      smp).reshape(len(drones), S)
        np.testing.assert_allclose(cost[drones], ref, rtol=RTOL, atol=1e-4)
    # the sets matter: the same rollouts on set 0 alone differ
    sim.set_params(sets[0])
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    same = sim.sample_rollouts(S, H, _seed_tensor(wl.seed), 0.2,
                               torch.tensor(wl.goals, dtype=torch.float32, device="cuda"),
                               wl.obstacles, wl.w_obs).cpu().numpy().astype(np.float64)
    assert np.abs(same - cost)[sow[world] != 0].min() > 1e-6


def test_zero_noise_hover_cost_closed_form():
    n_w = [4, 9]
    wl, x0 = _scene(72, n_w)
    x0[:, 3:13] = 0
    x0[:, 6] = 1.0
    sim = _sim_for(n_w, wl.params, x0)
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    obs = wl.obstacles.copy()
    obs[0, 0:3] = x0[0, 0:3] + [0.05, 0.0, 0.0]  # drone 0 sits inside obstacle 0
    obs[0, 3] = 0.2
    H = 30
    cost = sim.sample_rollouts(3, H, _seed_tensor(1), 0.0, goals, obs, 1000.0).cpu().numpy()
    x0f = x0.astype(np.float32).astype(np.float64)
    world = np.repeat(np.arange(2), n_w)
    p0 = x0f[:, 0:3]
    g = wl.goals.astype(np.float32).astype(np.float64)[world]
    o = obs.astype(np.float32).astype(np.float64)
    pen = np.clip(o[None, :, 3] - np.linalg.norm(p0[:, None] - o[None, :, 0:3], axis=-1), 0, None)
    expect = H * (np.linalg.norm(p0 - g, axis=-1) + 1000.0 * pen.sum(-1))
    np.testing.assert_allclose(cost, np.repeat(expect[:, None], 3, 1), rtol=2e-5)
    assert pen[0].sum() > 0


def test_nominal_sequence_and_uniform_handle():
    """Per-world nominal command sequences on a uniform (M x N) handle."""
    M, N, S, H = 3, 20, 8, 40
    wl, x0 = _scene(73, [N] * M)
    sim = Sim(M, N, 0, RK4, 1 / 500)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    nominal = np.random.default_rng(2).uniform(-0.3, 0.3, (M, H, 4))
    cost = sim.sample_rollouts(S, H, _seed_tensor(wl.seed), 0.1,
                               torch.tensor(wl.goals, dtype=torch.float32, device="cuda"),
                               wl.obstacles, wl.w_obs,
                               nominal=torch.tensor(nominal, dtype=torch.float32, device="cuda"))
    drones = np.repeat(np.arange(M * N), S)
    samples = np.tile(np.arange(S), M * N)
    ref = _oracle(x0, wl.goals, wl.obstacles, wl.params, S, H, 0.1, wl.seed, wl.w_obs, [N] * M,
                  drones, samples, nominal=nominal).reshape(M * N, S)
    np.testing.assert_allclose(cost.cpu().numpy(), ref, rtol=RTOL, atol=1e-4)


def test_uneven_sampling_full_size_sampled():
    """The uneven sampling workload: 512 worlds with log-uniform drone counts in [1, 4000], 256
    samples each, 50 RK4 steps; 64 sampled (drone, sample) pairs against the
    oracle."""
    wl = W.uneven_sampling_rk4()
    sim = _sim_for(wl.n_per_world, wl.params, wl.x0)
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    cost = sim.sample_rollouts(wl.S, wl.H, _seed_tensor(wl.seed), wl.sigma, goals, wl.obstacles,
                               wl.w_obs)
    assert sim.status() == 0
    c = cost.cpu().numpy()
    assert np.isfinite(c).all()
    rng = np.random.default_rng(5)
    n = len(wl.x0)
    drones = rng.integers(0, n, 64)
    samples = rng.integers(0, wl.S, 64)
    ref = _oracle(wl.x0, wl.goals, wl.obstacles, wl.params, wl.S, wl.H, wl.sigma, wl.seed,
                  wl.w_obs, wl.n_per_world, drones, samples)
    np.testing.assert_allclose(c[drones, samples], ref, rtol=RTOL, atol=1e-4)


def test_graph_replay_reads_a_fresh_seed():
    n_w = [17, 3, 60]
    wl, x0 = _scene(74, n_w)
    sim = _sim_for(n_w, wl.params, x0)
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    seed = _seed_tensor(111)
    cost = torch.empty(sum(n_w), 16, device="cuda")
    eager = {}
    for s in (111, 222):
        seed.copy_(_seed_tensor(s))
        eager[s] = sim.sample_rollouts(16, 25, seed, 0.2, goals, wl.obstacles, wl.w_obs).clone()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            sim.sample_rollouts(16, 25, seed, 0.2, goals, wl.obstacles, wl.w_obs, cost=cost,
                                stream=st)
    torch.cuda.current_stream().wait_stream(st)
    for s in (222, 111):
        seed.copy_(_seed_tensor(s))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(cost, eager[s])
    assert not torch.equal(eager[111], eager[222])


def test_moving_drones_near_obstacle_shells():
    """Drones with initial velocity and obstacles placed on shells around the
    start positions (inside, near and beyond what the horizon can reach), high
    noise: costs match the oracle, so no reachable obstacle is skipped."""
    n_w = [6, 10]
    wl, x0 = _scene(75, n_w)
    rng = np.random.default_rng(8)
    x0[:, 7:10] = rng.uniform(-2.0, 2.0, (16, 3))
    obs = []
    for d in range(0, 16, 3):
        for dist in (0.05, 0.2, 0.35, 0.5, 0.8):
            u = rng.normal(size=3)
            u /= np.linalg.norm(u)
            obs.append(list(x0[d, 0:3] + (dist + 0.15) * u) + [0.15])
    obs = np.array(obs[:64])
    sim = _sim_for(n_w, wl.params, x0)
    S, H = 24, 60
    cost = sim.sample_rollouts(S, H, _seed_tensor(5), 0.6,
                               torch.tensor(wl.goals, dtype=torch.float32, device="cuda"), obs, 1000.0)
    drones = np.repeat(np.arange(16), S)
    samples = np.tile(np.arange(S), 16)
    ref = _oracle(x0, wl.goals, obs, wl.params, S, H, 0.6, 5, 1000.0, n_w, drones, samples).reshape(16, S)
    np.testing.assert_allclose(cost.cpu().numpy(), ref, rtol=RTOL, atol=1e-4)
    # the scene does put obstacles inside the reachable region
    assert (ref > H * 0.0 + 1.0).any()


@pytest.mark.parametrize("integrator", [RK4, EULER])
def test_obstacles_along_the_path_over_many_culling_windows(integrator):
    """A 0.8 s horizon at 100 Hz is eight culling windows of 0.1 s: drones fly at
    up to 3 m/s and obstacles sit on and beside their straight-line paths at
    0.05-0.75 s, so most penalties fall in windows after the first.  Costs match
    the oracle, which tests every obstacle at every step."""
    n_w = [7, 9]
    wl, x0 = _scene(76, n_w)
    rng = np.random.default_rng(9)
    v = rng.uniform(-3.0, 3.0, (16, 3))
    x0[:, 7:10] = v
    obs = []
    for d in range(16):
        for t in (0.05, 0.3, 0.55, 0.75):
            off = rng.normal(size=3) * 0.05
            obs.append(list(x0[d, 0:3] + v[d] * t + off) + [0.2])
    obs = np.array(obs[:64])
    dt, S, H = 1 / 100, 12, 80
    sim = _sim_for(n_w, wl.params, x0, integrator, dt)
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    cost = sim.sample_rollouts(S, H, _seed_tensor(6), 0.3, goals, obs, 1000.0)
    assert sim.status() == 0
    drones = np.repeat(np.arange(16), S)
    samples = np.tile(np.arange(S), 16)
    ref = _oracle(x0, wl.goals, obs, wl.params, S, H, 0.3, 6, 1000.0, n_w, drones, samples,
                  dt=dt, integrator=integrator).reshape(16, S)
    np.testing.assert_allclose(cost.cpu().numpy(), ref, rtol=RTOL, atol=1e-4)
    # the obstacles matter: without them the costs drop for most drones
    free = _oracle(x0, wl.goals, obs, wl.params, S, H, 0.3, 6, 0.0, n_w, drones, samples,
                   dt=dt, integrator=integrator).reshape(16, S)
    assert ((ref - free) > 1.0).mean() > 0.5
