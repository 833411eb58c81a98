"""GPU parity of the rotor extensions (rotor inertia: gyroscopic + reaction
torques; polynomial thrust / drag-torque curves), the torque interface and the
abstracted model without thrust dynamics, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import physics as ph
from paper_2606_01478_b300 import Sim

from gpu_util import assert_parity, make_sim

pytestmark = pytest.mark.gpu


def _models_of(wl):
    return np.asarray(wl.model_of_world)[np.arange(wl.M * wl.N) // wl.N]


def _run(wl, tpb=None):
    sim = make_sim(wl, tpb=tpb)
    sim.run(wl.steps, wl.K)
    out = sim.get_state().cpu().numpy()
    assert sim.status() == 0
    return out


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_rotor_inertia_and_polynomial_curves(integrator):
    wl = W.attitude_swarm_rk4(M=400, steps=150, K=50)
    wl.integrator = integrator
    wl.params = [W.crazyflie_params(J_p=3e-8, kf1=1.5e-7, kf0=-0.002, km1=4e-9, cv_up=40.0,
                                    cv_down=25.0, cd_up=2e-4)]
    gpu = _run(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_torque_interface(integrator):
    wl = W.attitude_swarm_rk4(M=300, steps=120, K=40)
    wl.integrator, wl.ctrl = integrator, ph.CTRL_TORQUE
    p = W.crazyflie_params()
    rng = np.random.default_rng(6)
    T = p["mass"] * p["g"] * rng.uniform(0.8, 1.3, wl.cmd.shape[:2])
    tau = rng.uniform(-1, 1, wl.cmd.shape[:2] + (3,)) * np.array([1e-5, 1e-5, 5e-6])
    wl.cmd = np.concatenate([T[..., None], tau], -1)
    gpu = _run(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_abstracted_without_thrust_dynamics(integrator):
    wl = W.mixed_swarm_euler(M=4, N=150, steps=120, K=60)
    wl.integrator = integrator
    wl.model_of_world = np.full(wl.M, 2, np.int32)
    wl.x0[:, 3:6] = np.random.default_rng(2).uniform(-0.5, 0.5, (wl.M * wl.N, 3))
    wl.x0[:, 6:13] = 0
    gpu = _run(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


def test_three_models_in_one_launch():
    """Worlds of all three models (and uneven sizes) in one persistent launch."""
    n = np.array([33, 7, 64, 1, 90, 40])
    models = np.array([0, 1, 2, 2, 1, 0], np.int32)
    bw = W.batched_workload(17, n, np.minimum(models, 1), integrator=ph.RK4, steps=80, K=40, hold=20)
    bw.model_of_world = models
    sim = Sim.batched(bw.n_per_world, bw.model_of_world, bw.integrator, bw.dt,
                      max_cmd_blocks=bw.cmd.shape[0])
    sim.set_params(bw.params, np.arange(bw.M))
    sim.set_state(torch.tensor(bw.x0, dtype=torch.float32, device="cuda"))
    sim.set_commands(torch.tensor(bw.cmd, dtype=torch.float32, device="cuda"), bw.hold)
    sim.run(bw.steps, bw.K)
    gpu = sim.get_state().cpu().numpy()
    world = bw.world_of_drone()
    ref = ph.rollout(bw.x0, bw.cmd, bw.hold, bw.steps, bw.params, world, models[world], bw.dt,
                     bw.integrator, bw.ctrl).numpy()
    assert_parity(gpu, ref, models[world])
