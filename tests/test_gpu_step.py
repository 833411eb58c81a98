"""GPU parity of the fused forward step against the FP64 oracle (through the
C-ABI), plus properties that hold at any size (fused K == repeated K = 1,
determinism, layout round trip, non-finite detection)."""
import ctypes
import dataclasses

import numpy as np
import pytest
import torch

import workloads as W
from oracle import physics as ph
from paper_2606_01478_b300 import Sim
from paper_2606_01478_b300 import _lib as L

from gpu_util import assert_parity, make_sim

pytestmark = pytest.mark.gpu


def _models_of(wl, drones=None):
    n = wl.M * wl.N
    idx = np.arange(n) if drones is None else np.asarray(drones)
    return np.asarray(wl.model_of_world)[idx // wl.N]


def _run_gpu(wl, steps=None, K=None, tpb=None):
    sim = make_sim(wl, tpb=tpb)
    sim.run(wl.steps if steps is None else steps, K or wl.K)
    out = sim.get_state().cpu().numpy()
    assert sim.status() == 0
    return out, sim


def test_single_drone_position_error_below_1e4_m():
    """1 world x 1 drone, position PID, Euler at 500 Hz, 1000 steps in ONE
    launch: |p_GPU - p_FP64| <= 1e-4 m (the stated bar)."""
    wl = W.position_hold_single()
    gpu, sim = _run_gpu(wl)
    assert sim.launches >= 1
    ref = ph.rollout_workload(wl).numpy()
    errs = assert_parity(gpu, ref, _models_of(wl))
    assert np.abs(gpu[0, 0:3] - ref[0, 0:3]).max() <= 1e-4, errs


@pytest.mark.parametrize("tpb", [32, 128, 256])
def test_attitude_swarm_small_rk4(tpb):
    """The RK4 attitude-swarm recipe at 1000 drones (ragged tail for every block size),
    RK4, 250 steps as launches of K = 100 (command blocks of 50 change inside
    and across launches)."""
    wl = W.attitude_swarm_rk4(M=1000, steps=250, K=100)
    gpu, _ = _run_gpu(wl, tpb=tpb)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
@pytest.mark.parametrize("ctrl", [ph.CTRL_ROTOR_SPEED, ph.CTRL_ATTITUDE, ph.CTRL_POSITION])
def test_first_principles_all_controls(integrator, ctrl):
    wl = W.attitude_swarm_rk4(M=333, steps=120, K=37)
    wl.integrator, wl.ctrl = integrator, ctrl
    rng = np.random.default_rng(5)
    if ctrl == ph.CTRL_ROTOR_SPEED:
        wl.cmd = rng.uniform(9000, 19000, wl.cmd.shape)
    elif ctrl == ph.CTRL_POSITION:
        wl.cmd = np.concatenate([rng.uniform(-1, 1, wl.cmd.shape[:2] + (2,)),
                                 rng.uniform(0.5, 1.5, wl.cmd.shape[:2] + (1,)),
                                 rng.uniform(-0.5, 0.5, wl.cmd.shape[:2] + (1,))], -1)
        wl.x0[:, 17:20] = rng.uniform(-0.05, 0.05, (wl.M, 3))
    gpu, _ = _run_gpu(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
@pytest.mark.parametrize("batched", [False, True], ids=["uniform", "batched"])
def test_asymmetric_inertia_lag_rotors(integrator, batched):
    """Jx != Jy on the lag rotor model: the kernels keep the yaw rate's gyroscopic
    term (their Jx = Jy variants leave it out); body rates up to 8 rad/s make the
    term count.  Batched: two parameter sets, only one of them asymmetric, which
    must select the asymmetric variant for every world."""
    wl = W.attitude_swarm_rk4(M=300, steps=150, K=50)
    wl.integrator = integrator
    rng = np.random.default_rng(9)
    wl.x0[:, 10:13] = rng.uniform(-8.0, 8.0, (wl.M, 3))
    asym = W.crazyflie_params(Jx=1.2e-5, Jy=1.8e-5)
    if batched:
        wl.params = [W.crazyflie_params(), asym]
        wl.param_set_of_world = (np.arange(wl.M) % 2).astype(np.int32)
        sim = Sim.batched(np.ones(wl.M, np.int64), np.zeros(wl.M, np.int32), integrator, wl.dt,
                          ctrl=wl.ctrl, max_cmd_blocks=wl.cmd.shape[0])
        sim.set_params(wl.params, wl.param_set_of_world)
        sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
        sim.set_commands(torch.tensor(wl.cmd, dtype=torch.float32, device="cuda"), wl.hold)
        sim.run(wl.steps, wl.K)
        gpu = sim.get_state().cpu().numpy()
        assert sim.status() == 0
    else:
        wl.params = [asym]
        gpu, _ = _run_gpu(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_general_motor_and_drag(integrator):
    """Asymmetric rotor coefficients with quadratic terms (Eq. 6 general form)
    and non-zero body drag, per-world parameter sets."""
    wl = W.attitude_swarm_rk4(M=300, steps=100, K=50)
    wl.integrator = integrator
    rng = np.random.default_rng(8)
    base = W.crazyflie_params(cv_up=40.0, cd_up=1e-3, cv_down=20.0, cd_down=5e-4,
                              Ca_x=-0.01, Ca_y=-0.012, Ca_z=-0.02)
    wl.params = [dict(base, mass=base["mass"] * s) for s in rng.uniform(0.95, 1.05, 5)]
    wl.param_set_of_world = rng.integers(0, 5, wl.M).astype(np.int32)
    gpu, _ = _run_gpu(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_abstracted_model_per_world_coefficients(integrator):
    wl = W.mixed_swarm_euler(M=6, N=100, steps=150, K=64)
    keep = wl.model_of_world == 1
    # an all-abstracted uniform batch: take the odd worlds of the mixed-swarm recipe
    worlds = np.nonzero(keep)[0]
    drones = (worlds[:, None] * wl.N + np.arange(wl.N)[None, :]).ravel()
    wl.x0 = wl.x0[drones]
    wl.cmd = wl.cmd[:, drones]
    wl.params = [wl.params[w] for w in worlds]
    wl.M = len(worlds)
    wl.param_set_of_world = np.arange(wl.M, dtype=np.int32)
    wl.model_of_world = np.ones(wl.M, np.int32)
    wl.integrator = integrator
    gpu, _ = _run_gpu(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_abstracted_model_drag_and_general_variant(integrator):
    """Abstracted worlds in the general rotor-model kernel variant: every other
    world with body drag (the Euler step through the derivative), the rest
    without drag (the Euler step with the step size folded into its terms),
    against the FP64 oracle."""
    wl = W.mixed_swarm_euler(M=8, N=64, steps=120, K=40)
    worlds = np.nonzero(wl.model_of_world == 1)[0]
    drones = (worlds[:, None] * wl.N + np.arange(wl.N)[None, :]).ravel()
    wl.x0 = wl.x0[drones]
    wl.cmd = wl.cmd[:, drones]
    params = []
    for i, w in enumerate(worlds):
        p = dict(wl.params[w])
        if i % 2 == 0:
            p.update(Ca_x=-0.01, Ca_y=-0.012, Ca_z=-0.02)
        else:
            p.update(cv_up=40.0, cv_down=20.0)  # no drag, general rotor-model variant
        params.append(p)
    wl.params = params
    wl.M = len(worlds)
    wl.param_set_of_world = np.arange(wl.M, dtype=np.int32)
    wl.model_of_world = np.ones(wl.M, np.int32)
    wl.integrator = integrator
    gpu, _ = _run_gpu(wl)
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(gpu, ref, _models_of(wl))
    # the drag worlds do move differently from drag-free ones with the same inputs
    free = [dict(p, Ca_x=0.0, Ca_y=0.0, Ca_z=0.0) for p in params]
    ref_free = ph.rollout_workload(dataclasses.replace(wl, params=free)).numpy()
    drag_rows = np.repeat(np.arange(wl.M) % 2 == 0, wl.N)
    assert np.abs(ref_free[drag_rows, 6:9] - ref[drag_rows, 6:9]).max() > 1e-4


def test_attitude_swarm_full_size_sampled():
    """The RK4 attitude swarm at full size (16384 worlds, RK4, 1000 steps as 10 launches of
    K = 100, the launch configuration the benchmark times); the oracle checks
    a sample of 48 drones (exact, since drones do not interact)."""
    wl = W.attitude_swarm_rk4()
    gpu, _ = _run_gpu(wl)
    sample = np.random.default_rng(0).choice(wl.M, 48, replace=False)
    ref = ph.rollout_workload(wl, drones=sample).numpy()
    assert_parity(gpu[sample], ref, _models_of(wl, sample))


def test_hover_fixed_point_on_gpu():
    wl = W.attitude_swarm_rk4(M=256, steps=1000, K=250)
    P = wl.params[0]
    wl.x0[:] = 0
    wl.x0[:, 0:3] = np.random.default_rng(1).uniform(-1, 1, (256, 3))
    wl.x0[:, 6] = 1.0
    wl.x0[:, 13:17] = W.hover_rpm(P)
    wl.cmd[:] = 0
    gpu, _ = _run_gpu(wl)
    x0 = wl.x0.astype(np.float32)
    assert np.abs(gpu[:, 0:3] - x0[:, 0:3]).max() < 1e-5
    assert np.abs(gpu[:, 7:13]).max() < 1e-5


@pytest.mark.parametrize("integrator", [ph.RK4, ph.EULER])
def test_fused_K_equals_single_steps(integrator):
    """One launch of K steps and K launches of one step run the same float
    operations: the states agree bit for bit (Euler: the fused hold loop is
    unrolled by two, and K = 7 leaves odd remainders in every command block)."""
    wl = W.attitude_swarm_rk4(M=500, steps=60, K=60)
    wl.integrator = integrator
    a, _ = _run_gpu(wl, K=60)
    b, _ = _run_gpu(wl, K=1)
    c, _ = _run_gpu(wl, K=7)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_deterministic_and_resumable():
    wl = W.attitude_swarm_rk4(M=700, steps=100, K=100)
    a, _ = _run_gpu(wl)
    b, _ = _run_gpu(wl)
    assert np.array_equal(a, b)
    # stop after 50 steps, read the state back, reload it into a fresh handle
    sim = make_sim(wl)
    sim.run(50, 50)
    mid = sim.get_state()
    sim2 = make_sim(wl)
    sim2.set_state(mid)
    sim2.set_commands(torch.tensor(wl.cmd[1:], dtype=torch.float32, device="cuda").contiguous(), 50)
    sim2.run(50, 50)
    assert np.array_equal(sim2.get_state().cpu().numpy(), a)


def test_state_roundtrip_host_and_device():
    wl = W.attitude_swarm_rk4(M=1234, steps=1)
    sim = make_sim(wl)
    x = torch.tensor(wl.x0, dtype=torch.float32)
    assert torch.equal(sim.get_state().cpu(), x)
    host_out = torch.empty_like(x).pin_memory()
    sim.get_state(out=host_out)
    torch.cuda.synchronize()
    assert torch.equal(host_out, x)
    y = (x + 1.0).pin_memory()
    sim.set_state(y)
    torch.cuda.synchronize()
    assert torch.equal(sim.get_state().cpu(), y)


def test_nonfinite_state_sets_status_flag():
    wl = W.attitude_swarm_rk4(M=100, steps=5, K=5)
    wl.x0[17, 7] = np.nan
    sim = make_sim(wl)
    sim.run(5, 5)
    assert sim.status() & L.SIM_FLAG_NONFINITE
    assert sim.status() == 0  # reading clears the word
    wl2 = W.attitude_swarm_rk4(M=100, steps=5, K=5)
    sim2 = make_sim(wl2)
    sim2.run(5, 5)
    assert sim2.status() == 0


def test_bounded_wait_gives_up_and_reports_timeout():
    """Failure detection without a GPU fault: a barrier phase that nothing completes
    makes the bounded in-kernel wait (the rollout adjoint's hand-off wait) give up;
    the kernel returns, SIM_FLAG_TIMEOUT reaches the host, and the context stays
    usable for a normal step afterwards."""
    import time
    wl = W.attitude_swarm_rk4(M=100, steps=5, K=5)
    sim = make_sim(wl)
    assert sim.status() == 0
    stream = torch.cuda.current_stream().cuda_stream
    t0 = time.perf_counter()
    assert sim.lib.sim_selftest_wait_timeout(sim.h, ctypes.c_void_p(stream)) == L.SIM_OK
    flags = sim.status()
    elapsed = time.perf_counter() - t0
    assert flags & L.SIM_FLAG_TIMEOUT
    assert elapsed < 20.0  # the wait limit is about a second
    sim.run(5, 5)
    assert sim.status() == 0
    ref = ph.rollout_workload(wl).numpy()
    assert_parity(sim.get_state().cpu().numpy(), ref, np.zeros(wl.M, np.int64))


def test_call_order_and_argument_errors():
    sim = Sim(4, 4, ph.FIRST_PRINCIPLES, ph.EULER, 0.002)
    with pytest.raises(L.SimError) as e:
        sim.step(1)
    assert e.value.code == L.SIM_ESTATE
    sim.set_params(W.crazyflie_params())
    with pytest.raises(L.SimError) as e:
        sim.set_params(W.crazyflie_params(mass=-1.0))
    assert e.value.code == L.SIM_EINVAL
    with pytest.raises(L.SimError):
        sim.set_params([W.crazyflie_params()] * 2, set_of_world=np.array([0, 1, 2, 0]))
    x = torch.zeros(16, 20, dtype=torch.float32, device="cuda")
    sim.set_state(x)
    c = torch.zeros(2, 16, 4, device="cuda")
    with pytest.raises(L.SimError) as e:
        sim.set_commands(c, 10)  # only 1 block fits the workspace
    assert e.value.code == L.SIM_EINVAL
    sim.set_commands(c[:1].contiguous(), 10)
    sim.step(3)
    assert sim.steps_taken == 3


@pytest.mark.parametrize("where", ["pinned", "pageable", "device"])
def test_run_host_equals_separate_calls(where):
    """sim_run_host (state rows read and written in place, commands gathered by a
    kernel, when the buffers are pinned or on the device) gives the bits of
    set_state + set_commands + run + get_state from device buffers: 777 drones,
    RK4, 230 steps as launches of K = 40 (last one short), hold 30, 12 command
    blocks (more than the 230 steps read)."""
    wl = W.attitude_swarm_rk4(M=777, steps=230, K=40)
    cmd = np.random.default_rng(3).uniform(-0.5, 0.5, (12, 777, 4))
    a = make_sim(wl, max_blocks=12)
    a.set_commands(torch.tensor(cmd, dtype=torch.float32, device="cuda"), 30)
    a.run(230, 40)
    ref = a.get_state().cpu()
    b = make_sim(wl, max_blocks=12)
    x0 = torch.tensor(wl.x0, dtype=torch.float32)
    c = torch.tensor(cmd, dtype=torch.float32)
    out = None
    if where == "pinned":
        x0, c = x0.pin_memory(), c.pin_memory()
    elif where == "device":
        x0, c = x0.cuda(), c.cuda()
        out = torch.empty(777, 20, device="cuda")
    got = b.run_host(x0, c, 30, 230, 40, out=out)
    torch.cuda.synchronize()
    assert torch.equal(got.cpu(), ref)
    assert b.steps_taken == 230
    # the handle continues from there like the separate calls
    a.run(20, 20)
    b.run(20, 20)
    assert torch.equal(a.get_state().cpu(), b.get_state().cpu())
