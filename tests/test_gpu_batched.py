"""GPU parity of uneven / mixed-model batches (one persistent launch over warp
tiles) against the FP64 oracle, plus equivalence with the uniform path."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import physics as ph
from paper_2606_01478_b300 import Sim

from gpu_util import FP_SLICES, TOL_FP, assert_parity, make_sim

pytestmark = pytest.mark.gpu


def _gpu_batched(bw, tpb=None, K=None, steps=None):
    sim = Sim.batched(bw.n_per_world, bw.model_of_world, bw.integrator, bw.dt, ctrl=bw.ctrl,
                      max_cmd_blocks=bw.cmd.shape[0])
    if tpb:
        sim.set_block_size(tpb)
    sim.set_params(bw.params, np.arange(bw.M))
    sim.set_state(torch.tensor(bw.x0, dtype=torch.float32, device="cuda"))
    sim.set_commands(torch.tensor(bw.cmd, dtype=torch.float32, device="cuda"), bw.hold)
    sim.run(bw.steps if steps is None else steps, K or bw.K)
    out = sim.get_state().cpu().numpy()
    assert sim.status() == 0
    return out


def _oracle_batched(bw, drones=None, steps=None):
    world = bw.world_of_drone()
    idx = np.arange(bw.ntot) if drones is None else np.asarray(drones)
    return ph.rollout(bw.x0[idx], bw.cmd[:, idx], bw.hold, bw.steps if steps is None else steps,
                      bw.params, world[idx], bw.model_of_world[world[idx]], bw.dt, bw.integrator,
                      bw.ctrl).numpy()


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
@pytest.mark.parametrize("tpb", [64, 256])
def test_uneven_mixed_parity(integrator, tpb):
    """World sizes 1..200 (none a multiple of 32 but one), models mixed at
    random, per-world abstracted coefficients; 120 steps as launches of 50."""
    rng = np.random.default_rng(3)
    n = np.array([1, 37, 200, 5, 64, 33, 17, 129, 2, 90, 31, 63])
    models = rng.integers(0, 2, len(n))
    bw = W.batched_workload(11, n, models, integrator=integrator, steps=120, K=50, hold=40)
    gpu = _gpu_batched(bw, tpb=tpb)
    ref = _oracle_batched(bw)
    assert_parity(gpu, ref, bw.model_of_world[bw.world_of_drone()])


def test_log_uniform_swarms_first_principles():
    n = W.log_uniform_counts(5, 40, 300)
    bw = W.batched_workload(12, n, np.zeros(len(n), np.int32), integrator=ph.RK4, steps=100,
                            K=100, hold=50)
    gpu = _gpu_batched(bw)
    sample = np.random.default_rng(1).choice(bw.ntot, 400, replace=False)
    ref = _oracle_batched(bw, drones=sample)
    assert_parity(gpu[sample], ref, np.zeros(400, np.int64))


def test_batched_matches_uniform_path():
    """A batched handle over equal worlds of one model computes the same
    formulas as the uniform handle.  The two are separate kernels (per-world
    parameters in registers vs constant-bank operands), so the compiler may
    fuse multiply-adds differently: agreement to float32 rounding, not bits --
    per field, 1/100 of the field's parity tolerance against the FP64 oracle
    plus 1e-6 relative (a few float32 ulp)."""
    wl = W.attitude_swarm_rk4(M=777, steps=90, K=45)
    a = make_sim(wl)
    a.run(90, 45)
    sa = a.get_state().cpu().numpy()
    b = Sim.batched(np.ones(777, np.int64), np.zeros(777, np.int32), wl.integrator, wl.dt,
                    max_cmd_blocks=wl.cmd.shape[0])
    b.set_params(wl.params, np.zeros(777, np.int32))
    b.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
    b.set_commands(torch.tensor(wl.cmd, dtype=torch.float32, device="cuda"), wl.hold)
    b.run(90, 45)
    sb = b.get_state().cpu().numpy()
    for k, sl in FP_SLICES.items():
        np.testing.assert_allclose(sb[:, sl], sa[:, sl], rtol=1e-6, atol=1e-2 * TOL_FP[k], err_msg=k)


def test_mixed_swarm_full_size_sampled():
    """The mixed swarm at full size: 1000 worlds x 4000 drones (4M), even worlds
    first-principles, odd worlds abstracted with per-world coefficients,
    Euler, 200 steps in one launch; the oracle checks 64 sampled drones of each
    model.  The same 200 steps as 200 single-step launches (the HBM-bound mode,
    a kernel of its own) give the same bits on every drone."""
    wl = W.mixed_swarm_euler()
    sim = make_sim(wl)
    sim.run(wl.steps, wl.K)
    fused = sim.get_state()
    gpu = fused.cpu().numpy()
    assert sim.status() == 0
    single = make_sim(wl)
    single.run(wl.steps, 1)
    assert single.status() == 0
    assert torch.equal(single.get_state(), fused)
    del single
    rng = np.random.default_rng(2)
    models = wl.model_of_world[np.arange(wl.M * wl.N) // wl.N]
    sample = np.concatenate([rng.choice(np.nonzero(models == m)[0], 64, replace=False)
                             for m in (0, 1)])
    ref = ph.rollout_workload(wl, drones=sample).numpy()
    assert_parity(gpu[sample], ref, models[sample])


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_single_step_launches_match_fused(integrator):
    """K = 1 launches (the HBM-bound single-step mode, a kernel of its own) and
    fused launches give identical states on a mixed batch, both at parity with the
    oracle.  K = 7 splits every 10-step command block into odd runs of steps (the
    fused Euler loop is unrolled by two)."""
    bw = W.batched_workload(13, [100, 250, 3, 77], [0, 1, 1, 0], integrator=integrator, steps=40,
                            K=40, hold=10)
    a = _gpu_batched(bw, K=40)
    b = _gpu_batched(bw, K=1)
    c = _gpu_batched(bw, K=7)
    assert_parity(b, _oracle_batched(bw), bw.model_of_world[bw.world_of_drone()])
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)
