"""GPU BPTT training loop: the Adam kernel against the oracle's Adam, a few
training iterations against the FP64 oracle loop, and CUDA-graph replay of
whole iterations against eager iterations."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import policy as po
from oracle import training as tr
from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
from paper_2606_01478_b300 import _lib as L
from paper_2606_01478_b300.rollout import PolicyRollout
from paper_2606_01478_b300.train import PolicyTrainer

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_adam_kernel_matches_oracle():
    rng = np.random.default_rng(0)
    n = 5316
    w, g = rng.normal(size=n), rng.normal(size=n) * 0.1
    m, v = rng.normal(size=n) * 0.01, np.abs(rng.normal(size=n)) * 1e-3
    wt, gt, mt, vt = (torch.tensor(a, dtype=torch.float32, device="cuda") for a in (w, g, m, v))
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    step = torch.tensor([4], dtype=torch.int32, device="cuda")
    lib = L.load()
    r = lib.sim_adam_step(_p(gt), _p(wt), _p(mt), _p(vt), _p(wb), n, _p(step), 1e-2, 0.9, 0.999, 1e-8,
                          None)
    assert r == L.SIM_OK
    torch.cuda.synchronize()
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    # the kernel receives float32 hyper-parameters: give the oracle the same values
    h = lambda x: float(np.float32(x))
    w2, m2, v2 = tr.adam(f(w), f(g), f(m), f(v), 5, h(1e-2), h(0.9), h(0.999), h(1e-8))
    np.testing.assert_allclose(wt.cpu().numpy(), w2, rtol=1e-5, atol=1e-7)
    # m cancels (0.9 m + 0.1 g with both terms ~1e-2): compare at the terms' fp32 rounding
    np.testing.assert_allclose(mt.cpu().numpy(), m2, rtol=1e-5, atol=3e-8)
    np.testing.assert_allclose(vt.cpu().numpy(), v2, rtol=1e-5, atol=1e-12)
    assert torch.equal(wb, wt.to(torch.bfloat16))
    assert step.item() == 5
    assert lib.sim_adam_step(_p(gt), _p(wt), _p(mt), _p(vt), _p(wb), n, _p(step), 1e-2, 1.0, 0.999,
                             1e-8, None) == L.SIM_EINVAL


def _trainer(rw, lr, reward=None):
    sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, reward=reward, action_repeat=rw.repeat)
    w0 = torch.tensor(po.pack(rw.weights), dtype=torch.float32, device="cuda")
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
    return PolicyTrainer(runner, w0, lr), x0, p_ref


def test_training_iterations_match_oracle_loop():
    rw = W.policy_bptt(seed=61, M=64, H=40, C=10)
    lr, iters = 3e-3, 5
    tr_gpu, x0, p_ref = _trainer(rw, lr)
    losses = []
    for _ in range(iters):
        losses.append(tr_gpu.iteration(x0, p_ref).item())
    ref_losses, w_ref = tr.train(rw.x0.astype(np.float32).astype(np.float64),
                                 rw.p_ref.astype(np.float32).astype(np.float64), rw.params,
                                 po.pack(rw.weights), iters, lr, rw.dt, rw.H, rw.w_act)
    np.testing.assert_allclose(losses, ref_losses, rtol=1e-3)
    w_gpu = tr_gpu.w.cpu().numpy().astype(np.float64)
    w0 = po.pack(rw.weights)
    # the weights' displacement from the start agrees to 1e-3 of its size
    assert np.linalg.norm((w_gpu - w0) - (w_ref - w0)) <= 1e-3 * np.linalg.norm(w_ref - w0)
    assert tr_gpu.step.item() == iters


def test_reward_training_iterations_match_oracle_loop():
    """The paper's setting: 16 environments, 40 policy steps per rollout at
    50 Hz (10 physics steps each), the tracking reward; five iterations against
    the FP64 oracle loop."""
    rw = W.policy_bptt(seed=62, M=16, H=40, C=40, repeat=10)
    lr, iters = 3e-3, 5
    tr_gpu, x0, p_ref = _trainer(rw, lr, po.TRACKING_REWARD)
    losses = [tr_gpu.iteration(x0, p_ref).item() for _ in range(iters)]
    ref_losses, w_ref = tr.train(rw.x0.astype(np.float32).astype(np.float64),
                                 rw.p_ref.astype(np.float32).astype(np.float64), rw.params,
                                 po.pack(rw.weights), iters, lr, rw.dt, rw.H, rw.w_act,
                                 reward=po.TRACKING_REWARD, repeat=rw.repeat)
    np.testing.assert_allclose(losses, ref_losses, rtol=1e-3)
    w_gpu = tr_gpu.w.cpu().numpy().astype(np.float64)
    w0 = po.pack(rw.weights)
    assert np.linalg.norm((w_gpu - w0) - (w_ref - w0)) <= 1e-3 * np.linalg.norm(w_ref - w0)


def test_graph_replay_equals_eager_iterations():
    rw = W.policy_bptt(seed=62, M=128, H=30, C=10)
    a, x0, p_ref = _trainer(rw, 1e-2)
    for _ in range(4):
        a.iteration(x0, p_ref)
    b, _, _ = _trainer(rw, 1e-2)
    g = b.capture(x0, p_ref)
    assert b.step.item() == 0
    for _ in range(4):
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.w, b.w) and torch.equal(a.wb, b.wb) and b.step.item() == 4
    assert torch.equal(a.loss, b.loss)
