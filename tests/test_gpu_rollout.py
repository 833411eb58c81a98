"""GPU parity of the differentiable policy rollout (forward loss, dL/dW and
dL/dx0 from the hand-written adjoint kernels) against the FP64 oracle, whose
autograd gradient is itself pinned by central finite differences.  Bar:
relative error <= 1e-3 (norm-wise, per parameter tensor and per state group)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import policy as po
from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
from paper_2606_01478_b300.rollout import TRACKING_REWARD, PolicyRollout, rollout_loss

pytestmark = pytest.mark.gpu

TOL = 1e-3
GROUPS = {"p": slice(0, 3), "q": slice(3, 7), "v": slice(7, 10), "w": slice(10, 13),
          "W": slice(13, 17)}


# tracking-reward weights that exercise every action channel
REWARD_GENERAL = {"w_theta": 0.23, "w_act": (0.3, 0.05, 0.2, 0.11), "w_dact": (0.7, 1.3, 0.4, 0.9)}


def _gpu_inputs(rw, reward=None):
    sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, reward=reward, action_repeat=rw.repeat)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
    w = torch.tensor(po.pack(rw.weights), dtype=torch.float32, device="cuda")
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
    return sim, runner, x0, w, p_ref


def _as_oracle_inputs(rw):
    """The FP32-rounded inputs the GPU sees, held exactly in float64."""
    x0 = rw.x0.astype(np.float32).astype(np.float64)
    p_ref = rw.p_ref.astype(np.float32).astype(np.float64)
    return x0, p_ref


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-30))


def _check(rw, loss, dW, dx0, drones=None, reward=None):
    x0, p_ref = _as_oracle_inputs(rw)
    sel = np.arange(rw.M) if drones is None else np.asarray(drones)
    L_ref, per, dW_ref, dx_ref = po.rollout_grad(x0[sel], rw.weights, p_ref[:, sel], rw.params,
                                                 rw.dt, rw.H, rw.w_act, reward, rw.repeat)
    dx_ref = dx_ref * len(sel) / rw.M  # the GPU loss is the mean over all M drones
    errs = {}
    if drones is None:
        errs["loss"] = abs(loss - L_ref) / abs(L_ref)
        for k in po.NAMES:
            errs[k] = _rel(po.unpack(dW)[k], dW_ref[k])
    for gname, s in GROUPS.items():
        errs["dx0_" + gname] = _rel(dx0[sel][:, s], dx_ref[:, s])
    bad = {k: v for k, v in errs.items() if not v <= TOL}
    assert not bad, f"relative errors above {TOL}: {bad}; all: {errs}"
    return errs


def test_rollout_gradient_small_ragged():
    """200 drones (ragged last CTA of 8), H = 30, C = 7 (last segment short)."""
    rw = W.policy_bptt(seed=31, M=200, H=30, C=7)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    assert torch.isfinite(dW).all() and torch.isfinite(dx0).all()
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64))
    assert torch.all(dx0[:, 17:20] == 0)


@pytest.mark.parametrize("C", [25, 250, 1])
def test_rollout_gradient_full_horizon(C):
    """The full BPTT horizon (H = 250 Euler steps at 500 Hz) at 256 drones, with
    checkpoint intervals 25 (the configured), 250 (one segment) and 1."""
    rw = W.policy_bptt(seed=32, M=256, H=250, C=C)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64))


def test_rollout_full_size_sampled_and_linearity():
    """The full BPTT workload (8192 drones, H = 250, C = 25): dL/dx0 of 16 sampled
    drones against the oracle (exact per drone), and dW consistent with the
    drone-count-weighted gradients of two disjoint halves."""
    rw = W.policy_bptt()
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    wb = w.to(torch.bfloat16)
    loss, dW, dx0 = runner.grad(x0, wb, p_ref)
    sample = np.random.default_rng(9).choice(rw.M, 16, replace=False)
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64), drones=sample)
    halves = []
    for lo, hi in ((0, 4096), (4096, 8192)):
        s2 = Sim(hi - lo, 1, FIRST_PRINCIPLES, EULER, rw.dt)
        s2.set_params(rw.params)
        r2 = PolicyRollout(s2, rw.H, rw.C, rw.w_act)
        l2, g2, _ = r2.grad(x0[lo:hi].contiguous(), wb, p_ref[:, lo:hi].contiguous())
        halves.append((l2.item(), g2))
    comb = 0.5 * (halves[0][1] + halves[1][1])
    assert _rel(dW.cpu().numpy(), comb.cpu().numpy()) < 1e-5
    assert abs(loss.item() - 0.5 * (halves[0][0] + halves[1][0])) < 1e-5 * abs(loss.item())


def test_rollout_gradient_1024_drones_against_oracle():
    """dW over 16 CTAs of 64 drones (1024 drones, ragged-free), the full horizon
    H = 250 with C = 25: the per-CTA partials and their fixed-order reduction
    against the oracle's FP64 adjoint, with dL/dx0 of every drone."""
    rw = W.policy_bptt(seed=43, M=1024, H=250, C=25)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64))


def test_rollout_deterministic():
    rw = W.policy_bptt(seed=33, M=300, H=40, C=10)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    wb = w.to(torch.bfloat16)
    a = runner.grad(x0, wb, p_ref)
    b = runner.grad(x0, wb, p_ref)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


@pytest.mark.parametrize("M,H,C,repeat,reward,prec", [
    (300, 40, 10, 1, None, "hilo"),            # ragged last CTA, four segments
    (100, 23, 5, 1, TRACKING_REWARD, "hilo"),  # ragged last segment, tracking reward
    (64, 7, 7, 1, None, "bf16"),               # one segment: the forward pass records it
    (70, 12, 6, 10, TRACKING_REWARD, "bf16"),  # two segments, actions held for 10 steps
    (1, 1, 1, 1, None, "hilo"),                # one drone (63 padded rows), one step
    (33, 2, 1, 1, TRACKING_REWARD, "hilo"),    # two one-step segments
    (96, 5, 2, 3, None, "hilo"),               # three segments, the last of one step
])
def test_fused_gradient_equals_forward_then_backward(M, H, C, repeat, reward, prec):
    """sim_rollout_grad runs the forward pass inside the adjoint launch; its loss,
    dW and dx0 equal sim_rollout_fwd followed by sim_rollout_bwd bit for bit, and a
    backward after it (from the checkpoints it left) gives the same again."""
    rw = W.policy_bptt(seed=35, M=M, H=H, C=C, repeat=repeat)
    sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, reward=reward, action_repeat=rw.repeat, precision=prec)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
    wb = torch.tensor(po.pack(rw.weights), dtype=torch.float32, device="cuda").to(torch.bfloat16)
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
    one = torch.ones(1, device="cuda")
    loss_f = runner.forward(x0, wb, p_ref)
    dW_s, dx_s = runner.backward(x0, wb, p_ref, one)
    loss_g, dW_g, dx_g = runner.grad(x0, wb, p_ref)
    dW_b, dx_b = runner.backward(x0, wb, p_ref, one)
    torch.cuda.synchronize()
    assert sim.status() == 0
    assert torch.isfinite(dW_g).all() and torch.isfinite(dx_g).all()
    assert torch.equal(loss_f, loss_g)
    for a, b in ((dW_s, dW_g), (dx_s, dx_g), (dW_s, dW_b), (dx_s, dx_b)):
        assert torch.equal(a, b)


def test_autograd_function_matches_direct_call():
    rw = W.policy_bptt(seed=34, M=128, H=20, C=5)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    xr = x0.clone().requires_grad_(True)
    wr = w.clone().requires_grad_(True)
    L = rollout_loss(xr, wr, runner, p_ref)
    (3.0 * L).backward()
    assert torch.allclose(L.detach(), loss[0])
    # the upstream gradient scales the adjoint seed inside the kernel, so fp32
    # rounding differs from scaling the unit-seed result afterwards
    assert _rel(wr.grad.cpu().numpy(), 3.0 * dW.cpu().numpy()) < 1e-5
    assert _rel(xr.grad.cpu().numpy(), 3.0 * dx0.cpu().numpy()) < 1e-5


def test_zero_policy_hover_loss():
    """Zero weights: a = 0 (hover command); drones at hover on a stationary
    reference displaced by a constant offset give loss H |offset|^2."""
    rw = W.policy_bptt(seed=35, M=64, H=50, C=10)
    rw.weights = {k: np.zeros(po.SIZES[k]) for k in po.NAMES}
    rw.x0[:, 7:13] = 0
    rw.x0[:, 3:7] = [0, 0, 0, 1]
    off = np.array([0.05, -0.1, 0.2], dtype=np.float32)
    rw.p_ref = np.broadcast_to(rw.x0[None, :, 0:3].astype(np.float32) + off,
                               (rw.H + 1, rw.M, 3)).copy()
    sim, runner, x0, w, p_ref = _gpu_inputs(rw)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    expect = rw.H * float((off.astype(np.float64) ** 2).sum())
    assert abs(loss.item() - expect) <= 1e-5 * expect


# ---------------------------------------------------------------- tracking reward


@pytest.mark.parametrize("reward", [TRACKING_REWARD, REWARD_GENERAL], ids=["paper", "general"])
def test_reward_gradient_small_ragged(reward):
    """The paper's tracking reward: 200 drones (ragged last CTA), H = 30, C = 7
    (the smoothness adjoint crosses segment boundaries)."""
    rw = W.policy_bptt(seed=35, M=200, H=30, C=7)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw, reward)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    assert torch.isfinite(dW).all() and torch.isfinite(dx0).all()
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64), reward=reward)


@pytest.mark.parametrize("C", [40, 1])
def test_reward_gradient_training_shape(C):
    """The paper's BPTT setting (16 environments, 40 steps) and a long horizon
    (256 drones, H = 250, C = 25)."""
    rw = W.policy_bptt(seed=36, M=16, H=40, C=C)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw, TRACKING_REWARD)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64), reward=TRACKING_REWARD)
    rw = W.policy_bptt(seed=37, M=256, H=250, C=25)
    sim, runner, x0, w, p_ref = _gpu_inputs(rw, TRACKING_REWARD)
    loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
    _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64), reward=TRACKING_REWARD)


def test_objectives_share_a_handle():
    """Two runners with different objectives on one handle: each call applies its
    own objective (the results equal those of separate handles)."""
    rw = W.policy_bptt(seed=38, M=96, H=24, C=6)
    sim, sq, x0, w, p_ref = _gpu_inputs(rw)
    rew = PolicyRollout(sim, rw.H, rw.C, rw.w_act, reward=TRACKING_REWARD)
    wb = w.to(torch.bfloat16)
    a1 = [t.clone() for t in sq.grad(x0, wb, p_ref)]
    b1 = [t.clone() for t in rew.grad(x0, wb, p_ref)]
    a2 = sq.grad(x0, wb, p_ref)
    for u, v in zip(a1, a2):
        assert torch.equal(u, v)
    _, ref_runner, _, _, _ = _gpu_inputs(rw, TRACKING_REWARD)
    b2 = ref_runner.grad(x0, wb, p_ref)
    for u, v in zip(b1, b2):
        assert torch.equal(u, v)
    assert not torch.equal(a1[1], b1[1])


@pytest.mark.parametrize("reward", [None, TRACKING_REWARD], ids=["squared", "reward"])
def test_held_action_gradient(reward):
    """Policy actions held for R = 10 physics steps (50 Hz policy, 500 Hz
    physics): 100 drones (ragged), H = 16 policy steps, C = 5 (ragged last
    segment); and the paper's training shape, 16 environments x 40 steps."""
    for rw in (W.policy_bptt(seed=39, M=100, H=16, C=5, repeat=10),
               W.policy_bptt(seed=40, M=16, H=40, C=10, repeat=10)):
        sim, runner, x0, w, p_ref = _gpu_inputs(rw, reward)
        loss, dW, dx0 = runner.grad(x0, w.to(torch.bfloat16), p_ref)
        assert torch.isfinite(dW).all()
        _check(rw, loss.item(), dW.cpu().numpy(), dx0.cpu().numpy().astype(np.float64), reward=reward)


def test_plain_bf16_operands_mode():
    """SIM_MLP_BF16 (plain bf16 tensor-core operands) at the full BPTT horizon
    (H = 250, C = 25, 256 drones): gradients against the FP64 oracle within
    the 1e-3 norm-wise relative bar (the measured errors are printed), and
    measurably less accurate than the default hi + lo split, so the mode really
    changes the arithmetic."""
    rw = W.policy_bptt(seed=41, M=256, H=250, C=25)
    x0, p_ref = _as_oracle_inputs(rw)
    L_ref, _, dW_ref, dx_ref = po.rollout_grad(x0, rw.weights, p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    errs = {}
    for prec in ("hilo", "bf16"):
        sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt)
        sim.set_params(rw.params)
        runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, precision=prec)
        xg = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
        w = torch.tensor(po.pack(rw.weights), dtype=torch.float32, device="cuda").to(torch.bfloat16)
        pg = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
        loss, dW, dx0 = runner.grad(xg, w, pg)
        g = po.pack(dW_ref)
        errs[prec] = (abs(loss.item() - L_ref) / abs(L_ref),
                      _rel(dW.cpu().numpy(), g), _rel(dx0.cpu().numpy(), dx_ref))
    print("relative errors (loss, dW, dx0):", errs)
    assert max(errs["hilo"]) <= TOL
    assert max(errs["bf16"]) <= TOL
    assert errs["bf16"][1] > errs["hilo"][1]
