"""Pins of the policy-rollout oracle: float64 central finite differences of the
loss (so the autograd gradient is checked against an independent numerical
derivative), the zero-policy hover case and MLP structure."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import physics as ph
from oracle import policy as po

F64 = torch.float64


def _small(M=6, H=30, seed=3):
    return W.policy_bptt(seed=seed, M=M, H=H, C=10)


def _loss(rw, x0, weights):
    Wt = po.weights_tensors(weights)
    L, _, _ = po.rollout_loss(torch.tensor(x0), Wt, rw.p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    return float(L)


def test_gradient_matches_central_differences_weights():
    rw = _small()
    L, _, dW, _ = po.rollout_grad(rw.x0, rw.weights, rw.p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    flat = po.pack(rw.weights)
    g = po.pack(dW)
    rng = np.random.default_rng(0)
    h = 1e-5
    # individual coordinates of every tensor + random directions over all
    idx = [0, 5, 12, 832 + 3, 896 + 100, 896 + 4095, 4992 + 7, 5056 + 200, 5312, 5315]
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (_loss(rw, rw.x0, po.unpack(flat + e)) - _loss(rw, rw.x0, po.unpack(flat - e))) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
    for _ in range(3):
        d = rng.normal(size=flat.shape)
        d /= np.linalg.norm(d)
        fd = (_loss(rw, rw.x0, po.unpack(flat + h * d)) - _loss(rw, rw.x0, po.unpack(flat - h * d))) / (2 * h)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(g @ d))


def test_gradient_matches_central_differences_initial_state():
    rw = _small(M=4, H=25)
    _, _, _, dx0 = po.rollout_grad(rw.x0, rw.weights, rw.p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    h = 1e-6
    for (w, j) in [(0, 0), (1, 2), (2, 4), (3, 6), (0, 8), (1, 11), (2, 12), (3, 15)]:
        xp, xm = rw.x0.copy(), rw.x0.copy()
        scale = 1e4 if j >= 13 else 1.0  # rotor speeds are O(1e4) RPM
        xp[w, j] += h * scale
        xm[w, j] -= h * scale
        fd = (_loss(rw, xp, rw.weights) - _loss(rw, xm, rw.weights)) / (2 * h * scale)
        assert abs(fd - dx0[w, j]) <= 1e-6 * max(1.0, abs(dx0[w, j])) + 1e-10, (w, j, fd, dx0[w, j])
    assert np.all(dx0[:, 17:20] == 0)


def test_zero_policy_at_hover_has_closed_form_loss():
    """All-zero weights give a = tanh(0) = 0: hover command, so a drone at hover
    stays put; the loss is H |offset|^2 for a reference displaced by a constant
    offset (and exactly 0 without offset), and the action term vanishes."""
    rw = _small(M=3, H=40)
    zero = {k: np.zeros(po.SIZES[k]) for k in po.NAMES}
    x0 = np.zeros((3, 20))
    x0[:, 0:3] = [[0.0, 0.0, 1.0], [0.3, -0.2, 1.5], [-1.0, 2.0, 0.5]]
    x0[:, 6] = 1.0
    x0[:, 13:17] = W.hover_rpm(rw.params)
    ref = np.broadcast_to(x0[None, :, 0:3], (rw.H + 1, 3, 3)).copy()
    Wt = po.weights_tensors(zero)
    L0, _, xf = po.rollout_loss(torch.tensor(x0), Wt, ref, rw.params, rw.dt, rw.H, rw.w_act)
    assert float(L0) < 1e-20
    assert np.abs(xf.numpy()[:, 0:13] - x0[:, 0:13]).max() < 1e-12
    off = np.array([0.1, -0.2, 0.05])
    L1, per, _ = po.rollout_loss(torch.tensor(x0), Wt, ref + off, rw.params, rw.dt, rw.H, rw.w_act)
    np.testing.assert_allclose(per.numpy(), rw.H * (off ** 2).sum(), rtol=1e-12)


def test_mlp_odd_symmetry_and_linear_limit():
    rng = np.random.default_rng(4)
    Wd = {k: rng.normal(0, 0.3, po.SIZES[k]) for k in po.NAMES}
    for k in ("b1", "b2", "b3"):
        Wd[k][:] = 0
    Wt = po.weights_tensors(Wd)
    obs = torch.tensor(rng.normal(size=(7, 13)))
    assert torch.allclose(po.mlp(-obs, Wt), -po.mlp(obs, Wt), atol=0)
    # tiny inputs: tanh is the identity to first order, so the MLP is the matrix product
    eps = 1e-7
    lin = obs @ (Wt["W3"] @ Wt["W2"] @ Wt["W1"]).T
    assert torch.allclose(po.mlp(eps * obs, Wt) / eps, lin, rtol=1e-9, atol=1e-12)


def test_policy_weights_are_bf16_values():
    w = W.policy_weights(7)
    for k in po.NAMES:
        a = np.asarray(w[k], dtype=np.float32)
        assert np.all((a.view(np.uint32) & 0xFFFF) == 0)
        assert np.array_equal(a.astype(np.float64), w[k])


# ---------------------------------------------------------------- tracking reward

REWARD_GENERAL = {"w_theta": 0.23, "w_act": (0.3, 0.05, 0.2, 0.11), "w_dact": (0.7, 1.3, 0.4, 0.9)}


def _rloss(rw, x0, weights, reward):
    Wt = po.weights_tensors(weights)
    L, _, _ = po.rollout_loss(torch.tensor(x0), Wt, rw.p_ref, rw.params, rw.dt, rw.H, rw.w_act, reward)
    return float(L)


def test_tilt_matches_rotation_matrix():
    """theta against arccos of scipy's R[2, 2] (an independent rotation
    library); yaw does not change it; a pure roll gives |roll|."""
    from scipy.spatial.transform import Rotation
    rot = Rotation.random(200, random_state=5)
    q = rot.as_quat()
    ref = np.arccos(np.clip(rot.as_matrix()[:, 2, 2], -1, 1))
    th = po.tilt(torch.tensor(q)).numpy()
    np.testing.assert_allclose(th, ref, atol=1e-7)
    yawed = (Rotation.from_euler("z", np.linspace(-3, 3, 200)[:, None]) * rot).as_quat()
    np.testing.assert_allclose(po.tilt(torch.tensor(yawed)).numpy(), th, atol=1e-12)
    roll = np.linspace(-3.1, 3.1, 41)
    qr = Rotation.from_euler("x", roll[:, None]).as_quat()
    np.testing.assert_allclose(po.tilt(torch.tensor(qr)).numpy(), np.abs(roll), atol=1e-12)


def test_reward_zero_policy_at_hover_closed_form():
    """Zero weights: a = 0 = a_hover, the drone stays at hover, upright: every
    step earns exp(-2 |offset|), so the loss is -H exp(-2 |offset|)."""
    rw = _small(M=3, H=40)
    zero = {k: np.zeros(po.SIZES[k]) for k in po.NAMES}
    x0 = np.zeros((3, 20))
    x0[:, 0:3] = [[0.0, 0.0, 1.0], [0.3, -0.2, 1.5], [-1.0, 2.0, 0.5]]
    x0[:, 6] = 1.0
    x0[:, 13:17] = W.hover_rpm(rw.params)
    ref = np.broadcast_to(x0[None, :, 0:3], (rw.H + 1, 3, 3)).copy()
    Wt = po.weights_tensors(zero)
    for reward in (po.TRACKING_REWARD, REWARD_GENERAL):
        _, per, _ = po.rollout_loss(torch.tensor(x0), Wt, ref, rw.params, rw.dt, rw.H, 0.0, reward)
        np.testing.assert_allclose(per.numpy(), -rw.H, rtol=1e-14)
        off = np.array([0.1, -0.2, 0.05])
        _, per, _ = po.rollout_loss(torch.tensor(x0), Wt, ref + off, rw.params, rw.dt, rw.H, 0.0, reward)
        np.testing.assert_allclose(per.numpy(), -rw.H * np.exp(-2 * np.linalg.norm(off)), rtol=1e-12)


def test_reward_constant_policy_penalties_closed_form():
    """A policy whose output is the constant a = tanh(b3) (W3 = 0): the action
    penalty is H sum_i w_act,i a_i^2 and the smoothness penalty only sees the
    first step (from a_{-1} = a_hover = 0): sum_i w_dact,i a_i^2.  The
    dynamics terms cancel in the difference of two objectives."""
    rw = _small(M=4, H=30)
    wts = {k: np.array(v, dtype=np.float64) for k, v in rw.weights.items()}
    wts["W3"] = np.zeros_like(wts["W3"])
    wts["b3"] = np.array([0.4, -0.25, 0.1, 0.3])
    a = np.tanh(wts["b3"])
    base = dict(REWARD_GENERAL, w_act=(0, 0, 0, 0), w_dact=(0, 0, 0, 0))
    diff = _rloss(rw, rw.x0, wts, REWARD_GENERAL) - _rloss(rw, rw.x0, wts, base)
    expect = rw.H * (np.array(REWARD_GENERAL["w_act"]) * a * a).sum() + \
        (np.array(REWARD_GENERAL["w_dact"]) * a * a).sum()
    assert abs(diff - expect) <= 1e-12 * abs(expect)


def _tilted(rw, seed=11):
    """The BPTT workload starts upright with zero body rate, so the tilt sits on its
    kink for the first steps; finite differences need states off the kink."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    x0 = rw.x0.copy()
    x0[:, 3:7] = Rotation.from_euler("xyz", rng.uniform(-0.2, 0.2, (len(x0), 3))).as_quat()
    x0[:, 10:13] = rng.uniform(-1, 1, (len(x0), 3))
    rw.x0 = x0
    return rw


@pytest.mark.parametrize("reward", [po.TRACKING_REWARD, REWARD_GENERAL])
def test_reward_gradient_matches_central_differences(reward):
    rw = _tilted(_small(M=4, H=25))
    _, _, dW, dx0 = po.rollout_grad(rw.x0, rw.weights, rw.p_ref, rw.params, rw.dt, rw.H, 0.0, reward)
    flat = po.pack(rw.weights)
    g = po.pack(dW)
    h = 1e-5
    for i in [3, 832 + 9, 896 + 2000, 4992 + 60, 5056 + 17, 5056 + 255, 5313, 5315]:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (_rloss(rw, rw.x0, po.unpack(flat + e), reward) -
              _rloss(rw, rw.x0, po.unpack(flat - e), reward)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
    d = np.random.default_rng(9).normal(size=flat.shape)
    d /= np.linalg.norm(d)
    fd = (_rloss(rw, rw.x0, po.unpack(flat + h * d), reward) -
          _rloss(rw, rw.x0, po.unpack(flat - h * d), reward)) / (2 * h)
    assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(g @ d))
    hx = 1e-6
    for (w, j) in [(0, 1), (1, 3), (2, 5), (3, 9), (0, 12), (1, 14)]:
        xp, xm = rw.x0.copy(), rw.x0.copy()
        scale = 1e4 if j >= 13 else 1.0
        xp[w, j] += hx * scale
        xm[w, j] -= hx * scale
        fd = (_rloss(rw, xp, rw.weights, reward) - _rloss(rw, xm, rw.weights, reward)) / (2 * hx * scale)
        assert abs(fd - dx0[w, j]) <= 1e-6 * max(1.0, abs(dx0[w, j])) + 1e-10, (w, j, fd, dx0[w, j])


def test_held_constant_policy_equals_single_steps():
    """A constant policy (W3 = 0) held R = 4 steps for H policy steps drives the
    same physics as H R single steps: identical final state, and the squared
    position terms of the held rollout are those of every R-th single step."""
    rw = _small(M=3, H=48)
    wts = {k: np.array(v, dtype=np.float64) for k, v in rw.weights.items()}
    wts["W3"] = np.zeros_like(wts["W3"])
    wts["b3"] = np.array([0.2, -0.1, 0.3, 0.15])
    Wt = po.weights_tensors(wts)
    R, Hp = 4, 12
    ref_single = rw.p_ref  # [49, M, 3]
    ref_held = rw.p_ref[::R]  # [13, M, 3]
    x0 = torch.tensor(rw.x0)
    _, per1, xf1 = po.rollout_loss(x0, Wt, ref_single, rw.params, rw.dt, Hp * R, 0.0)
    _, perR, xfR = po.rollout_loss(x0, Wt, ref_held, rw.params, rw.dt, Hp, 0.0, repeat=R)
    assert torch.equal(xf1, xfR)
    # position terms at every R-th step, recomputed from a single-step trajectory
    x = x0.clone()
    P = ph.param_batch([rw.params], [0] * 3)
    a = torch.tanh(torch.tensor(wts["b3"]))[None, :].expand(3, 4)
    expect = torch.zeros(3, dtype=F64)
    for k in range(Hp * R):
        x = ph.step(x, a, P, rw.dt, ph.EULER, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        if (k + 1) % R == 0:
            expect += ((x[:, 0:3] - torch.tensor(ref_single[k + 1])) ** 2).sum(-1)
    np.testing.assert_allclose(perR.numpy(), expect.numpy(), rtol=1e-13)


def test_held_policy_gradient_matches_central_differences():
    rw = _tilted(_small(M=3, H=12))
    R = 3
    _, _, dW, _ = po.rollout_grad(rw.x0, rw.weights, rw.p_ref, rw.params, rw.dt, rw.H, 0.0,
                                  po.TRACKING_REWARD, R)
    flat = po.pack(rw.weights)
    g = po.pack(dW)

    def f(v):
        Wt = po.weights_tensors(po.unpack(v))
        return float(po.rollout_loss(torch.tensor(rw.x0), Wt, rw.p_ref, rw.params, rw.dt, rw.H, 0.0,
                                     po.TRACKING_REWARD, R)[0])
    h = 1e-5
    for i in [7, 832 + 30, 896 + 3000, 5056 + 100, 5314]:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (f(flat + e) - f(flat - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_gradient_central_differences_step_1e4():
    """The BPTT workload's check as stated: FP64 central differences with h = 1e-4 on
    weights of every tensor and on initial-state entries (truncation error
    O(h^2) relative to the smooth loss; bound 1e-5 relative)."""
    rw = _small(M=8, H=40)
    L, _, dW, dx0 = po.rollout_grad(rw.x0, rw.weights, rw.p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    flat = po.pack(rw.weights)
    g = po.pack(dW)
    h = 1e-4
    for i in [1, 832 + 40, 896 + 1234, 4992 + 33, 5056 + 77, 5314]:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (_loss(rw, rw.x0, po.unpack(flat + e)) - _loss(rw, rw.x0, po.unpack(flat - e))) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (i, fd, g[i])
    for (w, j) in [(0, 1), (3, 5), (5, 9), (7, 11)]:
        xp, xm = rw.x0.copy(), rw.x0.copy()
        xp[w, j] += h
        xm[w, j] -= h
        fd = (_loss(rw, xp, rw.weights) - _loss(rw, xm, rw.weights)) / (2 * h)
        assert abs(fd - dx0[w, j]) <= 1e-5 * max(1.0, abs(dx0[w, j])), (w, j, fd, dx0[w, j])
