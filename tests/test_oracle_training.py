"""Pins of the training-loop oracle: Adam's closed forms and convergence,
bf16 rounding against torch's independent conversion, and the loss falling
over a few BPTT iterations."""
import numpy as np
import torch

import workloads as W
from oracle import policy as po
from oracle import training as tr


def test_adam_first_step_and_constant_gradient_closed_form():
    rng = np.random.default_rng(0)
    w0 = rng.normal(size=100)
    g = rng.normal(size=100)
    lr, eps = 0.01, 1e-8
    w, m, v = w0.copy(), np.zeros(100), np.zeros(100)
    for t in range(1, 6):
        w_prev = w
        w, m, v = tr.adam(w, g, m, v, t, lr, eps=eps)
        # bias correction makes m_hat = g and v_hat = g^2 for a constant gradient
        np.testing.assert_allclose(w - w_prev, -lr * g / (np.abs(g) + eps), rtol=1e-9, atol=1e-15)


def test_adam_converges_on_a_quadratic():
    rng = np.random.default_rng(1)
    target = rng.normal(size=50)
    w = np.zeros(50)
    m = v = np.zeros(50)
    for t in range(1, 3001):
        w, m, v = tr.adam(w, w - target, m, v, t, 0.05)
    assert np.abs(w - target).max() < 1e-3


def test_round_bf16_matches_torch():
    x = np.random.default_rng(2).normal(0, 3, 100_000)
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(tr.round_bf16(x), ref)


def test_loss_falls_over_iterations():
    rw = W.policy_bptt(seed=51, M=16, H=40, C=10)
    losses, w = tr.train(rw.x0, rw.p_ref, rw.params, po.pack(rw.weights), 8, 3e-3, rw.dt, rw.H,
                         rw.w_act)
    assert losses[-1] < losses[0]


def test_reward_loss_falls_over_iterations():
    """The loop under the paper's tracking reward (16 environments, 40 steps)
    improves the reward."""
    rw = W.policy_bptt(seed=51, M=16, H=40, C=10)
    losses, _ = tr.train(rw.x0, rw.p_ref, rw.params, po.pack(rw.weights), 8, 3e-3, rw.dt, rw.H,
                         0.0, reward=po.TRACKING_REWARD)
    assert losses[-1] < losses[0]
    assert np.all(losses > -rw.H)  # the reward of a step is at most 1
