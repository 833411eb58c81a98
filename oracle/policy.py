"""FP64 oracle of the differentiable policy rollout (BPTT).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper trains tracking policies by backpropagation through time through
the full dynamics and the onboard controller stack (Results, Trajectory
Tracking Benchmark; Materials and Methods, Backpropagation Through Time).  This
module computes, for a batch of M independent drones:

    obs_k = [p_k - r_k, q_k, v_k, w_k]                      (13)
    a_k   = tanh(W3 tanh(W2 tanh(W1 obs_k + b1) + b2) + b3) (4, attitude action)
    x_{k+1} = step^R(x_k, a_k) first-principles model, attitude interface, Euler;
                               the action is held for R >= 1 physics steps (R = 10
                               runs a 50 Hz policy on 500 Hz physics, the paper's
                               recommended attitude-interface rate)
    L = (1/M) sum_w sum_{k=0}^{H-1} ( |p_{k+1} - r_{k+1}|^2 + w_act |a_k|^2 )

with r_k the reference position table (a figure-8 sampled per drone; an input).

Second objective, the paper's trajectory-tracking reward (Materials and
Methods, Backpropagation Through Time: the reward equation and the BPTT
hyper-parameter table), discount 1, as a loss to minimise:

    L = (1/M) sum_w sum_{k=0}^{H-1} -( exp(-2 |p_{k+1} - r_{k+1}|) - w_theta theta_{k+1}
            - sum_i w_act,i (a_k,i - a_hover,i)^2 - sum_i w_dact,i (a_k,i - a_{k-1},i)^2 )

theta = angle between the body z axis and world z (tilt from upright; yaw does
not count), a_hover = 0 (the attitude action map puts hover at a = 0), and
a_{-1} = a_hover.  The kinks of |p - r| and theta at zero get gradient 0.

The policy weights are bf16 values held exactly in float64.  The gradient of L
with respect to all weights and biases and the initial state is that of this
exact discrete computation, taken with torch.autograd.

Parity status: the squared loss is the reading adopted here; parity unpinned
against the paper.  The tracking reward follows the paper's equation and table
(a_hover, a_{-1} and the tilt definition are readings).  Pinned in
tests/test_oracle_policy.py by central finite differences of both losses
(float64), the zero-policy hover case (loss and closed-form offset loss, for
both objectives), the action and smoothness penalties of a constant policy in
closed form, the tilt angle against scipy's rotation matrices, a constant
policy held R steps against R times as many single steps, and structural
properties of the MLP.
"""
from __future__ import annotations

import torch

from . import physics as ph

F64 = torch.float64
NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")
SIZES = {"W1": (64, 13), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (4, 64), "b3": (4,)}


def weights_tensors(weights: dict, requires_grad: bool = False) -> dict:
    return {k: torch.tensor(weights[k], dtype=F64, requires_grad=requires_grad) for k in NAMES}


def mlp(obs: torch.Tensor, W: dict) -> torch.Tensor:
    """13 -> 64 -> 64 -> 4 with tanh after every layer."""
    h1 = torch.tanh(obs @ W["W1"].T + W["b1"])
    h2 = torch.tanh(h1 @ W["W2"].T + W["b2"])
    return torch.tanh(h2 @ W["W3"].T + W["b3"])


def observation(x: torch.Tensor, r: torch.Tensor) -> torch.Tensor:
    return torch.cat([x[:, 0:3] - r, x[:, 3:13]], dim=-1)


# weights of the paper's tracking reward (BPTT hyper-parameter table)
TRACKING_REWARD = {"w_theta": 0.1, "w_act": (0.12, 0.12, 0.0, 0.02), "w_dact": (1.4, 1.4, 0.0, 0.8)}


def _norm(v: torch.Tensor) -> torch.Tensor:
    """Euclidean norm over the last axis whose gradient at 0 is 0."""
    n2 = (v * v).sum(-1)
    pos = n2 > 0
    return torch.where(pos, torch.sqrt(torch.where(pos, n2, torch.ones_like(n2))), torch.zeros_like(n2))


def tilt(q: torch.Tensor) -> torch.Tensor:
    """Angle from upright of unit quaternions [x, y, z, w]: the body z axis is
    R(q) e_z, whose world-z component is 1 - 2 (x^2 + y^2) = cos(theta), so
    theta = 2 atan2(|(x, y)|, |(z, w)|)."""
    return 2.0 * torch.atan2(_norm(q[:, 0:2]), _norm(q[:, 2:4]))


def tracking_reward(x_next, r_next, a, a_prev, reward: dict) -> torch.Tensor:
    """Per-drone reward of one step (the paper's tracking reward, a_hover = 0)."""
    w_act = torch.tensor(reward["w_act"], dtype=F64)
    w_dact = torch.tensor(reward["w_dact"], dtype=F64)
    return (torch.exp(-2.0 * _norm(x_next[:, 0:3] - r_next)) - reward["w_theta"] * tilt(x_next[:, 3:7])
            - (w_act * a * a).sum(-1) - (w_dact * (a - a_prev) ** 2).sum(-1))


def rollout_loss(x0, W: dict, p_ref, params: dict, dt: float, H: int, w_act: float,
                 reward: dict | None = None, repeat: int = 1):
    """Returns (L, per-drone loss [M], final state [M, 20]).  reward=None: the
    squared tracking loss with action weight w_act; otherwise the paper's
    tracking reward with the weights in `reward` (w_act is then unused).  Each
    of the H policy actions is held for `repeat` physics steps of dt."""
    x = torch.as_tensor(x0, dtype=F64) if not torch.is_tensor(x0) else x0
    r = torch.as_tensor(p_ref, dtype=F64)
    M = x.shape[0]
    P = ph.param_batch([params], [0] * M)
    per = torch.zeros(M, dtype=F64)
    a_prev = torch.zeros(M, 4, dtype=F64)
    for k in range(H):
        a = mlp(observation(x, r[k]), W)
        for _ in range(repeat):
            x = ph.step(x, a, P, dt, ph.EULER, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        if reward is None:
            per = per + ((x[:, 0:3] - r[k + 1]) ** 2).sum(-1) + w_act * (a * a).sum(-1)
        else:
            per = per - tracking_reward(x, r[k + 1], a, a_prev, reward)
        a_prev = a
    return per.sum() / M, per, x


def rollout_grad(x0, weights: dict, p_ref, params: dict, dt: float, H: int, w_act: float,
                 reward: dict | None = None, repeat: int = 1):
    """Loss and its gradient w.r.t. the weights (dict of float64 arrays) and the
    initial state [M, 20] (the three integrator slots get zero gradient: the
    attitude interface does not use them)."""
    W = weights_tensors(weights, requires_grad=True)
    x0t = torch.tensor(x0, dtype=F64, requires_grad=True)
    L, per, _ = rollout_loss(x0t, W, p_ref, params, dt, H, w_act, reward, repeat)
    grads = torch.autograd.grad(L, [x0t] + [W[k] for k in NAMES])
    dx0 = grads[0].detach().numpy()
    dW = {k: g.detach().numpy() for k, g in zip(NAMES, grads[1:])}
    return float(L.detach()), per.detach().numpy(), dW, dx0


def pack(weights: dict):
    """Concatenate W1, b1, W2, b2, W3, b3 (row-major) into one flat array."""
    import numpy as np
    return np.concatenate([np.asarray(weights[k], dtype=np.float64).ravel() for k in NAMES])


def unpack(flat):
    import numpy as np
    out, o = {}, 0
    for k in NAMES:
        n = int(np.prod(SIZES[k]))
        out[k] = np.asarray(flat[o:o + n]).reshape(SIZES[k])
        o += n
    return out
