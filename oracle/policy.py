"""FP64 oracle of the differentiable policy rollout (BPTT).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper trains tracking policies by backpropagation through time through
the full dynamics and the onboard controller stack (Results, Trajectory
Tracking Benchmark; Materials and Methods, Backpropagation Through Time).  This
module computes, for a batch of M independent drones:

    obs_k = [p_k - r_k, q_k, v_k, w_k]                      (13)
    a_k   = tanh(W3 tanh(W2 tanh(W1 obs_k + b1) + b2) + b3) (4, attitude action)
    x_{k+1} = step(x_k, a_k)   first-principles model, attitude interface, Euler
    L = (1/M) sum_w sum_{k=0}^{H-1} ( |p_{k+1} - r_{k+1}|^2 + w_act |a_k|^2 )

with r_k the reference position table (a figure-8 sampled per drone; an input).
The policy weights are bf16 values held exactly in float64.  The gradient of L
with respect to all weights and biases and the initial state is that of this
exact discrete computation, taken with torch.autograd.

Parity status: the loss is this build's reading (the paper's BPTT reward is a
different, exponential tracking reward with action penalties); parity
unpinned against the paper.  Pinned in tests/test_oracle_policy.py by central
finite differences of the loss (float64), the zero-policy hover case (loss and
closed-form offset loss), and structural properties of the MLP.
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


def rollout_loss(x0, W: dict, p_ref, params: dict, dt: float, H: int, w_act: float):
    """Returns (L, per-drone loss [M], final state [M, 20])."""
    x = torch.as_tensor(x0, dtype=F64) if not torch.is_tensor(x0) else x0
    r = torch.as_tensor(p_ref, dtype=F64)
    M = x.shape[0]
    P = ph.param_batch([params], [0] * M)
    per = torch.zeros(M, dtype=F64)
    for k in range(H):
        a = mlp(observation(x, r[k]), W)
        x = ph.step(x, a, P, dt, ph.EULER, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        per = per + ((x[:, 0:3] - r[k + 1]) ** 2).sum(-1) + w_act * (a * a).sum(-1)
    return per.sum() / M, per, x


def rollout_grad(x0, weights: dict, p_ref, params: dict, dt: float, H: int, w_act: float):
    """Loss and its gradient w.r.t. the weights (dict of float64 arrays) and the
    initial state [M, 20] (the three integrator slots get zero gradient: the
    attitude interface does not use them)."""
    W = weights_tensors(weights, requires_grad=True)
    x0t = torch.tensor(x0, dtype=F64, requires_grad=True)
    L, per, _ = rollout_loss(x0t, W, p_ref, params, dt, H, w_act)
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
