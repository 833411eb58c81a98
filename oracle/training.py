"""FP64 oracle of the BPTT training loop: rollout gradient + Adam.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper trains its tracking policy by BPTT with all environment rollouts
and optimisation steps fused into one graph (Materials and Methods,
Backpropagation Through Time, with its hyper-parameter table: learning rate
4.6e-2, 16 environments, 40 steps per rollout).  One iteration here:

    g = dL/dw(bf16(w))                      (oracle.policy.rollout_grad)
    Adam (Kingma & Ba, ICLR 2015), t = 1, 2, ...:
      m <- b1 m + (1 - b1) g;   v <- b2 v + (1 - b2) g^2
      w <- w - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
    the rollout of the next iteration uses bf16(w) (round to nearest even)

Parity status: Adam is the published definition; pinned by its closed forms
(first step and constant gradients move every weight by lr g / (|g| + eps)) and
by convergence on a quadratic.  The loop is pinned through its parts.
"""
from __future__ import annotations

import numpy as np

from . import policy as po


def adam(w, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step at step number t (1-based); returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def round_bf16(x):
    """Nearest bfloat16 value (ties to even) of float32(x), as float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def train(x0, p_ref, params: dict, w0_flat, iters: int, lr: float, dt: float, H: int, w_act: float,
          b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8, reward: dict | None = None,
          repeat: int = 1):
    """`iters` iterations from master weights w0_flat (5316, float64).  Returns
    (losses [iters], final master weights)."""
    w = np.asarray(w0_flat, dtype=np.float64).copy()
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    losses = []
    for t in range(1, iters + 1):
        wb = po.unpack(round_bf16(w))
        L, _, dW, _ = po.rollout_grad(x0, wb, p_ref, params, dt, H, w_act, reward, repeat)
        losses.append(L)
        w, m, v = adam(w, po.pack(dW), m, v, t, lr, b1, b2, eps)
    return np.array(losses), w
