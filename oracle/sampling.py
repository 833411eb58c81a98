"""FP64 oracle of the batched sampling rollouts (MPPI-style rollouts + cost).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's MPPI/iCEM controller uses the full simulation as its forward
model and evaluates 500k sampled command sequences per control step (Results,
Control in Cluttered Environments; Materials and Methods, Model Predictive Path
Integral).  For every drone d and sample s this module computes

    xi_{s,k} = 4 standard normals from Philox4x32-10 (counter-based RNG of
               Salmon et al., SC'11) with counter (id_lo, id_hi, k, 0) and key
               (seed_lo, seed_hi), id = d * S + s, by Box-Muller on the top 23
               bits of each word
    a_{s,k}  = clip(nominal_k + sigma xi_{s,k}, -1, 1)        (attitude action)
    x_{k+1}  = RK4 step of the first-principles model from x_0 = the drone's state
    cost_s   = sum_{k=1..H} ( |p_k - g_w| + w_obs sum_o max(0, r_o - |p_k - c_o|) )

with g_w the goal of the drone's world and (c_o, r_o) spherical obstacles.

Parity status: Philox is pinned bit-exactly by its published known-answer
vectors (tests/golden/philox4x32_10_kat.txt); the Box-Muller map by exact
uniform values and moments; the cost (the reading adopted here: the paper prints
no cost) by the closed form at hover with zero noise and by a scalar
brute-force evaluation on a tiny instance.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import physics as ph

F64 = torch.float64
_M0, _M1 = 0xD2511F53, 0xCD9E8D57  # Philox multipliers
_W0, _W1 = 0x9E3779B9, 0xBB67AE85  # Weyl key increments
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ctr [..., 4], key [..., 2] (integers < 2^32);
    returns uint32 [..., 4].  One round: (c0, c1, c2, c3) ->
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key is
    bumped by the Weyl constants between rounds."""
    c = [np.asarray(ctr[..., j], dtype=np.uint64) & _MASK for j in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & _MASK
    for _ in range(10):
        p0 = np.uint64(_M0) * c[0]
        p1 = np.uint64(_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(_W0)) & _MASK
        k1 = (k1 + np.uint64(_W1)) & _MASK
    return np.stack(c, axis=-1).astype(np.uint32)


def uniform24(words: np.ndarray) -> np.ndarray:
    """((w >> 9) + 0.5) * 2^-23 = (2k + 1) / 2^24: uniforms in (0, 1) with 24
    significant bits, exact in fp32 and fp64."""
    return ((words.astype(np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def box_muller(u1: np.ndarray, u2: np.ndarray):
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)


def normals(seed: int, sample_ids: np.ndarray, step: int) -> np.ndarray:
    """[n, 4] standard normals for the given 64-bit sample ids at one step."""
    ids = np.asarray(sample_ids, dtype=np.uint64)
    ctr = np.stack([ids & _MASK, ids >> np.uint64(32), np.full_like(ids, step),
                    np.zeros_like(ids)], axis=-1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, np.broadcast_to(key, ctr.shape[:-1] + (2,)))
    u = uniform24(w)
    z0, z1 = box_muller(u[:, 0], u[:, 1])
    z2, z3 = box_muller(u[:, 2], u[:, 3])
    return np.stack([z0, z1, z2, z3], axis=-1)


def cost_of_actions(x0_rows, goal_rows, obstacles, params: dict, actions, dt: float, w_obs: float,
                    integrator: int = ph.RK4):
    """Cost of fixed action sequences: x0_rows [n, 20], goal_rows [n, 3],
    actions [n, H, 4] (already clipped)."""
    x = torch.tensor(np.asarray(x0_rows), dtype=F64)
    g = torch.tensor(np.asarray(goal_rows), dtype=F64)
    obs = torch.tensor(np.asarray(obstacles), dtype=F64).reshape(-1, 4)
    a_all = torch.tensor(np.asarray(actions), dtype=F64)
    n = x.shape[0]
    P = ph.param_batch([params], [0] * n)
    cost = torch.zeros(n, dtype=F64)
    for k in range(a_all.shape[1]):
        x = ph.step(x, a_all[:, k], P, dt, integrator, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        p = x[:, 0:3]
        cost = cost + torch.linalg.vector_norm(p - g, dim=-1)
        d = torch.linalg.vector_norm(p[:, None, :] - obs[None, :, 0:3], dim=-1)
        cost = cost + w_obs * torch.clamp(obs[None, :, 3] - d, min=0.0).sum(-1)
    return cost.numpy()


def sampled_actions(seed: int, ids, H: int, nominal_rows, sigma: float, rho: float = 0.0):
    """Actions [n, H, 4] of the samples with the given ids: clip(nominal + sigma
    eps, -1, 1) with eps_0 = xi_0, eps_k = rho eps_{k-1} + sqrt(1 - rho^2) xi_k
    (AR(1) temporal correlation; rho = 0 is white noise).  nominal_rows
    [n, H, 4] or None."""
    ids = np.asarray(ids, dtype=np.uint64)
    n = len(ids)
    out = np.zeros((n, H, 4))
    eps = np.zeros((n, 4))
    c = np.sqrt(1.0 - rho * rho)
    for k in range(H):
        xi = normals(seed, ids, k)
        eps = xi if k == 0 else rho * eps + c * xi
        a = sigma * eps
        if nominal_rows is not None:
            a = a + np.asarray(nominal_rows)[:, k]
        out[:, k] = np.clip(a, -1.0, 1.0)
    return out


def rollout_cost(x0, goals, obstacles, params: dict, S: int, H: int, dt: float, sigma: float,
                 seed: int, w_obs: float, drones, samples, world_of_drone, nominal=None,
                 integrator: int = ph.RK4):
    """Costs of the (drone, sample) pairs listed in `drones`, `samples` (equal
    length).  x0 [Ntot, 20], goals [M, 3], obstacles [O, 4], world_of_drone
    [Ntot]; nominal [M, H, 4] or None (zeros); integrator ph.RK4 or ph.EULER."""
    drones = np.asarray(drones, dtype=np.int64)
    samples = np.asarray(samples, dtype=np.int64)
    ids = drones.astype(np.uint64) * np.uint64(S) + samples.astype(np.uint64)
    world = np.asarray(world_of_drone)[drones]
    nom = None if nominal is None else np.asarray(nominal)[world]
    acts = sampled_actions(seed, ids, H, nom, sigma)
    return cost_of_actions(np.asarray(x0)[drones], np.asarray(goals)[world], obstacles, params,
                           acts, dt, w_obs, integrator)
