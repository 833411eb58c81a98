"""FP64 oracle of one MPPI / iCEM control iteration on top of the sampled rollouts.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's sampling controller (Materials and Methods, Model Predictive Path
Integral) runs several independent controllers in parallel, keeps the best
fraction of each controller's trajectories (iCEM), uses temporally correlated
noise, warm-starts from the previous mean, averages the elites with
exponential (MPPI) weights and applies the best controller's sequence.  For
every drone d, with n_ctrl controllers of S_c = S / n_ctrl samples each:

    sample s belongs to controller c = s // S_c; its actions are
        clip(mean[d, c, k] + sigma eps_{s,k}, -1, 1),  eps AR(1) with rho
        (Philox noise of sample id d * S + s, see oracle.sampling)
    elites E_c: the n_e = clamp(ceil(elite_frac S_c - 1e-4), 1, 32) smallest costs
        (ties: lower sample index first)
    w_e = exp(-(J_e - J_min,c) / lam),  mean'[d, c] = sum_e w_e a_e / sum_e w_e
    c* = argmin_c J_min,c (ties: lower c);  plan[d] = mean'[d, c*]
    warm start: mean[d, c, k] <- mean'[d, c, k + 1] (last step repeated)

Parity status: the iCEM/MPPI structure follows the paper's description; the
noise correlation model (AR(1)), the elite cap and the parameter values are the
reading adopted here (the paper defers them to its supplementary code).  Pinned in
tests/test_oracle_mppi.py by: a single elite reproducing the best sample's
sequence exactly, the infinite-temperature limit (plain elite mean), the warm
start shift, AR(1) noise statistics, and cost decrease over iterations.
"""
from __future__ import annotations

import math

import numpy as np

from . import sampling as sa

MAX_ELITES = 32


def n_elites(S_c: int, elite_frac: float) -> int:
    """clamp(ceil(elite_frac S_c - 1e-4), 1, 32): the 1e-4 guard makes a
    fraction given in float32 (0.1 -> 0.100000001) count as intended."""
    return int(min(MAX_ELITES, max(1, math.ceil(elite_frac * S_c - 1e-4))))


def select_elites(costs_c: np.ndarray, n_e: int) -> np.ndarray:
    """Indices of the n_e smallest costs, ties broken by lower index (stable)."""
    return np.argsort(costs_c, kind="stable")[:n_e]


def update(costs, mean, seed: int, S: int, H: int, n_ctrl: int, sigma: float, rho: float,
           elite_frac: float, lam: float, drones):
    """MPPI update of the listed drones.  costs [n, S] (rows for `drones`),
    mean [n, n_ctrl, H, 4].  Returns (mean_next (warm-started) [n, n_ctrl, H, 4],
    plan [n, H, 4], best_cost [n])."""
    drones = np.asarray(drones, dtype=np.int64)
    costs = np.asarray(costs, dtype=np.float64)
    mean = np.asarray(mean, dtype=np.float64)
    n = len(drones)
    S_c = S // n_ctrl
    n_e = n_elites(S_c, elite_frac)
    new_mean = np.zeros_like(mean)
    plan = np.zeros((n, H, 4))
    best = np.zeros(n)
    for i, d in enumerate(drones):
        jmin = np.zeros(n_ctrl)
        for c in range(n_ctrl):
            cc = costs[i, c * S_c:(c + 1) * S_c]
            el = select_elites(cc, n_e)
            J = cc[el]
            jmin[c] = J[0]
            w = np.exp(-(J - J[0]) / lam)
            ids = np.uint64(d) * np.uint64(S) + (np.uint64(c * S_c) + el.astype(np.uint64))
            acts = sa.sampled_actions(seed, ids, H, np.broadcast_to(mean[i, c], (n_e, H, 4)),
                                      sigma, rho)
            new_mean[i, c] = (w[:, None, None] * acts).sum(0) / w.sum()
        cbest = int(np.argmin(jmin))
        plan[i] = new_mean[i, cbest]
        best[i] = jmin[cbest]
    shifted = np.concatenate([new_mean[:, :, 1:], new_mean[:, :, -1:]], axis=2)
    return shifted, plan, best


def sample_costs(x0, goals, obstacles, params, S: int, H: int, n_ctrl: int, dt: float,
                 sigma: float, rho: float, seed: int, w_obs: float, mean, world_of_drone, drones,
                 integrator=None):
    """Costs [n, S] of every sample of the listed drones under the MPPI
    sampling (per-controller means, AR(1) noise)."""
    from . import physics as ph
    drones = np.asarray(drones, dtype=np.int64)
    mean = np.asarray(mean, dtype=np.float64)
    S_c = S // n_ctrl
    rows_d = np.repeat(drones, S)
    rows_i = np.repeat(np.arange(len(drones)), S)
    s = np.tile(np.arange(S), len(drones))
    ids = rows_d.astype(np.uint64) * np.uint64(S) + s.astype(np.uint64)
    nom = mean[rows_i, s // S_c]
    acts = sa.sampled_actions(seed, ids, H, nom, sigma, rho)
    world = np.asarray(world_of_drone)[rows_d]
    c = sa.cost_of_actions(np.asarray(x0)[rows_d], np.asarray(goals)[world], obstacles, params, acts,
                           dt, w_obs, ph.RK4 if integrator is None else integrator)
    return c.reshape(len(drones), S)
