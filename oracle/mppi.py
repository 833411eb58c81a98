"""FP64 oracle of one MPPI / iCEM control iteration on top of the sampled rollouts.

TEST INFRASTRUCTURE ONLY (see the package header).

The paper's sampling controller (Materials and Methods, Model Predictive Path
Integral) runs several independent controllers in parallel, keeps the top 1 %
of each controller's trajectories as elites (iCEM), uses temporally correlated
noise, warm-starts from the previous mean, averages the elites with
exponential (MPPI) weights and applies the best controller's sequence.  For
every drone d, with n_ctrl controllers of S_c = S / n_ctrl samples each:

    sample s belongs to controller c = s // S_c; its actions are
        clip(mean[d, c, k] + sigma eps_{s,k}, -1, 1),  eps AR(1) with rho
        (Philox noise of sample id d * S + s, see oracle.sampling)
    elites E_c: the n_e smallest costs of the controller (ties: lower sample
        index first); the paper's "top 1 %" is n_e = n_elites(S_c, 0.01)
        = ceil(S_c / 100), e.g. 1000 of the 100 000 samples each of its five
        controllers draw (500k trajectories in all)
    w_e = exp(-(J_e - J_min,c) / lam),  mean'[d, c] = sum_e w_e a_e / sum_e w_e
    c* = argmin_c J_min,c (ties: lower c);  plan[d] = mean'[d, c*]
    warm start: mean[d, c, k] <- mean'[d, c, k + 1] (last step repeated)

Parity status: the iCEM/MPPI structure follows the paper's description; the
noise correlation model (AR(1)) and the parameter values are the reading
adopted here (the paper defers them to its supplementary code).  Pinned in
tests/test_oracle_mppi.py by: a single elite reproducing the best sample's
sequence exactly, finite-temperature weights on hand-picked costs (two and
three elites whose cost gaps are lam ln 3, lam ln 2 and lam ln 4, so the plan
must equal (3 a1 + a2) / 4 and (4 a1 + 2 a2 + a3) / 7), the infinite-
temperature limit (plain elite mean) with brute-force elite sets beyond 32
elites, the elite counts of the paper's sizes, the warm start shift, AR(1)
noise statistics, and cost decrease over iterations.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import sampling as sa


def n_elites(S_c: int, elite_frac) -> int:
    """The top fraction of a controller's S_c samples: ceil(elite_frac S_c),
    at least one.  The fraction is taken as the decimal it is written as (0.01
    is exactly one hundredth), so the count is exact: 1 % of 100 000 is 1000,
    1 % of 150 is 2."""
    f = elite_frac if isinstance(elite_frac, Fraction) else Fraction(str(elite_frac))
    if not 0 < f <= 1:
        raise ValueError("elite_frac must lie in (0, 1]")
    return max(1, math.ceil(f * S_c))


def select_elites(costs_c: np.ndarray, n_e: int) -> np.ndarray:
    """Indices of the n_e smallest costs, ties broken by lower index (stable)."""
    return np.argsort(costs_c, kind="stable")[:n_e]


def update(costs, mean, seed: int, S: int, H: int, n_ctrl: int, sigma: float, rho: float,
           n_e: int, lam: float, drones):
    """MPPI update of the listed drones with n_e elites per controller.  costs
    [n, S] (rows for `drones`), mean [n, n_ctrl, H, 4].  Returns (mean_next
    (warm-started) [n, n_ctrl, H, 4], plan [n, H, 4], best_cost [n])."""
    drones = np.asarray(drones, dtype=np.int64)
    costs = np.asarray(costs, dtype=np.float64)
    mean = np.asarray(mean, dtype=np.float64)
    n = len(drones)
    S_c = S // n_ctrl
    n_e = int(n_e)
    if not 1 <= n_e <= S_c:
        raise ValueError("need 1 <= n_e <= S / n_ctrl")
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
