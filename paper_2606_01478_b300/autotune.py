"""Autotuner binding: sim_autotune times the candidate launch shapes inside
the library (CUDA events on the handle's own data and stream), applies the
fastest and caches it in $CRAZYFLOW_AUTOTUNE_CACHE (default
~/.cache/crazyflow_b300/autotune.jsonl) under a key naming the GPU, the
operation, the batch shape and model mix, the integrator, the control
interface, the rotor model and the run length (see include/crazyflow.h).
This module only marshals the request and the result.
"""
from __future__ import annotations

import ctypes

from . import _lib as L
from .sim import _stream_ptr, on_device

DEFAULT_TPB = (32, 64, 128, 256)
DEFAULT_K = (1, 5, 10, 25, 50, 100, 200)


def _request(op: int, tpbs, Ks, reps: int, use_cache: bool) -> L.TuneRequest:
    if len(tpbs) > L.TUNE_MAX or len(Ks) > L.TUNE_MAX:
        raise ValueError(f"at most {L.TUNE_MAX} candidates per list")
    r = L.TuneRequest()
    r.op, r.reps, r.use_cache = op, int(reps), int(bool(use_cache))
    r.n_tpb = len(tpbs)
    for i, t in enumerate(tpbs):
        r.tpb[i] = int(t)
    r.n_K = len(Ks)
    for i, k in enumerate(Ks):
        r.K[i] = int(k)
    return r


def _result(res: L.TuneResult, tpbs, Ks) -> dict:
    table = [{"tpb": int(t), "K": int(k), "ms": float(res.trial_ms[i * L.TUNE_MAX + j])}
             for i, t in enumerate(tpbs) for j, k in enumerate(Ks)
             if res.trial_ms[i * L.TUNE_MAX + j] > 0]
    return {"tpb": res.tpb, "K": res.K, "ms": res.ms, "from_cache": bool(res.from_cache),
            "key": res.key.decode(), "table": table}


class _Runner:
    def __init__(self, sim):
        self.sim = sim

    @on_device
    def call(self, req):
        res = L.TuneResult()
        self.sim._check(self.sim.lib.sim_autotune(self.sim.h, ctypes.byref(req), ctypes.byref(res),
                                                  _stream_ptr(None)))
        return res


def tune_step(sim, n_steps: int, tpbs=DEFAULT_TPB, Ks=DEFAULT_K, reps: int = 3,
              use_cache: bool = True) -> dict:
    """Pick (threads per block, steps per launch) minimising the time of
    `n_steps` steps on `sim` (parameters, state and commands set).  The state
    and the command schedule are the same afterwards; the block size is
    applied.  Returns {tpb, K, ms, from_cache, key, table}."""
    req = _request(L.TUNE_STEP, tpbs, Ks, reps, use_cache)
    req.n_steps = int(n_steps)
    kept = [k for k in Ks if k <= n_steps] or [min(int(n_steps), 100000)]
    return _result(_Runner(sim).call(req), tpbs, kept)


def tune_sample(sim, S: int, H: int, seed, sigma: float, goals, obstacles, w_obs: float, cost,
                nominal=None, tpbs=(64, 128, 256), reps: int = 1, use_cache: bool = True) -> dict:
    """Pick the sampling launch's threads per block for this sim_sample_rollouts
    call (its arguments as for Sim.sample_rollouts; `cost` is written)."""
    import numpy as np
    req = _request(L.TUNE_SAMPLE, tpbs, (1,), reps, use_cache)
    obs = np.ascontiguousarray(np.asarray(obstacles, dtype=np.float32).reshape(-1, 4))
    req.S, req.H, req.sigma, req.w_obs, req.n_obs = int(S), int(H), float(sigma), float(w_obs), obs.shape[0]
    req.seed = seed.data_ptr()
    req.goals = goals.data_ptr()
    req.cost = cost.data_ptr()
    req.nominal = None if nominal is None else nominal.data_ptr()
    req.obstacles = obs.ctypes.data
    return _result(_Runner(sim).call(req), tpbs, (1,))


def key_of(sim, op: int = L.TUNE_STEP, n_steps: int = 1, S: int = 1, H: int = 1, n_obs: int = 0) -> str:
    """The cache key sim_autotune uses (no device work)."""
    req = _request(op, (), (), 1, True)
    req.n_steps, req.S, req.H, req.n_obs = int(n_steps), int(S), int(H), int(n_obs)
    buf = ctypes.create_string_buffer(512)
    sim._check(sim.lib.sim_autotune_key(sim.h, ctypes.byref(req), buf, 512))
    return buf.value.decode()
