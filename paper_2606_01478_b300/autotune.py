"""Autotuner for the fused step: threads per block and steps per launch.

Each candidate (tpb, K) is timed with CUDA events on the handle's own data
(state saved and restored around the trials, command schedule re-armed), and
the fastest is cached in a JSON file keyed by GPU name, batch shape, model mix,
integrator and control interface.  The cache lives in
$CRAZYFLOW_AUTOTUNE_CACHE or ~/.cache/crazyflow_b300/autotune.json.
"""
from __future__ import annotations

import json
import os

import torch

DEFAULT_TPB = (32, 64, 128, 256)
DEFAULT_K = (1, 5, 10, 25, 50, 100, 200)


def cache_path() -> str:
    return os.environ.get("CRAZYFLOW_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "crazyflow_b300",
                                       "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def key_of(sim, n_steps: int, tag: str = "") -> str:
    name = torch.cuda.get_device_name(sim.device)
    return f"{name}|step|{tag}|ntot={sim.ntot}|steps={n_steps}"


def tune_step(sim, n_steps: int, tag: str = "", tpbs=DEFAULT_TPB, Ks=DEFAULT_K, reps: int = 3,
              use_cache: bool = True) -> dict:
    """Pick (tpb, K) minimising the time of `n_steps` steps on `sim` (which must
    have parameters, state and commands set).  The state and the command
    schedule are restored afterwards; the chosen block size is applied."""
    key = key_of(sim, n_steps, tag)
    db = _load() if use_cache else {}
    if key in db:
        best = db[key]
        sim.set_block_size(best["tpb"])
        return best
    saved = sim.get_state().clone()
    cmd, hold = sim._cmd_src, sim._hold
    table = []
    stream = torch.cuda.current_stream(sim.device)
    for tpb in tpbs:
        sim.set_block_size(tpb)
        for K in Ks:
            if K > n_steps:
                continue
            times = []
            for r in range(reps + 1):
                sim.set_state(saved)
                sim.set_commands(cmd, hold)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                torch.cuda._sleep(200_000)
                e0.record(stream)
                sim.run(n_steps, K)
                e1.record(stream)
                e1.synchronize()
                if r:
                    times.append(e0.elapsed_time(e1))
            table.append({"tpb": tpb, "K": K, "ms": min(times)})
    best = min(table, key=lambda r: r["ms"])
    sim.set_state(saved)
    sim.set_commands(cmd, hold)
    sim.set_block_size(best["tpb"])
    result = {"tpb": best["tpb"], "K": best["K"], "ms": best["ms"], "table": table}
    if use_cache:
        db[key] = result
        _store(db)
    return result
