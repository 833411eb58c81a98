"""CUDA-graph capture of fused rollouts and the block-size / steps-per-launch
autotuner (GPU)."""
import os

import numpy as np
import pytest
import torch

import workloads as W
from paper_2606_01478_b300 import Sim
from paper_2606_01478_b300 import autotune

from gpu_util import make_sim

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager():
    wl = W.attitude_swarm_rk4(M=2000, steps=300, K=100)
    eager = make_sim(wl)
    eager.run(300, 100)
    ref = eager.get_state().cpu()
    sim = make_sim(wl)
    g = sim.capture_run(300, 100)
    assert sim.steps_taken == 0  # capture does not advance the schedule
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sim.get_state().cpu(), ref)
    # a second replay from the same initial state gives the same result
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sim.get_state().cpu(), ref)


def test_graph_replay_uneven_mixed():
    bw = W.batched_workload(21, [3, 130, 64, 1000, 7], [1, 0, 1, 0, 1], steps=100, K=25, hold=20)
    def build():
        s = Sim.batched(bw.n_per_world, bw.model_of_world, bw.integrator, bw.dt,
                        max_cmd_blocks=bw.cmd.shape[0])
        s.set_params(bw.params, np.arange(bw.M))
        s.set_state(torch.tensor(bw.x0, dtype=torch.float32, device="cuda"))
        s.set_commands(torch.tensor(bw.cmd, dtype=torch.float32, device="cuda"), bw.hold)
        return s
    a = build()
    a.run(100, 25)
    b = build()
    g = b.capture_run(100, 25)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(a.get_state(), b.get_state())


def test_fused_uneven_launches_repeat_with_any_grid():
    """Fused launches of an uneven batch take their tiles from a device counter that each
    grid's last warp resets: chained launches at several block sizes and a graph replayed
    several times all give the eager state, bit for bit."""
    bw = W.batched_workload(22, [3, 130, 64, 1000, 7, 45, 300], [1, 0, 1, 0, 1, 0, 1], steps=100,
                            K=25, hold=20)
    x0 = torch.tensor(bw.x0, dtype=torch.float32, device="cuda")
    cmd = torch.tensor(bw.cmd, dtype=torch.float32, device="cuda")

    def build(tpb=None):
        s = Sim.batched(bw.n_per_world, bw.model_of_world, bw.integrator, bw.dt,
                        max_cmd_blocks=bw.cmd.shape[0])
        s.set_params(bw.params, np.arange(bw.M))
        if tpb:
            s.set_block_size(tpb)
        s.set_state(x0)
        s.set_commands(cmd, bw.hold)
        return s
    ref = build()
    ref.run(100, 25)
    expect = ref.get_state().clone()
    for tpb in (32, 96, 256):
        s = build(tpb)
        s.run(100, 25)
        assert torch.equal(s.get_state(), expect), tpb
        assert s.status() == 0
    b = build()
    g = b.capture_run(100, 25)
    for _ in range(3):
        b.set_state(x0)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.get_state(), expect)


def test_autotuner_restores_state_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("CRAZYFLOW_AUTOTUNE_CACHE", str(tmp_path / "tune.jsonl"))
    wl = W.attitude_swarm_rk4(M=4096, steps=100, K=100)
    sim = make_sim(wl)
    before = sim.get_state().clone()
    best = autotune.tune_step(sim, 100, tpbs=(32, 128), Ks=(10, 50, 100), reps=1)
    assert best["tpb"] in (32, 128) and best["K"] in (10, 50, 100)
    assert len(best["table"]) == 6 and all(r["ms"] > 0 for r in best["table"])
    assert torch.equal(sim.get_state(), before)
    assert sim.steps_taken == 0
    # the tuned run gives the same states as the default configuration
    sim.run(100, best["K"])
    ref = make_sim(wl)
    ref.run(100, 100)
    assert torch.equal(sim.get_state(), ref.get_state())
    assert os.path.exists(tmp_path / "tune.jsonl")
    again = autotune.tune_step(sim, 100)
    assert again["from_cache"] and again["tpb"] == best["tpb"] and again["K"] == best["K"]


def _req(op, tpbs, Ks, reps, use_cache, n_steps):
    from paper_2606_01478_b300 import _lib as L
    r = L.TuneRequest()
    r.op, r.reps, r.use_cache, r.n_steps = op, reps, use_cache, n_steps
    r.n_tpb, r.n_K = len(tpbs), len(Ks)
    for i, t in enumerate(tpbs):
        r.tpb[i] = t
    for i, k in enumerate(Ks):
        r.K[i] = k
    return r


def test_sim_autotune_through_the_c_abi(tmp_path, monkeypatch):
    """sim_autotune called directly: the candidates are timed, the best is
    applied and appended to the cache file as one JSON line; a cached call
    returns it without timing; a bad request is refused."""
    import ctypes
    import json
    from paper_2606_01478_b300 import _lib as L
    path = tmp_path / "c_abi.jsonl"
    monkeypatch.setenv("CRAZYFLOW_AUTOTUNE_CACHE", str(path))
    wl = W.attitude_swarm_rk4(M=3000, steps=60, K=20)
    sim = make_sim(wl)
    lib = sim.lib
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    res = L.TuneResult()
    req = _req(L.TUNE_STEP, (64, 256), (20, 60), 1, 1, 60)
    assert lib.sim_autotune(sim.h, ctypes.byref(req), ctypes.byref(res), st) == L.SIM_OK
    assert res.n_trials == 4 and not res.from_cache and res.cache_written
    assert res.tpb in (64, 256) and res.K in (20, 60) and res.ms > 0
    lines = [json.loads(ln) for ln in path.read_text().splitlines()]
    assert lines == [{"key": res.key.decode(), "tpb": res.tpb, "K": res.K, "ms": pytest.approx(res.ms, rel=1e-5)}]
    again = L.TuneResult()
    assert lib.sim_autotune(sim.h, ctypes.byref(req), ctypes.byref(again), st) == L.SIM_OK
    assert again.from_cache and again.n_trials == 0 and (again.tpb, again.K) == (res.tpb, res.K)
    bad = _req(L.TUNE_STEP, (48,), (20,), 1, 0, 60)
    assert lib.sim_autotune(sim.h, ctypes.byref(bad), ctypes.byref(again), st) == L.SIM_EINVAL


def test_handles_differing_only_by_integrator_get_separate_entries(tmp_path, monkeypatch):
    import json
    from paper_2606_01478_b300 import EULER, RK4
    path = tmp_path / "integ.jsonl"
    monkeypatch.setenv("CRAZYFLOW_AUTOTUNE_CACHE", str(path))
    keys = []
    for integ in (EULER, RK4):
        wl = W.attitude_swarm_rk4(M=2048, steps=40, K=20)
        wl.integrator = integ
        sim = make_sim(wl)
        r = autotune.tune_step(sim, 40, tpbs=(64, 128), Ks=(20, 40), reps=1)
        assert not r["from_cache"]
        keys.append(r["key"])
    assert keys[0] != keys[1]
    assert [json.loads(ln)["key"] for ln in path.read_text().splitlines()] == keys


def test_sampling_block_size_from_the_autotuner(tmp_path, monkeypatch):
    monkeypatch.setenv("CRAZYFLOW_AUTOTUNE_CACHE", str(tmp_path / "sample.jsonl"))
    from paper_2606_01478_b300 import RK4
    wl = W.uneven_sampling_rk4(M=6)
    sim = Sim.batched(wl.n_per_world, np.zeros(wl.M, np.int32), RK4, wl.dt)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device="cuda"))
    goals = torch.tensor(wl.goals, dtype=torch.float32, device="cuda")
    seed = torch.tensor([5], dtype=torch.int64, device="cuda")
    cost = torch.empty(len(wl.x0), 32, device="cuda")
    r = autotune.tune_sample(sim, 32, 10, seed, 0.2, goals, wl.obstacles, 1000.0, cost, tpbs=(64, 256))
    assert r["tpb"] in (64, 256) and len(r["table"]) == 2 and "op=sample" in r["key"]
    ref = sim.sample_rollouts(32, 10, seed, 0.2, goals, wl.obstacles, 1000.0).clone()
    sim.set_block_size(64 if r["tpb"] == 256 else 256)
    assert torch.equal(sim.sample_rollouts(32, 10, seed, 0.2, goals, wl.obstacles, 1000.0), ref)
