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


def test_autotuner_restores_state_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("CRAZYFLOW_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    wl = W.attitude_swarm_rk4(M=4096, steps=100, K=100)
    sim = make_sim(wl)
    before = sim.get_state().clone()
    best = autotune.tune_step(sim, 100, tag="test", tpbs=(32, 128), Ks=(10, 50, 100), reps=1)
    assert best["tpb"] in (32, 128) and best["K"] in (10, 50, 100)
    assert len(best["table"]) == 6 and all(r["ms"] > 0 for r in best["table"])
    assert torch.equal(sim.get_state(), before)
    assert sim.steps_taken == 0
    # the tuned run gives the same states as the default configuration
    sim.run(100, best["K"])
    ref = make_sim(wl)
    ref.run(100, 100)
    assert torch.equal(sim.get_state(), ref.get_state())
    assert os.path.exists(tmp_path / "tune.json")
    again = autotune.tune_step(sim, 100, tag="test")
    assert again["tpb"] == best["tpb"] and again["K"] == best["K"]
