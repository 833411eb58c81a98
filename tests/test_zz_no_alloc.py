"""The workspace-free rollout gradient (sim_rollout_grad_noalloc).

Callers that cannot allocate device memory when they need a gradient -- a
control loop with a hard deadline, or a plugin whose host framework owns all
device allocations -- use this entry point; its scratch is a fixed array
inside the library.  This test calls it through the C-ABI and checks it
against the workspace entry point (sim_rollout_grad) on two calls in a row,
with different inputs, so stale scratch contents from the first call would
show in the second.  Both entry points run the same deterministic kernels on
the same inputs, so their results must be bit-identical.  A third check reads
the device's free memory around repeated calls: a call must not allocate.
It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import policy as po
from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
from paper_2606_01478_b300 import _lib as L
from paper_2606_01478_b300.rollout import PolicyRollout

pytestmark = pytest.mark.gpu

def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs(seed, M, H, C):
    rw = W.policy_bptt(seed=seed, M=M, H=H, C=C)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device="cuda")
    w = torch.tensor(po.pack(rw.weights), dtype=torch.bfloat16, device="cuda")
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device="cuda").contiguous()
    return rw, x0, w, p_ref


def _noalloc(sim, x0, w, p_ref, H, C, w_act):
    dev = x0.device
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    dW = torch.empty(L.POLICY_NPARAMS, dtype=torch.float32, device=dev)
    dx0 = torch.empty_like(x0)
    r = sim.lib.sim_rollout_grad_noalloc(sim.h, _p(x0), _p(w), _p(p_ref), H, C, w_act, _p(loss),
                                         _p(dW), _p(dx0),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == L.SIM_OK, sim.lib.sim_last_error(sim.h).decode()
    return loss, dW, dx0


def test_noalloc_matches_workspace_entry_point_twice():
    M, H, C = 512, 100, 10
    sim = Sim(M, 1, FIRST_PRINCIPLES, EULER, 1 / 500)
    sim.set_params(W.crazyflie_params())
    runner = PolicyRollout(sim, H, C, 1e-3)
    for seed in (41, 42):  # two calls in a row, different inputs
        rw, x0, w, p_ref = _inputs(seed, M, H, C)
        ref = runner.grad(x0, w, p_ref)
        got = _noalloc(sim, x0, w, p_ref, H, C, rw.w_act)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.isfinite(a).all()
            assert torch.equal(a, b)


def test_noalloc_call_allocates_no_device_memory():
    M, H, C = 256, 50, 10
    sim = Sim(M, 1, FIRST_PRINCIPLES, EULER, 1 / 500)
    sim.set_params(W.crazyflie_params())
    rw, x0, w, p_ref = _inputs(44, M, H, C)
    outs = _noalloc(sim, x0, w, p_ref, H, C, rw.w_act)  # first call: looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(5):
        r = sim.lib.sim_rollout_grad_noalloc(sim.h, p(x0), p(w), p(p_ref), H, C, rw.w_act, p(outs[0]),
                                             p(outs[1]), p(outs[2]), st)
        assert r == L.SIM_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the driver's own bookkeeping can move free memory by a page or two
    assert abs(free1 - free0) <= 4 << 20, (free0, free1)


def test_noalloc_rejects_batches_beyond_its_scratch():
    cap = ctypes.c_size_t()
    lib = L.load()
    assert lib.sim_rollout_noalloc_max_bytes(ctypes.byref(cap)) == L.SIM_OK
    M, H, C = 8192, 250, 25  # needs ~170 MB of scratch
    sim = Sim(M, 1, FIRST_PRINCIPLES, EULER, 1 / 500)
    sim.set_params(W.crazyflie_params())
    need = ctypes.c_size_t()
    assert lib.sim_rollout_workspace_bytes(sim.h, H, C, ctypes.byref(need)) == L.SIM_OK
    assert need.value > cap.value
    x0 = torch.zeros(M, 20, device="cuda")
    w = torch.zeros(L.POLICY_NPARAMS, dtype=torch.bfloat16, device="cuda")
    p_ref = torch.zeros(H + 1, M, 3, device="cuda")
    out = torch.zeros(1, device="cuda")
    dW = torch.zeros(L.POLICY_NPARAMS, device="cuda")
    dx0 = torch.zeros_like(x0)
    r = lib.sim_rollout_grad_noalloc(sim.h, _p(x0), _p(w), _p(p_ref), H, C, 1e-3, _p(out), _p(dW),
                                     _p(dx0), None)
    assert r == L.SIM_EINVAL
    assert b"built-in scratch" in lib.sim_last_error(sim.h)
