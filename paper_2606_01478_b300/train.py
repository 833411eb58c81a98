"""BPTT training loop on the device: rollout gradient + Adam, graph-capturable.

``PolicyTrainer(runner, w0, lr)`` keeps fp32 master weights, the Adam moments,
the device step counter and the bf16 copy the rollout reads; ``iteration()``
issues the rollout-gradient kernels and the Adam kernel on the current stream
(no host synchronisation), and ``capture()`` records one iteration into a CUDA
graph whose replays run successive iterations.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .rollout import PolicyRollout, _p
from .sim import _stream_ptr, on_device


class PolicyTrainer:
    def __init__(self, runner: PolicyRollout, w0: torch.Tensor, lr: float, betas=(0.9, 0.999),
                 eps: float = 1e-8):
        dev = runner.sim.device
        if w0.numel() != L.POLICY_NPARAMS:
            raise ValueError("w0 must hold 5316 values")
        self.runner = runner
        self.sim = runner.sim
        self.lr, self.b1, self.b2, self.eps = float(lr), float(betas[0]), float(betas[1]), float(eps)
        self.w = w0.detach().to(device=dev, dtype=torch.float32).contiguous().clone()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.wb = self.w.to(torch.bfloat16)
        self.step = torch.zeros(1, dtype=torch.int32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.dW = torch.zeros(L.POLICY_NPARAMS, dtype=torch.float32, device=dev)
        self.dx0 = None

    @on_device
    def iteration(self, x0: torch.Tensor, p_ref: torch.Tensor, stream=None):
        if self.dx0 is None or self.dx0.shape != x0.shape:
            self.dx0 = torch.empty_like(x0)
        self.runner.grad(x0, self.wb, p_ref, stream=stream, loss=self.loss, dW=self.dW, dx0=self.dx0)
        lib = self.runner.sim.lib
        r = lib.sim_adam_step(_p(self.dW), _p(self.w), _p(self.m), _p(self.v), _p(self.wb),
                              L.POLICY_NPARAMS, _p(self.step), self.lr, self.b1, self.b2, self.eps,
                              _stream_ptr(stream))
        if r != L.SIM_OK:
            raise L.SimError(r, "sim_adam_step rejected its arguments")
        return self.loss

    def capture(self, x0: torch.Tensor, p_ref: torch.Tensor) -> torch.cuda.CUDAGraph:
        dev = self.runner.sim.device
        if self.dx0 is None or self.dx0.shape != x0.shape:
            self.dx0 = torch.empty_like(x0)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.iteration(x0, p_ref, stream=s)
        torch.cuda.current_stream(dev).wait_stream(s)
        return g
