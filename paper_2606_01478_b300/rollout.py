"""Differentiable policy rollout: thin binding of sim_rollout_fwd / _bwd.

``PolicyRollout(sim, H, C, w_act, reward=None, action_repeat=1)`` owns the
rollout workspace; ``action_repeat`` = R holds each policy action for R physics
steps (H and C count policy steps);
``precision`` = "hilo" (default) or "bf16" picks the MLP's tensor-core operand
precision (sim_rollout_set_precision); ``reward`` selects the paper's tracking reward (weights as in
``TRACKING_REWARD``) instead of the squared tracking loss;
``rollout_loss(x0, w, runner, p_ref)`` is a torch.autograd.Function whose
forward and backward are the library's CUDA kernels (the upstream gradient
is read on the device, so backward does not synchronise).  ``w`` holds the
5316 policy parameters in the packed order W1[64][13] b1 W2[64][64] b2
W3[4][64] b3; the kernels use its bf16 rounding, and the gradient returned
for ``w`` is the gradient with respect to those bf16 values.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .sim import _stream_ptr, on_device


# the paper's BPTT tracking-reward weights (hyper-parameter table); action
# order roll, pitch, yaw, thrust
TRACKING_REWARD = {"w_theta": 0.1, "w_act": (0.12, 0.12, 0.0, 0.02), "w_dact": (1.4, 1.4, 0.0, 0.8)}

POLICY_ORDER = (("W1", (64, 13)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                ("W3", (4, 64)), ("b3", (4,)))


def pack_policy(weights: dict):
    """Flatten {W1, b1, W2, b2, W3, b3} (row-major) into the packed vector of
    SIM_POLICY_NPARAMS = 5316 values the rollout entry points take."""
    import numpy as np
    parts = []
    for name, shape in POLICY_ORDER:
        a = np.asarray(weights[name], dtype=np.float64)
        if a.shape != shape:
            raise ValueError(f"{name} must have shape {shape}")
        parts.append(a.ravel())
    return np.concatenate(parts)


def _p(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


class PolicyRollout:
    def __init__(self, sim, H: int, C: int, w_act: float = 1e-3, reward: dict | None = None,
                 action_repeat: int = 1, precision: str = "hilo"):
        self.sim, self.H, self.C, self.w_act = sim, int(H), int(C), float(w_act)
        self.repeat = int(action_repeat)
        if precision not in ("hilo", "bf16"):
            raise ValueError("precision must be 'hilo' or 'bf16'")
        self.precision = L.MLP_HILO if precision == "hilo" else L.MLP_BF16
        self.objective = L.Objective()
        if reward is not None:
            self.objective.kind = L.OBJ_TRACKING_REWARD
            self.objective.w_theta = float(reward["w_theta"])
            for i in range(4):
                self.objective.w_act[i] = float(reward["w_act"][i])
                self.objective.w_dact[i] = float(reward["w_dact"][i])
        self._apply_objective()
        nb = ctypes.c_size_t()
        sim._check(sim.lib.sim_rollout_workspace_bytes(sim.h, self.H, self.C, ctypes.byref(nb)))
        self.ws = torch.empty(nb.value, dtype=torch.uint8, device=sim.device)
        self.one = torch.ones(1, dtype=torch.float32, device=sim.device)

    def _apply_objective(self):
        """Objective and action repeat are settings of the handle; set them before
        every call so that runners sharing one handle do not see each other's."""
        self.sim._check(self.sim.lib.sim_rollout_set_objective(self.sim.h, ctypes.byref(self.objective)))
        self.sim._check(self.sim.lib.sim_rollout_set_action_repeat(self.sim.h, self.repeat))
        self.sim._check(self.sim.lib.sim_rollout_set_precision(self.sim.h, self.precision))

    def _check_inputs(self, x0, w_bf16, p_ref):
        self._apply_objective()
        n = self.sim.ntot
        if x0.dtype != torch.float32 or tuple(x0.shape) != (n, L.STATE_DIM) or not x0.is_contiguous():
            raise ValueError(f"x0 must be contiguous float32 [{n}, {L.STATE_DIM}]")
        if w_bf16.dtype != torch.bfloat16 or w_bf16.numel() != L.POLICY_NPARAMS:
            raise ValueError("w must hold 5316 bf16 values")
        if p_ref.dtype != torch.float32 or tuple(p_ref.shape) != (self.H + 1, n, 3) or not p_ref.is_contiguous():
            raise ValueError(f"p_ref must be contiguous float32 [{self.H + 1}, {n}, 3]")

    @on_device
    def forward(self, x0, w_bf16, p_ref, loss=None, stream=None):
        self._check_inputs(x0, w_bf16, p_ref)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=self.sim.device)
        s = self.sim
        s._check(s.lib.sim_rollout_fwd(s.h, _p(x0), _p(w_bf16), _p(p_ref), self.H, self.C, self.w_act,
                                       _p(self.ws), self.ws.numel(), _p(loss), _stream_ptr(stream)))
        return loss

    @on_device
    def backward(self, x0, w_bf16, p_ref, dL, dW=None, dx0=None, stream=None):
        self._check_inputs(x0, w_bf16, p_ref)
        dev = self.sim.device
        if dW is None:
            dW = torch.empty(L.POLICY_NPARAMS, dtype=torch.float32, device=dev)
        if dx0 is None:
            dx0 = torch.empty_like(x0)
        s = self.sim
        s._check(s.lib.sim_rollout_bwd(s.h, _p(x0), _p(w_bf16), _p(p_ref), self.H, self.C, self.w_act,
                                       _p(self.ws), self.ws.numel(), _p(dL), _p(dW), _p(dx0),
                                       _stream_ptr(stream)))
        return dW, dx0

    @on_device
    def grad(self, x0, w_bf16, p_ref, stream=None, loss=None, dW=None, dx0=None):
        """Loss, dL/dw and dL/dx0 in one call (sim_rollout_grad: one adjoint launch that
        runs the forward pass first, then the loss and dW reductions)."""
        self._check_inputs(x0, w_bf16, p_ref)
        dev = self.sim.device
        loss = torch.empty(1, dtype=torch.float32, device=dev) if loss is None else loss
        dW = torch.empty(L.POLICY_NPARAMS, dtype=torch.float32, device=dev) if dW is None else dW
        dx0 = torch.empty_like(x0) if dx0 is None else dx0
        s = self.sim
        s._check(s.lib.sim_rollout_grad(s.h, _p(x0), _p(w_bf16), _p(p_ref), self.H, self.C,
                                        self.w_act, _p(self.ws), self.ws.numel(), _p(loss),
                                        _p(self.one), _p(dW), _p(dx0), _stream_ptr(stream)))
        return loss, dW, dx0


class _RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, w, runner, p_ref):
        w_bf16 = w.detach().to(torch.bfloat16).contiguous()
        x0c = x0.detach().contiguous()
        loss = runner.forward(x0c, w_bf16, p_ref)
        ctx.runner = runner
        ctx.save_for_backward(x0c, w_bf16, p_ref)
        return loss[0]

    @staticmethod
    def backward(ctx, gL):
        x0, w_bf16, p_ref = ctx.saved_tensors
        dL = gL.detach().reshape(1).to(torch.float32).contiguous()
        dW, dx0 = ctx.runner.backward(x0, w_bf16, p_ref, dL)
        return dx0, dW, None, None


def rollout_loss(x0: torch.Tensor, w: torch.Tensor, runner: PolicyRollout, p_ref: torch.Tensor):
    """Differentiable mean tracking loss of the policy rollout (scalar tensor)."""
    return _RolloutFn.apply(x0, w, runner, p_ref)
