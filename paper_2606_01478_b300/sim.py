"""Thin Python binding of the C-ABI: argument marshalling only.

PyTorch supplies device memory (one uint8 workspace tensor per handle) and the
stream; every step of the simulation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L


def _stream_ptr(stream, device=None) -> ctypes.c_void_p:
    """The CUDA stream handle for a call on `device` (default: the current
    device): the given stream, which must belong to that device, or the
    device's current stream."""
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    device = torch.device(device)
    if stream is None:
        stream = torch.cuda.current_stream(device)
    _check_same_device(stream.device, device, "stream")
    return ctypes.c_void_p(stream.cuda_stream)


def _check_same_device(got, want, what: str) -> None:
    """Refuse a stream or tensor on another GPU than the one the call runs on:
    the library launches on the current device, and a kernel given another
    device's memory would fault."""
    got, want = torch.device(got), torch.device(want)
    if got.type != want.type:
        raise ValueError(f"{what} is on {got}, the call runs on {want}")
    gi = got.index if got.index is not None else torch.cuda.current_device()
    wi = want.index if want.index is not None else torch.cuda.current_device()
    if gi != wi:
        raise ValueError(f"{what} is on {got}, the call runs on {want}")


def on_device(method):
    """Run a method of an object with a ``device`` (or ``sim.device``) attribute
    with that CUDA device current, so that the library's launches and the
    default stream belong to the device that holds the object's memory."""
    import functools

    @functools.wraps(method)
    def wrapped(self, *args, **kwargs):
        dev = getattr(self, "device", None)
        if dev is None:
            dev = self.sim.device
        with torch.cuda.device(dev):
            return method(self, *args, **kwargs)
    return wrapped


def pack_params(params) -> np.ndarray:
    """dict or list of dicts (names of ``PARAM_ORDER``) -> float32 [n_sets, 48]."""
    if isinstance(params, dict):
        params = [params]
    out = np.zeros((len(params), L.NPARAMS), dtype=np.float32)
    for s, p in enumerate(params):
        for k, name in enumerate(L.PARAM_ORDER):
            out[s, k] = p[name]
    return out


def select_elites(cost: torch.Tensor, n_e: int, stream=None):
    """The MPPI elite selection on its own (sim_mppi_select_elites): for every row of
    cost [rows, S_c] (float32, CUDA), the indices of its n_e smallest costs (ties to
    the lower index, NaN never selected) in increasing index order, -1 past the row's
    number of non-NaN costs, and the row's smallest cost.  Runs on the device that
    holds `cost` (a given stream must belong to it).  Returns (idx [rows, n_e] int32,
    jmin [rows] float32)."""
    if cost.dim() != 2 or cost.dtype != torch.float32 or not cost.is_cuda or not cost.is_contiguous():
        raise ValueError("cost must be a contiguous float32 CUDA tensor [rows, S_c]")
    rows, S_c = cost.shape
    with torch.cuda.device(cost.device):
        st = _stream_ptr(stream, cost.device)
        idx = torch.empty(rows, max(int(n_e), 0), dtype=torch.int32, device=cost.device)
        jmin = torch.empty(rows, dtype=torch.float32, device=cost.device)
        r = L.load().sim_mppi_select_elites(ctypes.c_void_p(cost.data_ptr()), rows, S_c, int(n_e),
                                            ctypes.c_void_p(idx.data_ptr()),
                                            ctypes.c_void_p(jmin.data_ptr()), st)
    if r != L.SIM_OK:
        raise L.SimError(r, f"sim_mppi_select_elites rejected n_e = {n_e}, S_c = {S_c}, rows = {rows}: "
                            f"need 1 <= n_e <= {L.MAX_ELITES} and S_c >= 1")
    return idx, jmin


class Sim:
    """One batch of drones bound to a device workspace.

    Sim(M, N, model, integrator, dt) for uniform batches, or
    Sim.batched(n_per_world, model_per_world, integrator, dt)."""

    def __init__(self, M=None, N=None, model=L.FIRST_PRINCIPLES, integrator=L.EULER, dt=1 / 500,
                 ctrl=L.CTRL_ATTITUDE, max_cmd_blocks=1, device="cuda", _handle=None):
        self.lib = L.load()
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        if _handle is None:
            self._check_create(self.lib.sim_create(ctypes.byref(h), int(M), int(N), int(model),
                                                   int(integrator), float(dt)))
        else:
            h = _handle
        self.h = h
        self.ntot = int(self.lib.sim_num_drones(h))
        self._check(self.lib.sim_set_control(h, int(ctrl)))
        self.max_cmd_blocks = int(max_cmd_blocks)
        nbytes = ctypes.c_size_t()
        self._check(self.lib.sim_workspace_bytes(h, self.max_cmd_blocks, ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            self._check(self.lib.sim_bind(h, ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                          self.max_cmd_blocks, _stream_ptr(None)))

    @classmethod
    def batched(cls, n_per_world, model_per_world, integrator=L.EULER, dt=1 / 500,
                ctrl=L.CTRL_ATTITUDE, max_cmd_blocks=1, device="cuda"):
        lib = L.load()
        n = np.ascontiguousarray(n_per_world, dtype=np.int64)
        m = np.ascontiguousarray(model_per_world, dtype=np.int32)
        if n.shape != m.shape:
            raise ValueError("n_per_world and model_per_world differ in length")
        h = ctypes.c_void_p()
        r = lib.sim_create_batched(ctypes.byref(h), len(n),
                                   n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                   m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   int(integrator), float(dt))
        if r != L.SIM_OK:
            raise L.SimError(r, "sim_create_batched rejected its arguments")
        return cls(ctrl=ctrl, max_cmd_blocks=max_cmd_blocks, device=device, _handle=h)

    # ------------------------------------------------------------------ helpers
    def _check_create(self, r):
        if r != L.SIM_OK:
            raise L.SimError(r, "sim_create rejected its arguments")

    def _check(self, r):
        if r != L.SIM_OK:
            raise L.SimError(r, self.lib.sim_last_error(self.h).decode())

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            self.lib.sim_destroy(h)
            self.h = None

    # ------------------------------------------------------------------ API
    @on_device
    def set_params(self, params, set_of_world=None, stream=None):
        arr = pack_params(params)
        sow = None
        if set_of_world is not None:
            sow = np.ascontiguousarray(set_of_world, dtype=np.int32)
        self._check(self.lib.sim_set_params(
            self.h, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), arr.shape[0],
            None if sow is None else sow.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            _stream_ptr(stream)))
        self._keep = (arr, sow)

    @on_device
    def set_state(self, x: torch.Tensor, stream=None):
        if x.dtype != torch.float32 or not x.is_contiguous() or tuple(x.shape) != (self.ntot, L.STATE_DIM):
            raise ValueError(f"state must be contiguous float32 [{self.ntot}, {L.STATE_DIM}]")
        self._check(self.lib.sim_set_state(self.h, ctypes.c_void_p(x.data_ptr()), _stream_ptr(stream)))
        self._state_src = x

    @on_device
    def get_state(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.ntot, L.STATE_DIM, dtype=torch.float32, device=self.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != (self.ntot, L.STATE_DIM):
            raise ValueError("bad output tensor")
        self._check(self.lib.sim_get_state(self.h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    @on_device
    def set_commands(self, cmd: torch.Tensor, hold: int, stream=None):
        if cmd.dim() == 2:
            cmd = cmd[None]
        if cmd.dtype != torch.float32 or not cmd.is_contiguous() or cmd.shape[1:] != (self.ntot, L.CMD_DIM):
            raise ValueError(f"commands must be contiguous float32 [n_blocks, {self.ntot}, 4]")
        self._check(self.lib.sim_set_commands(self.h, ctypes.c_void_p(cmd.data_ptr()), cmd.shape[0],
                                              int(hold), _stream_ptr(stream)))
        self._cmd_src = cmd
        self._hold = int(hold)

    def set_block_size(self, tpb: int):
        self._check(self.lib.sim_set_block_size(self.h, int(tpb)))

    @on_device
    def step(self, K: int = 1, stream=None):
        self._check(self.lib.sim_step(self.h, int(K), _stream_ptr(stream)))

    @on_device
    def run(self, n_steps: int, K: int, stream=None):
        self._check(self.lib.sim_run(self.h, int(n_steps), int(K), _stream_ptr(stream)))

    @on_device
    def run_host(self, x0: torch.Tensor, cmd: torch.Tensor, hold: int, n_steps: int, K: int,
                 out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """One rollout from (pinned) host tensors to a host tensor, command blocks
        streamed in behind the first launches (sim_run_host)."""
        if cmd.dim() == 2:
            cmd = cmd[None]
        shape = (self.ntot, L.STATE_DIM)
        if x0.dtype != torch.float32 or not x0.is_contiguous() or tuple(x0.shape) != shape:
            raise ValueError(f"x0 must be contiguous float32 {list(shape)}")
        if cmd.dtype != torch.float32 or not cmd.is_contiguous() or cmd.shape[1:] != (self.ntot, L.CMD_DIM):
            raise ValueError(f"commands must be contiguous float32 [n_blocks, {self.ntot}, 4]")
        if out is None:
            out = torch.empty(shape, dtype=torch.float32, pin_memory=True)
        if out.dtype != torch.float32 or not out.is_contiguous() or tuple(out.shape) != shape:
            raise ValueError("bad output tensor")
        self._check(self.lib.sim_run_host(self.h, ctypes.c_void_p(x0.data_ptr()), ctypes.c_void_p(cmd.data_ptr()),
                                          cmd.shape[0], int(hold), int(n_steps), int(K),
                                          ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        self._cmd_src = cmd
        self._hold = int(hold)
        return out

    @on_device
    def capture_run(self, n_steps: int, K: int) -> torch.cuda.CUDAGraph:
        """Capture `n_steps` steps (launches of at most K) into a CUDA graph.

        The step counter that selects command blocks is baked into the captured
        launches: each replay re-runs steps t .. t + n_steps - 1 counted from
        the command schedule's state at capture time (normally right after
        set_commands), on whatever state the workspace holds."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        t0 = self.steps_taken
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run(n_steps, K, stream=s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        self._check(self.lib.sim_set_step_count(self.h, t0))
        return g

    @on_device
    def sample_rollouts(self, S: int, H: int, seed: torch.Tensor, sigma: float, goals: torch.Tensor,
                        obstacles, w_obs: float, nominal: torch.Tensor | None = None,
                        cost: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Costs [Ntot, S] of S sampled command sequences per drone over H steps
        (see sim_sample_rollouts).  seed: int64 device tensor of one element
        (its bits are the 64-bit Philox key); obstacles: [n_obs, 4] host array."""
        if seed.dtype != torch.int64 or seed.numel() != 1 or not seed.is_cuda:
            raise ValueError("seed must be a one-element int64 CUDA tensor")
        if goals.dtype != torch.float32 or not goals.is_contiguous() or goals.dim() != 2 or goals.shape[1] != 3:
            raise ValueError("goals must be contiguous float32 [M, 3]")
        obs = np.ascontiguousarray(np.asarray(obstacles, dtype=np.float32).reshape(-1, 4))
        if cost is None:
            cost = torch.empty(self.ntot, int(S), dtype=torch.float32, device=self.device)
        if nominal is not None and (nominal.dtype != torch.float32 or not nominal.is_contiguous()):
            raise ValueError("nominal must be contiguous float32 [M, H, 4]")
        self._check(self.lib.sim_sample_rollouts(
            self.h, int(S), int(H), ctypes.c_void_p(seed.data_ptr()), float(sigma),
            None if nominal is None else ctypes.c_void_p(nominal.data_ptr()),
            ctypes.c_void_p(goals.data_ptr()), obs.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
            obs.shape[0], float(w_obs), ctypes.c_void_p(cost.data_ptr()), _stream_ptr(stream)))
        return cost

    @on_device
    def mppi_iteration(self, cfg: dict, seed: torch.Tensor, goals: torch.Tensor, obstacles,
                       mean: torch.Tensor, plan: torch.Tensor | None = None,
                       cost: torch.Tensor | None = None, best_cost: torch.Tensor | None = None,
                       stream=None):
        """One MPPI / iCEM iteration (see sim_mppi_iteration).  cfg keys: S, H,
        n_ctrl, n_elite (elites per controller), sigma, rho, lam, w_obs.  mean
        [Ntot, n_ctrl, H, 4] is updated in place (warm-started).  Returns (plan,
        cost, best_cost)."""
        c = L.MppiConfig(int(cfg["S"]), int(cfg["H"]), int(cfg["n_ctrl"]), int(cfg["n_elite"]),
                         float(cfg["sigma"]), float(cfg["rho"]), float(cfg["lam"]), float(cfg["w_obs"]))
        dev = self.device
        if mean.dtype != torch.float32 or not mean.is_contiguous() or tuple(mean.shape) != (
                self.ntot, c.n_ctrl, c.H, 4):
            raise ValueError("mean must be contiguous float32 [Ntot, n_ctrl, H, 4]")
        if plan is None:
            plan = torch.empty(self.ntot, c.H, 4, dtype=torch.float32, device=dev)
        if cost is None:
            cost = torch.empty(self.ntot, c.S, dtype=torch.float32, device=dev)
        if best_cost is None:
            best_cost = torch.empty(self.ntot, dtype=torch.float32, device=dev)
        obs = np.ascontiguousarray(np.asarray(obstacles, dtype=np.float32).reshape(-1, 4))
        self._check(self.lib.sim_mppi_iteration(
            self.h, ctypes.byref(c), ctypes.c_void_p(seed.data_ptr()), ctypes.c_void_p(goals.data_ptr()),
            obs.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), obs.shape[0],
            ctypes.c_void_p(mean.data_ptr()), ctypes.c_void_p(plan.data_ptr()),
            ctypes.c_void_p(cost.data_ptr()), ctypes.c_void_p(best_cost.data_ptr()), _stream_ptr(stream)))
        return plan, cost, best_cost

    @on_device
    def render_depth(self, height: int, width: int, hfov: float, vfov: float, max_range: float,
                     spheres=(), boxes=(), out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        """Depth images [Ntot, height, width] from each drone's pinhole camera
        (see sim_render_depth).  spheres [n, 4], boxes [n, 6]: host arrays."""
        cam = L.Camera(int(height), int(width), float(hfov), float(vfov), float(max_range))
        sph = np.ascontiguousarray(np.asarray(spheres, dtype=np.float32).reshape(-1, 4))
        box = np.ascontiguousarray(np.asarray(boxes, dtype=np.float32).reshape(-1, 6))
        if out is None:
            out = torch.empty(self.ntot, int(height), int(width), dtype=torch.float32, device=self.device)
        self._check(self.lib.sim_render_depth(
            self.h, ctypes.byref(cam), sph.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), sph.shape[0],
            box.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), box.shape[0],
            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    @on_device
    def status(self, stream=None) -> int:
        v = ctypes.c_uint32()
        self._check(self.lib.sim_status(self.h, ctypes.byref(v), _stream_ptr(stream)))
        return v.value

    @property
    def launches(self) -> int:
        return int(self.lib.sim_launch_count(self.h))

    @property
    def steps_taken(self) -> int:
        return int(self.lib.sim_step_count(self.h))
