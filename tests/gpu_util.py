"""Helpers shared by the GPU parity tests: drive the CUDA path through the
binding and compare with the FP64 oracle element by element."""
import numpy as np
import torch

from paper_2606_01478_b300 import Sim

# Parity tolerances of the FP32 CUDA path against the FP64 oracle, per state
# field.  Position: the 1e-4 m bar after 1000 steps at 500 Hz.  The other
# fields scale with their magnitude in flight (quaternion ~1, velocity
# ~1 m/s, body rate ~1-10 rad/s, rotor speed ~1.5e4 RPM, integrator ~1 m s)
# times the same ~1e-4 relative budget (FP32 unit round-off 6e-8 amplified
# by ~1e3 steps and the closed loop).
TOL_FP = {"p": 1e-4, "q": 2e-5, "v": 2e-4, "w": 2e-3, "W": 0.1, "I": 1e-4}
TOL_ABS = {"p": 1e-4, "psi": 2e-5, "v": 2e-4, "psid": 2e-3, "f": 1e-6}

FP_SLICES = {"p": slice(0, 3), "q": slice(3, 7), "v": slice(7, 10), "w": slice(10, 13),
             "W": slice(13, 17), "I": slice(17, 20)}
ABS_SLICES = {"p": slice(0, 3), "psi": slice(3, 6), "v": slice(6, 9), "psid": slice(9, 12),
              "f": slice(12, 13)}


def make_sim(wl, max_blocks=None, tpb=None, device="cuda"):
    """CUDA Sim loaded with a workloads.Workload (uniform worlds)."""
    models = np.unique(wl.model_of_world)
    if len(models) == 1:
        sim = Sim(wl.M, wl.N, int(models[0]), wl.integrator, wl.dt, ctrl=wl.ctrl,
                  max_cmd_blocks=max_blocks or wl.cmd.shape[0], device=device)
    else:
        sim = Sim.batched(np.full(wl.M, wl.N), wl.model_of_world, wl.integrator, wl.dt,
                          ctrl=wl.ctrl, max_cmd_blocks=max_blocks or wl.cmd.shape[0], device=device)
    if tpb:
        sim.set_block_size(tpb)
    sim.set_params(wl.params, wl.param_set_of_world)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device=device).contiguous())
    sim.set_commands(torch.tensor(wl.cmd, dtype=torch.float32, device=device).contiguous(), wl.hold)
    return sim


def field_errors(gpu: np.ndarray, ref: np.ndarray, model_of_drone: np.ndarray) -> dict:
    """Max abs error per named field, split by model."""
    out = {}
    for model, slices in ((0, FP_SLICES), (1, ABS_SLICES), (2, ABS_SLICES)):
        sel = model_of_drone == model
        if not sel.any():
            continue
        for k, s in slices.items():
            out[(model, k)] = float(np.abs(gpu[sel, s] - ref[sel, s]).max())
    return out


def assert_parity(gpu, ref, model_of_drone, scale=1.0):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert np.isfinite(gpu).all()
    errs = field_errors(gpu, ref, model_of_drone)
    bad = {}
    for (model, k), e in errs.items():
        tol = (TOL_FP if model == 0 else TOL_ABS)[k] * scale
        if not e <= tol:
            bad[(model, k)] = (e, tol)
    assert not bad, f"parity failures (err, tol): {bad}; all errors: {errs}"
    return errs
