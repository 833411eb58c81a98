"""ctypes loader of libcrazyflow_b300.so (the C-ABI in include/crazyflow.h).

The loader fails loudly: there is no fallback of any kind.  ``load()`` raises
if the shared library has not been built (``python -m
paper_2606_01478_b300.build``) or lacks a symbol the header declares.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_float, c_int, c_int64, c_size_t, c_uint32, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcrazyflow_b300.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ESTATE = 0, -1, -2, -3, -4
SIM_FLAG_NONFINITE = 1
SIM_FLAG_TIMEOUT = 2
FIRST_PRINCIPLES, ABSTRACTED, ABSTRACTED_NOTHRUST = 0, 1, 2
EULER, RK4 = 0, 1
CTRL_ROTOR_SPEED, CTRL_ATTITUDE, CTRL_POSITION, CTRL_TORQUE = 0, 1, 2, 3
STATE_DIM, CMD_DIM, NPARAMS = 20, 4, 48
POLICY_NPARAMS = 5316
MAX_OBSTACLES = 64
MAX_ELITES = 4096

# Order of enum sim_param_index in include/crazyflow.h (checked by a CPU test).
PARAM_ORDER = (
    "mass", "Jx", "Jy", "Jz", "arm", "kf", "km",
    "cv_up", "cd_up", "cv_down", "cd_down", "omega_max",
    "Ca_x", "Ca_y", "Ca_z",
    "KR_x", "KR_y", "KR_z", "Kw_x", "Kw_y", "Kw_z",
    "Kp_x", "Kp_y", "Kp_z", "Kd_x", "Kd_y", "Kd_z", "Ki_x", "Ki_y", "Ki_z",
    "max_angle", "thrust_scale", "g",
    "c1_r", "c1_p", "c1_y", "c2_r", "c2_p", "c2_y", "c3_r", "c3_p", "c3_y",
    "c_tau", "c_f",
    "J_p", "kf0", "kf1", "km1",
)

class Camera(ctypes.Structure):
    """sim_camera (include/crazyflow.h)."""
    _fields_ = [("height", c_int), ("width", c_int), ("hfov", c_float), ("vfov", c_float),
                ("max_range", c_float)]


class Objective(ctypes.Structure):
    """sim_objective (include/crazyflow.h)."""
    _fields_ = [("kind", c_int), ("w_theta", c_float), ("w_act", c_float * 4), ("w_dact", c_float * 4)]


OBJ_SQUARED, OBJ_TRACKING_REWARD = 0, 1
MLP_HILO, MLP_BF16 = 0, 1


class MppiConfig(ctypes.Structure):
    """sim_mppi_config (include/crazyflow.h)."""
    _fields_ = [("S", c_int), ("H", c_int), ("n_ctrl", c_int), ("n_elite", c_int), ("sigma", c_float),
                ("rho", c_float), ("lambda_", c_float), ("w_obs", c_float)]


TUNE_STEP, TUNE_SAMPLE = 0, 1
TUNE_MAX = 16


class TuneRequest(ctypes.Structure):
    """sim_tune_request (include/crazyflow.h)."""
    _fields_ = [("op", c_int), ("reps", c_int), ("use_cache", c_int), ("n_tpb", c_int),
                ("tpb", c_int * TUNE_MAX), ("n_K", c_int), ("K", c_int * TUNE_MAX), ("n_steps", c_int64),
                ("S", c_int), ("H", c_int), ("seed", c_void_p), ("sigma", c_float), ("nominal", c_void_p),
                ("goals", c_void_p), ("obstacles", c_void_p), ("n_obs", c_int), ("w_obs", c_float),
                ("cost", c_void_p)]


class TuneResult(ctypes.Structure):
    """sim_tune_result (include/crazyflow.h)."""
    _fields_ = [("tpb", c_int), ("K", c_int), ("ms", c_float), ("from_cache", c_int), ("n_trials", c_int),
                ("cache_written", c_int), ("trial_ms", c_float * (TUNE_MAX * TUNE_MAX)),
                ("key", ctypes.c_char * 512)]


_SIGS = {
    "sim_create": (c_int, [POINTER(c_void_p), c_int64, c_int64, c_int, c_int, c_float]),
    "sim_create_batched": (c_int, [POINTER(c_void_p), c_int64, POINTER(c_int64), POINTER(ctypes.c_int32),
                                   c_int, c_float]),
    "sim_set_control": (c_int, [c_void_p, c_int]),
    "sim_workspace_bytes": (c_int, [c_void_p, c_int64, POINTER(c_size_t)]),
    "sim_bind": (c_int, [c_void_p, c_void_p, c_size_t, c_int64, c_void_p]),
    "sim_set_params": (c_int, [c_void_p, POINTER(c_float), c_int64, POINTER(ctypes.c_int32), c_void_p]),
    "sim_set_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "sim_get_state": (c_int, [c_void_p, c_void_p, c_void_p]),
    "sim_set_commands": (c_int, [c_void_p, c_void_p, c_int64, c_int, c_void_p]),
    "sim_step": (c_int, [c_void_p, c_int, c_void_p]),
    "sim_run": (c_int, [c_void_p, c_int64, c_int, c_void_p]),
    "sim_set_block_size": (c_int, [c_void_p, c_int]),
    "sim_status": (c_int, [c_void_p, POINTER(c_uint32), c_void_p]),
    "sim_num_drones": (c_int64, [c_void_p]),
    "sim_step_count": (c_int64, [c_void_p]),
    "sim_set_step_count": (c_int, [c_void_p, c_int64]),
    "sim_launch_count": (c_int64, [c_void_p]),
    "sim_selftest_wait_timeout": (c_int, [c_void_p, c_void_p]),
    "sim_sample_rollouts": (c_int, [c_void_p, c_int, c_int, c_void_p, c_float, c_void_p, c_void_p,
                                    POINTER(c_float), c_int, c_float, c_void_p, c_void_p]),
    "sim_mppi_iteration": (c_int, [c_void_p, POINTER(MppiConfig), c_void_p, c_void_p,
                                   POINTER(c_float), c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "sim_adam_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p,
                              c_float, c_float, c_float, c_float, c_void_p]),
    "sim_render_depth": (c_int, [c_void_p, POINTER(Camera), POINTER(c_float), c_int, POINTER(c_float),
                                 c_int, c_void_p, c_void_p]),
    "sim_mppi_select_elites": (c_int, [c_void_p, c_int64, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "sim_philox_normals": (c_int, [c_void_p, ctypes.c_uint64, c_int64, c_int, c_void_p, c_void_p,
                                   c_void_p]),
    "sim_run_host": (c_int, [c_void_p, c_void_p, c_void_p, c_int64, c_int, c_int64, c_int, c_void_p,
                             c_void_p]),
    "sim_rollout_set_objective": (c_int, [c_void_p, POINTER(Objective)]),
    "sim_rollout_set_action_repeat": (c_int, [c_void_p, c_int]),
    "sim_rollout_set_precision": (c_int, [c_void_p, c_int]),
    "sim_rollout_workspace_bytes": (c_int, [c_void_p, c_int, c_int, POINTER(c_size_t)]),
    "sim_rollout_fwd": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_float,
                                c_void_p, c_size_t, c_void_p, c_void_p]),
    "sim_rollout_bwd": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_float,
                                c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sim_rollout_grad_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int,
                                         c_float, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sim_rollout_noalloc_max_bytes": (c_int, [POINTER(c_size_t)]),
    "sim_rollout_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_float,
                                 c_void_p, c_size_t, c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p]),
    "sim_autotune": (c_int, [c_void_p, POINTER(TuneRequest), POINTER(TuneResult), c_void_p]),
    "sim_autotune_key": (c_int, [c_void_p, POINTER(TuneRequest), ctypes.c_char_p, c_size_t]),
    "sim_last_error": (c_char_p, [c_void_p]),
    "sim_destroy": (None, [c_void_p]),
}

_lib = None


class SimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def load():
    """Load the library (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2606_01478_b300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)  # AttributeError if the symbol is missing
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols() -> tuple:
    return tuple(_SIGS)
