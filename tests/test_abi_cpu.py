"""C-ABI checks that need no GPU: the library loads, exports every function
include/*.h declares, and validates arguments on the host (no call here
reaches a CUDA API)."""
import ctypes
import glob
import os
import re

import pytest

import workloads as W
from paper_2606_01478_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith(("defined",))))


@pytest.fixture(scope="module")
def lib():
    return L.load()


def test_library_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(L.declared_symbols()) <= set(declared)


def test_param_order_matches_header():
    src = open(os.path.join(ROOT, "include", "crazyflow.h")).read()
    body = src[src.index("enum sim_param_index"):]
    body = body[body.index("{") + 1:body.index("SIM_P_COUNT")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = [t.strip().split("=")[0].strip() for t in body.split(",") if t.strip()]
    assert len(names) == len(L.PARAM_ORDER) == 48
    for hname, pname in zip(names, L.PARAM_ORDER):
        assert hname == "SIM_P_" + pname.upper()
    assert tuple(W.PARAM_NAMES) == L.PARAM_ORDER


def _create(lib, M, N, model=0, integ=0, dt=0.002):
    h = ctypes.c_void_p()
    r = lib.sim_create(ctypes.byref(h), M, N, model, integ, dt)
    return r, h


def test_create_validates_arguments(lib):
    for args in [(0, 1), (1, 0), (-3, 2), (1 << 20, 1 << 12)]:
        r, h = _create(lib, *args)
        assert r == L.SIM_EINVAL and not h.value
    assert _create(lib, 4, 4, model=7)[0] == L.SIM_EINVAL
    assert _create(lib, 4, 4, integ=2)[0] == L.SIM_EINVAL
    assert _create(lib, 4, 4, dt=0.0)[0] == L.SIM_EINVAL
    assert _create(lib, 4, 4, dt=float("nan"))[0] == L.SIM_EINVAL
    r, h = _create(lib, 3, 5)
    assert r == L.SIM_OK and lib.sim_num_drones(h) == 15
    lib.sim_destroy(h)


def test_create_batched_validates(lib):
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 3)(4, 0, 2)
    m = (ctypes.c_int32 * 3)(0, 1, 0)
    assert lib.sim_create_batched(ctypes.byref(h), 3, n, m, 0, 0.002) == L.SIM_EINVAL
    n = (ctypes.c_int64 * 3)(4, 7, 2)
    m = (ctypes.c_int32 * 3)(0, 5, 0)
    assert lib.sim_create_batched(ctypes.byref(h), 3, n, m, 0, 0.002) == L.SIM_EINVAL
    m = (ctypes.c_int32 * 3)(0, 1, 0)
    assert lib.sim_create_batched(ctypes.byref(h), 3, n, m, 1, 0.002) == L.SIM_OK
    assert lib.sim_num_drones(h) == 13
    # abstracted drones accept attitude commands only
    assert lib.sim_set_control(h, L.CTRL_POSITION) == L.SIM_EINVAL
    assert b"attitude" in lib.sim_last_error(h)
    assert lib.sim_set_control(h, L.CTRL_ATTITUDE) == L.SIM_OK
    lib.sim_destroy(h)


def test_workspace_size_and_call_order(lib):
    r, h = _create(lib, 10, 3)
    nb = ctypes.c_size_t()
    assert lib.sim_workspace_bytes(h, 4, ctypes.byref(nb)) == L.SIM_OK
    # planes + 4 command blocks + staging dominate: 30*(80 + 64 + 80) bytes
    assert nb.value >= 30 * (80 + 4 * 16 + 80)
    assert nb.value % 256 == 0
    assert lib.sim_workspace_bytes(h, 0, ctypes.byref(nb)) == L.SIM_EINVAL
    # nothing may run before a workspace is bound
    assert lib.sim_step(h, 1, None) == L.SIM_ESTATE
    assert lib.sim_set_commands(h, ctypes.c_void_p(16), 1, 1, None) == L.SIM_ESTATE
    assert lib.sim_step(h, 0, None) == L.SIM_EINVAL
    assert lib.sim_set_block_size(h, 48) == L.SIM_EINVAL
    assert lib.sim_set_block_size(h, 512) == L.SIM_EINVAL
    assert lib.sim_set_block_size(h, 64) == L.SIM_OK
    assert lib.sim_set_control(h, 9) == L.SIM_EINVAL
    # a misaligned workspace is refused before any CUDA call
    assert lib.sim_bind(h, ctypes.c_void_p(0x1000 + 8), 1 << 20, 1, None) == L.SIM_EINVAL
    assert lib.sim_bind(h, ctypes.c_void_p(0x1000), 16, 1, None) == L.SIM_ENOMEM
    lib.sim_destroy(h)


def test_null_handle_is_rejected(lib):
    assert lib.sim_step(None, 1, None) == L.SIM_EINVAL
    assert lib.sim_num_drones(None) == -1
    assert lib.sim_last_error(None) == b"NULL handle"
    lib.sim_destroy(None)


def test_rollout_objective_validation(lib):
    r, h = _create(lib, 64, 1)
    nb0, nb1 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.sim_rollout_workspace_bytes(h, 40, 10, ctypes.byref(nb0)) == L.SIM_OK
    obj = L.Objective()
    obj.kind = 7
    assert lib.sim_rollout_set_objective(h, ctypes.byref(obj)) == L.SIM_EINVAL
    obj.kind = L.OBJ_TRACKING_REWARD
    obj.w_theta = 0.1
    obj.w_dact[2] = -1.0
    assert lib.sim_rollout_set_objective(h, ctypes.byref(obj)) == L.SIM_EINVAL
    obj.w_dact[2] = float("nan")
    assert lib.sim_rollout_set_objective(h, ctypes.byref(obj)) == L.SIM_EINVAL
    obj.w_dact[2] = 0.0
    assert lib.sim_rollout_set_objective(h, ctypes.byref(obj)) == L.SIM_OK
    # the reward keeps the previous action per checkpoint and segment step
    assert lib.sim_rollout_workspace_bytes(h, 40, 10, ctypes.byref(nb1)) == L.SIM_OK
    assert nb1.value >= nb0.value + 64 * 16 * (4 + 10)
    assert lib.sim_rollout_set_objective(h, None) == L.SIM_OK
    assert lib.sim_rollout_workspace_bytes(h, 40, 10, ctypes.byref(nb1)) == L.SIM_OK
    assert nb1.value == nb0.value
    lib.sim_destroy(h)


def test_rollout_action_repeat_validation(lib):
    r, h = _create(lib, 32, 1)
    nb1, nb10 = ctypes.c_size_t(), ctypes.c_size_t()
    assert lib.sim_rollout_workspace_bytes(h, 40, 10, ctypes.byref(nb1)) == L.SIM_OK
    for bad in (0, -2, 101):
        assert lib.sim_rollout_set_action_repeat(h, bad) == L.SIM_EINVAL
    assert lib.sim_rollout_set_action_repeat(h, 10) == L.SIM_OK
    assert lib.sim_rollout_workspace_bytes(h, 40, 10, ctypes.byref(nb10)) == L.SIM_OK
    # segments keep C R sub-step states of 80 bytes
    assert nb10.value >= nb1.value + 32 * 80 * 10 * 9
    lib.sim_destroy(h)


def test_run_host_validates_before_any_cuda_call(lib):
    r, h = _create(lib, 8, 2)
    buf = ctypes.c_void_p(0x1000)
    assert lib.sim_run_host(h, buf, buf, 1, 1, 10, 5, buf, None) == L.SIM_ESTATE
    assert b"bind" in lib.sim_last_error(h)
    lib.sim_destroy(h)


def test_rollout_precision_validation(lib):
    r, h = _create(lib, 16, 1)
    assert lib.sim_rollout_set_precision(h, 2) == L.SIM_EINVAL
    assert lib.sim_rollout_set_precision(h, L.MLP_BF16) == L.SIM_OK
    assert lib.sim_rollout_set_precision(h, L.MLP_HILO) == L.SIM_OK
    lib.sim_destroy(h)


def test_select_elites_refuses_host_tensors():
    """The elite selection's binding takes CUDA tensors only: a host tensor is an
    error, never a CPU computation."""
    import torch
    from paper_2606_01478_b300 import select_elites
    with pytest.raises(ValueError):
        select_elites(torch.zeros(2, 3), 1)


def test_calls_refuse_a_stream_or_tensor_of_another_device():
    """The binding refuses a stream that belongs to another GPU than the one the
    call runs on (checked on the host, before anything launches)."""
    import torch
    from paper_2606_01478_b300.sim import _check_same_device
    _check_same_device(torch.device("cuda", 1), torch.device("cuda", 1), "stream")
    with pytest.raises(ValueError):
        _check_same_device(torch.device("cuda", 1), torch.device("cuda", 0), "stream")
    with pytest.raises(ValueError):
        _check_same_device(torch.device("cpu"), torch.device("cuda", 0), "cost")



def test_autotune_keys_name_everything_the_timing_depends_on():
    """sim_autotune_key (no device work): handles that differ only by integrator,
    control interface, model mix or shape get different keys; identical handles
    share one; the key records the operation and the run length."""
    import ctypes
    import numpy as np
    lib = L.load()

    def key(h, op=L.TUNE_STEP, n_steps=100, S=1, H=1):
        r = L.TuneRequest()
        r.op, r.n_steps, r.S, r.H, r.reps = op, n_steps, S, H, 1
        buf = ctypes.create_string_buffer(512)
        assert lib.sim_autotune_key(h, ctypes.byref(r), buf, 512) == L.SIM_OK
        return buf.value.decode()

    def uniform(M, N, model, integ, ctrl=L.CTRL_ATTITUDE):
        h = ctypes.c_void_p()
        assert lib.sim_create(ctypes.byref(h), M, N, model, integ, 1 / 500) == L.SIM_OK
        assert lib.sim_set_control(h, ctrl) == L.SIM_OK
        return h

    def batched(n, models):
        h = ctypes.c_void_p()
        n = np.asarray(n, np.int64)
        m = np.asarray(models, np.int32)
        assert lib.sim_create_batched(ctypes.byref(h), len(n), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), L.EULER,
                                      1 / 500) == L.SIM_OK
        return h

    a = uniform(64, 1, 0, L.EULER)
    b = uniform(64, 1, 0, L.RK4)
    c = uniform(64, 1, 0, L.EULER)
    d = uniform(64, 1, 0, L.EULER, L.CTRL_TORQUE)
    e = uniform(32, 2, 0, L.EULER)
    assert key(a) == key(c)
    assert len({key(a), key(b), key(d), key(e)}) == 4
    assert "integrator=euler" in key(a) and "integrator=rk4" in key(b) and "ctrl=torque" in key(d)
    assert key(a, n_steps=100) != key(a, n_steps=200) and "steps=100" in key(a)
    assert "op=sample" in key(a, op=L.TUNE_SAMPLE, S=256, H=50) and "S=256|H=50" in key(a, op=L.TUNE_SAMPLE, S=256, H=50)
    f = batched([5, 7], [0, 1])
    g = batched([5, 7], [1, 0])
    h = batched([7, 5], [0, 1])
    assert len({key(f), key(g), key(h)}) == 3
    r = L.TuneRequest()
    r.op = 7
    buf = ctypes.create_string_buffer(512)
    assert lib.sim_autotune_key(a, ctypes.byref(r), buf, 512) == L.SIM_EINVAL
    for x in (a, b, c, d, e, f, g, h):
        lib.sim_destroy(x)



def test_autotune_refuses_bad_requests_before_any_device_work():
    """sim_autotune validates on the host: an unknown op, reps out of range, bad
    candidate block sizes or too many candidates are SIM_EINVAL; a handle with
    no bound workspace is SIM_ESTATE; nothing reaches the device."""
    import ctypes
    lib = L.load()
    h = ctypes.c_void_p()
    assert lib.sim_create(ctypes.byref(h), 8, 1, 0, L.EULER, 1 / 500) == L.SIM_OK
    res = L.TuneResult()

    def call(**kw):
        r = L.TuneRequest()
        r.op, r.reps, r.n_steps = L.TUNE_STEP, 1, 10
        for k, v in kw.items():
            setattr(r, k, v)
        return lib.sim_autotune(h, ctypes.byref(r), ctypes.byref(res), None)

    assert call(op=5) == L.SIM_EINVAL
    assert call(reps=0) == L.SIM_EINVAL
    assert call(reps=101) == L.SIM_EINVAL
    assert call(n_tpb=L.TUNE_MAX + 1) == L.SIM_EINVAL
    r = L.TuneRequest()
    r.op, r.reps, r.n_steps, r.n_tpb = L.TUNE_STEP, 1, 10, 1
    r.tpb[0] = 48  # not a multiple of 32
    assert lib.sim_autotune(h, ctypes.byref(r), ctypes.byref(res), None) == L.SIM_EINVAL
    assert call(n_steps=0) == L.SIM_EINVAL
    assert call() == L.SIM_ESTATE  # not bound: no workspace, state or commands
    assert b"sim_autotune" in lib.sim_last_error(h)
    assert lib.sim_autotune(h, None, ctypes.byref(res), None) == L.SIM_EINVAL
    lib.sim_destroy(h)
