"""Benchmark of the B300 drone physics step (one JSON line on stdout).

Default workload (the headline configuration, the paper's swarm scale): a
swarm of 1000 worlds x 4000 drones (4M drones), even worlds first-principles,
odd worlds the abstracted identified model with per-world coefficients,
attitude interface, Euler at dt = 1/500 s, 200 steps fused into one launch
(K from the autotuner).  One benchmark "step" is that whole 200-step rollout.
The metric is drone-steps per second; the line carries the fused launch's
FP32 roofline, the single-step (K = 1) launches' HBM roofline, the end-to-end
rate through the C-ABI with pinned host buffers, the FP64 oracle on the host
cores and the final-state error against it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload on the host cores.
Under torchrun (N > 1) every rank runs an independent shard of worlds (no
collective on the data path; "weak" scaling), and rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import flopcount  # noqa: E402
import workloads as W  # noqa: E402

METRIC = ("drone-steps/s (fwd, fused Euler, 4M-drone swarm of first-principles and abstracted "
          "drones, attitude controller)")
UNIT = "drone-steps/s"
# Algorithmic FP32 work per drone-step (flopcount.py: the method's formulas
# restated on an op-counting scalar; additions, subtractions, multiplications,
# divisions; the attitude decode amortised over 50-step command holds).
_FLOPS = flopcount.table()
FLOP_PER_DRONE_STEP = {(m, i, "attitude"): c["flop"] for (m, i), c in _FLOPS.items()}
MUFU_PER_DRONE_STEP = {(m, i, "attitude"): c["mufu"] for (m, i), c in _FLOPS.items()}
# Algorithmic HBM bytes of one single-step launch per drone: state in + out
# (first-principles 5 float4 planes, abstracted 4) + one float4 command.
BYTES_PER_DRONE_STEP = {"fp": 80 + 80 + 16, "abs": 64 + 64 + 16}
SM_COUNT = 148
FP32_LANES_PER_SM = 128


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# --------------------------------------------------------------------------- clocks


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# --------------------------------------------------------------------------- helpers


# Source files each profiled kernel is built from.
KERNEL_SOURCES = {
    "step_kernel": ("step.cu", "stepcore.cuh", "physics.cuh", "common.cuh"),
    "step_batched_kernel": ("step.cu", "stepcore.cuh", "physics.cuh", "common.cuh"),
    "step_batched_single_kernel": ("step.cu", "stepcore.cuh", "physics.cuh", "common.cuh"),
    "rollout_bwd_kernel": ("rollout.cu", "physics.cuh", "common.cuh"),
    "sample_kernel": ("sample.cu", "noise.cuh", "stepcore.cuh", "physics.cuh", "common.cuh"),
}


def _src_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_01478_b300", "csrc")
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(f"{kernel}:{workload}")
    if not rec or rec.get("src_hash") != _src_hash(kernel):
        return None
    return rec.get("bytes_per_launch")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _max_over_ranks(dist, x: float) -> float:
    if dist is None:
        return x
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(dist):
    if dist is not None:
        dist.barrier()


# --------------------------------------------------------------------------- reference arm


def oracle_sample(wl, n_drones: int, n_steps: int) -> tuple[float, int]:
    """Time the FP64 oracle on the first n_drones drones for n_steps steps.
    Returns (seconds, drone-steps)."""
    from oracle import physics as ph
    t = time.perf_counter()
    ph.rollout_workload(wl, steps=n_steps, drones=np.arange(n_drones))
    return time.perf_counter() - t, n_drones * n_steps


def _cpu_model() -> str:
    """The host CPU's model name (Linux), for the record beside the CPU timing."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def world_subset(wl, worlds: int):
    """The first `worlds` worlds of a uniform-N workload (an exact sub-problem:
    drones do not interact)."""
    import dataclasses
    n = worlds * wl.N
    return dataclasses.replace(wl, name=f"{wl.name}_first{worlds}worlds", M=worlds,
                               param_set_of_world=wl.param_set_of_world[:worlds],
                               model_of_world=wl.model_of_world[:worlds], x0=wl.x0[:n],
                               cmd=wl.cmd[:, :n])


def cpu_baseline(wl, budget_s: float = 12.0) -> dict:
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload (`wl` is already the sample's worlds): all its drones, as many
    steps as fit about budget_s seconds."""
    n = wl.M * wl.N
    dt1, _ = oracle_sample(wl, n, 2)
    steps = int(max(4, min(wl.steps, budget_s / max(dt1 / 2, 1e-6))))
    secs, units = oracle_sample(wl, n, steps)
    return {"value": units / secs, "unit": UNIT, "cores": torch.get_num_threads(),
            "cpu": _cpu_model(), "kind": "oracle",
            "sample": f"{n} drones ({wl.M} worlds x {wl.N}) x {steps} of {wl.steps} steps "
                      "(FP64 torch CPU oracle)"}


STATE_FIELDS = {"p_m": slice(0, 3), "q": slice(3, 7), "v_m_s": slice(7, 10), "w_rad_s": slice(10, 13),
                "W_rpm": slice(13, 17)}


def error_vs_fp64(wl, gpu_final: np.ndarray, n_drones: int = 256) -> dict:
    """Final-state error of the GPU rollout against the FP64 oracle on evenly
    spaced drones (whole rollouts from the float32 inputs the GPU received),
    max and median absolute error per state field (part of the CPU-baseline leg)."""
    import dataclasses
    from oracle import physics as ph
    idx = np.linspace(0, wl.M * wl.N - 1, n_drones).round().astype(np.int64)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    wl32 = dataclasses.replace(wl, x0=f32(wl.x0), cmd=f32(wl.cmd))
    ref = ph.rollout_workload(wl32, drones=idx).numpy()
    err = np.abs(np.asarray(gpu_final, np.float64)[idx] - ref)
    return {"drones": int(n_drones), "steps": int(wl.steps),
            "max_abs": {k: float(err[:, sl].max()) for k, sl in STATE_FIELDS.items()},
            "median_abs": {k: float(np.median(err[:, sl])) for k, sl in STATE_FIELDS.items()},
            "reference": "FP64 oracle from the same float32 inputs"}


ABS_FIELDS = {"p_m": slice(0, 3), "psi_rad": slice(3, 6), "v_m_s": slice(6, 9),
              "psidot_rad_s": slice(9, 12), "f_sigma_N": slice(12, 13)}


def mixed_sample(wl, per_model: int = 64, seed: int = 2):
    """Drones drawn from each model of a mixed workload, with their inputs, for
    the FP64 comparison of the CPU leg."""
    rng = np.random.default_rng(seed)
    models = wl.model_of_world[np.arange(wl.M * wl.N) // wl.N]
    sample = np.concatenate([rng.choice(np.nonzero(models == m)[0], per_model, replace=False)
                             for m in np.unique(models)])
    return {"drones": sample, "x0": wl.x0[sample].copy(), "cmd": wl.cmd[:, sample].copy(),
            "world": sample // wl.N, "wl": wl}


def mixed_error_vs_fp64(ms, gpu_rows) -> dict:
    """Final-state error of a mixed swarm's rollout against the FP64 oracle on
    the sampled drones of each model, from the float32 inputs the GPU received
    (part of the CPU-baseline leg)."""
    from oracle import physics as ph
    wl = ms["wl"]
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    world = ms["world"]
    models = wl.model_of_world[world]
    ref = ph.rollout(f32(ms["x0"]), f32(ms["cmd"]), wl.hold, wl.steps, wl.params,
                     wl.param_set_of_world[world], models, wl.dt, wl.integrator, wl.ctrl).numpy()
    err = np.abs(np.asarray(gpu_rows, np.float64) - ref)
    out = {"drones_per_model": int(len(ms["drones"]) // len(np.unique(models))), "steps": int(wl.steps),
           "reference": "FP64 oracle from the same float32 inputs"}
    for m, name, fields in ((0, "first_principles", STATE_FIELDS), (1, "abstracted", ABS_FIELDS)):
        e = err[models == m]
        if len(e):
            out[name] = {"max_abs": {k: float(e[:, sl].max()) for k, sl in fields.items()},
                         "median_abs": {k: float(np.median(e[:, sl])) for k, sl in fields.items()}}
    return out


def sampling_error_vs_fp64(drones, samples, seed, gpu_cost) -> dict:
    """Relative error of 64 sampled rollout costs of the uneven sampling workload
    (the last timed replay, its seed) against the FP64 oracle (CPU-baseline leg)."""
    from oracle import sampling as sa
    wl = W.uneven_sampling_rk4()
    world = np.repeat(np.arange(wl.M), wl.n_per_world)
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    ref = sa.rollout_cost(f32(wl.x0), f32(wl.goals), f32(wl.obstacles), wl.params, wl.S, wl.H, wl.dt,
                          wl.sigma, seed, wl.w_obs, drones, samples, world)
    rel = np.abs(np.asarray(gpu_cost, np.float64) - ref) / np.abs(ref)
    return {"pairs": int(len(drones)), "max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
            "reference": "FP64 oracle from the same float32 inputs, same Philox seed"}


CPU_WORLDS = 4  # the oracle's sample of the headline swarm: worlds 0-3 (two of each model)


def run_reference(args, wl):
    dist, rank, ws = _dist()
    if rank != 0:
        return 0
    sub = world_subset(wl, CPU_WORLDS)
    n = sub.M * sub.N
    n_steps = 10
    for _ in range(args.warmup):
        oracle_sample(sub, n, n_steps)
    secs, units = 0.0, 0
    for _ in range(args.steps):
        s, u = oracle_sample(sub, n, n_steps)
        secs += s
        units += u
    value = units / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(wl, args, wl.K),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
                         "cpu": _cpu_model(), "kind": "oracle",
                         "sample": f"{n} drones ({sub.M} worlds x {sub.N}, both models) x {n_steps} "
                                   f"of {wl.steps} steps per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(wl, args, K):
    return {"workload": wl.name, "worlds": wl.M, "drones_per_world": wl.N,
            "model": "mixed: first-principles (even worlds), abstracted (odd worlds, coefficients "
                     "x U(0.9, 1.1) per world)",
            "integrator": "euler", "control": "attitude", "dt": wl.dt, "steps_per_rollout": wl.steps,
            "K_fused": K, "parallelism": f"replicas x{args.gpus} (independent worlds)",
            "l2": "flushed (256 MiB write) before every timed iteration; the inputs (320 MB of "
                  "state planes, 256 MB of command blocks) exceed L2"}


def _fp32_peak():
    pk, kind = peaks()
    clk = pk.get("sm_max_mhz", 2032.0)
    return SM_COUNT * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12, clk, kind


# --------------------------------------------------------------------------- B300 arm


def run_b300(args, wl):
    from paper_2606_01478_b300 import Sim, autotune
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    n = wl.M * wl.N
    n_fp = int((wl.model_of_world == 0).sum()) * wl.N
    n_abs = n - n_fp

    sim = Sim.batched(np.full(wl.M, wl.N), wl.model_of_world, wl.integrator, wl.dt, ctrl=wl.ctrl,
                      max_cmd_blocks=wl.cmd.shape[0], device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0_host = torch.from_numpy(np.ascontiguousarray(wl.x0, dtype=np.float32)).pin_memory()
    cmd_host = torch.from_numpy(np.ascontiguousarray(wl.cmd, dtype=np.float32)).pin_memory()
    out_host = torch.empty_like(x0_host).pin_memory()
    x0_dev = x0_host.to(dev)
    cmd_dev = cmd_host.to(dev)
    # what the CPU leg needs, then drop the float64 arrays (1.2 GB)
    sub = world_subset(wl, CPU_WORLDS)
    sub.x0, sub.cmd = sub.x0.copy(), sub.cmd.copy()
    msample = mixed_sample(wl)
    wl.x0 = wl.cmd = None
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sim.set_state(x0_dev)
    sim.set_commands(cmd_dev, wl.hold)
    if args.tpb:
        sim.set_block_size(args.tpb)
        tuned = {"tpb": args.tpb, "K": wl.K, "source": "--tpb"}
    else:
        tuned = autotune.tune_step(sim, wl.steps, Ks=(50, 100, 200), reps=1)
        tuned = {k: v for k, v in tuned.items() if k != "table"}
    K = int(tuned["K"])
    n_launch = (wl.steps + K - 1) // K

    def reset():
        sim.set_state(x0_dev)
        sim.set_commands(cmd_dev, wl.hold)

    def timed(fn, it):
        reset()
        flush.fill_(it & 0xFF)
        # keep the device busy while the host enqueues the launches, so the
        # events time device execution and not host launch latency
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(args.warmup):
        reset()
        sim.run(wl.steps, K)
    torch.cuda.synchronize()
    assert sim.status() == 0, "non-finite state during warm-up"

    # device-resident timing (inputs already in HBM): two events per rollout
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    _barrier(dist)
    torch.cuda.synchronize()
    per_iter_ms = [timed(lambda: sim.run(wl.steps, K), it) for it in range(args.steps)]
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = sampler.stop()
    gpu_launches = args.steps * n_launch
    total_ms = _max_over_ranks(dist, sum(per_iter_ms))
    units = n * wl.steps * args.steps * ws
    value = units / (total_ms / 1e3)

    # the same rollout as 200 single-step launches (each reads and writes the
    # state planes once): the HBM roofline of the step
    k1_ms = statistics.median([timed(lambda: sim.run(wl.steps, 1), it) for it in range(3)])

    # end to end through the C-ABI with host buffers (pinned): state and command
    # blocks in, the final state out, inside the timed region
    e2e_ms = []
    for it in range(args.steps):
        flush.fill_(it & 0xFF)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.run_host(x0_host, cmd_host, wl.hold, wl.steps, K, out=out_host)
        t1.record(stream)
        t1.synchronize()
        e2e_ms.append(t0.elapsed_time(t1))
    e2e_total = _max_over_ranks(dist, sum(e2e_ms))
    assert sim.status() == 0
    h2d = x0_host.numel() * 4 + cmd_host.numel() * 4
    d2h = out_host.numel() * 4
    final_sample = out_host.numpy()[msample["drones"]].copy()
    del sim, x0_dev, cmd_dev, flush
    torch.cuda.empty_cache()

    if rank != 0:
        return 0
    fp32_peak, clk_max, pk_kind = _fp32_peak()
    f_fp = FLOP_PER_DRONE_STEP[("fp", "euler", "attitude")]
    f_abs = FLOP_PER_DRONE_STEP[("abs", "euler", "attitude")]
    flop_per_step = n_fp * f_fp + n_abs * f_abs
    # average launch duration over the timed region (rollout time / launches)
    avg_launch_s = total_ms / (args.steps * n_launch) / 1e3
    achieved = flop_per_step * K / avg_launch_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "traffic": _profiled_traffic("step_batched_kernel", wl.name),
            "kernel": "step_batched_kernel<Euler, attitude, lag rotors> (first-principles and "
                      "abstracted warps in one persistent launch)",
            "flop_per_drone_step": {"first_principles": f_fp, "abstracted": f_abs},
            "mufu_per_drone_step": {"first_principles": MUFU_PER_DRONE_STEP[("fp", "euler", "attitude")],
                                    "abstracted": MUFU_PER_DRONE_STEP[("abs", "euler", "attitude")]},
            "flop_source": "flopcount.py (the method's formulas on an op-counting scalar)",
            "launch_ms_timed_region": avg_launch_s * 1e3,
            "peak_basis": f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                          f"{clk_max:.0f} MHz (max SM clock, {pk_kind} peaks file)"}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (fp32_peak * clocks["sm_mhz"] / clk_max)
    # the special-function (XU) work charged at the XU rate: one warp instruction
    # per SM per cycle (32 operations), the peak ncu reports for this pipe
    mufu = (n_fp * MUFU_PER_DRONE_STEP[("fp", "euler", "attitude")]
            + n_abs * MUFU_PER_DRONE_STEP[("abs", "euler", "attitude")]) * K
    xu_peak = SM_COUNT * 32 * clk_max * 1e6 / 1e12
    roof["xu"] = {"achieved": mufu / avg_launch_s / 1e12, "peak": xu_peak, "unit": "Tops/s",
                  "frac": mufu / avg_launch_s / 1e12 / xu_peak,
                  "note": "sqrt, sin, cos per drone-step from flopcount.py; the FMA pipe binds"}
    pk, kind = peaks()
    byt = n_fp * BYTES_PER_DRONE_STEP["fp"] + n_abs * BYTES_PER_DRONE_STEP["abs"]
    hbm = byt * wl.steps / (k1_ms / 1e3) / 1e9
    single = {"value": n * wl.steps / (k1_ms / 1e3), "unit": UNIT, "ms": k1_ms, "K": 1,
              "launches": wl.steps,
              "roofline": {"bound": "hbm", "achieved": hbm, "peak": pk["hbm_gbs"], "unit": "GB/s",
                           "frac": hbm / pk["hbm_gbs"],
                           "traffic": _profiled_traffic("step_batched_single_kernel", wl.name + "_K1"),
                           "kernel": "step_batched_single_kernel", "bytes_per_launch": byt,
                           "peak_basis": f"{kind} HBM copy bandwidth"}}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(wl, args, K),
        "e2e": {"value": units / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "roofline": roof,
        "single_step": single,
        "clocks": clocks,
    }
    line["config"]["tpb"] = tuned["tpb"]
    line["autotune"] = tuned
    sd_final = bptt_sub = att = None
    if not args.no_extra:
        att, att_final = measure_attitude_swarm(dev)
        sd, sd_final = measure_single_drone(dev)
        bptt_sub = bptt_subset_gradients(dev)
        line["extra"] = {"attitude_swarm": att, "single_drone": sd, "policy_bptt": measure_policy_bptt(dev),
                         "sampling": measure_sampling(dev), "mppi": measure_mppi(dev),
                         "bptt_training": measure_bptt_training(dev), "depth": measure_depth(dev),
                         "swarm_scale": measure_swarm_scale(dev)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sub)
        line["error_vs_fp64"] = mixed_error_vs_fp64(msample, final_sample)
        if att is not None:
            awl = W.attitude_swarm_rk4()
            att["cpu_baseline"] = cpu_baseline(awl, budget_s=6.0)
            att["error_vs_fp64"] = error_vs_fp64(awl, att_final)
        if sd_final is not None:
            line["extra"]["single_drone"]["error_vs_fp64"] = error_vs_fp64(W.position_hold_single(), sd_final, n_drones=1)
        if bptt_sub is not None:
            line["extra"]["policy_bptt"]["gradient_error_vs_fp64"] = gradient_error_vs_fp64(*bptt_sub)
        if "extra" in line:
            sp = line["extra"]["sampling"]
            sp["cost_error_vs_fp64"] = sampling_error_vs_fp64(*sp["_cost_sample"])
    if "extra" in line:  # GPU results kept for the CPU leg, not part of the record
        line["extra"]["sampling"].pop("_cost_sample", None)
    print(json.dumps(line), flush=True)
    return 0


def measure_mixed(dev, reps: int = 3, worlds: int = 1000, models_of: str = "mixed") -> dict:
    """The headline swarm (or its first `worlds` worlds) on its own, as fused
    launches and as single-step launches: used for profiling."""
    from paper_2606_01478_b300 import Sim, autotune
    wl = W.mixed_swarm_euler(M=worlds, models_of=models_of)
    sim = Sim.batched(np.full(wl.M, wl.N), wl.model_of_world, wl.integrator, wl.dt, ctrl=wl.ctrl,
                      max_cmd_blocks=wl.cmd.shape[0], device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0 = torch.tensor(wl.x0, dtype=torch.float32, device=dev)
    cmd = torch.tensor(wl.cmd, dtype=torch.float32, device=dev)
    sim.set_state(x0)
    sim.set_commands(cmd, wl.hold)
    tuned = autotune.tune_step(sim, wl.steps, Ks=(wl.K,), reps=1)

    def run(K):
        sim.set_state(x0)
        sim.set_commands(cmd, wl.hold)
        sim.run(wl.steps, K)
    ms = _time_ms(lambda: run(wl.K), reps, dev)
    ms1 = _time_ms(lambda: run(1), reps, dev)
    assert sim.status() == 0
    units = wl.M * wl.N * wl.steps
    return {"workload": wl.name, "value": units / (ms / 1e3), "unit": UNIT, "ms": ms, "K": wl.K,
            "tpb": tuned["tpb"], "single_step": {"value": units / (ms1 / 1e3), "ms": ms1, "K": 1}}


def measure_attitude_swarm(dev, reps: int = 5):
    """16384 worlds x 1 drone, first-principles, attitude interface, RK4 at
    500 Hz, 1000 steps as 10 chained launches of K = 100: drone-steps/s, the
    fused launch's FP32 roofline, and end to end through the C-ABI with pinned
    host buffers.  Returns the record and the final state (its error against
    the FP64 oracle is taken in the CPU leg)."""
    from paper_2606_01478_b300 import Sim, autotune
    wl = W.attitude_swarm_rk4()
    stream = torch.cuda.current_stream(dev)
    sim = Sim(wl.M, wl.N, 0, wl.integrator, wl.dt, ctrl=wl.ctrl, max_cmd_blocks=wl.cmd.shape[0],
              device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0_dev = torch.tensor(wl.x0, dtype=torch.float32, device=dev).contiguous()
    cmd_dev = torch.tensor(wl.cmd, dtype=torch.float32, device=dev).contiguous()
    x0_host = torch.tensor(wl.x0, dtype=torch.float32).pin_memory()
    cmd_host = torch.tensor(wl.cmd, dtype=torch.float32).pin_memory()
    out_host = torch.empty_like(x0_host).pin_memory()
    sim.set_state(x0_dev)
    sim.set_commands(cmd_dev, wl.hold)
    tuned = autotune.tune_step(sim, wl.steps, Ks=(wl.K,), reps=2)
    n_launch = (wl.steps + wl.K - 1) // wl.K

    def rollout():
        sim.set_state(x0_dev)
        sim.set_commands(cmd_dev, wl.hold)
        _flush_l2(dev)
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(wl.steps, wl.K)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)
    rollout()
    ms = statistics.median([rollout() for _ in range(reps)])
    e2e = []
    for _ in range(reps):
        _flush_l2(dev)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.run_host(x0_host, cmd_host, wl.hold, wl.steps, wl.K, out=out_host)
        t1.record(stream)
        t1.synchronize()
        e2e.append(t0.elapsed_time(t1))
    assert sim.status() == 0
    units = wl.M * wl.steps
    peak, _, _ = _fp32_peak()
    flop = FLOP_PER_DRONE_STEP[("fp", "rk4", "attitude")]
    achieved = flop * units / (ms / 1e3) / 1e12
    rec = {"workload": wl.name, "value": units / (ms / 1e3), "unit": UNIT, "ms_per_rollout": ms,
           "K": wl.K, "launches": n_launch, "tpb": tuned["tpb"],
           "e2e": {"value": units / (statistics.median(e2e) / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": (x0_host.numel() + cmd_host.numel()) * 4,
                   "d2h_bytes_per_step": out_host.numel() * 4},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "flop_per_drone_step": flop,
                        "traffic": _profiled_traffic("step_kernel", wl.name),
                        "kernel": "step_kernel<first-principles, RK4, attitude>",
                        "note": "16384 drones = 512 warps < 592 SM sub-partitions: latency bound"}}
    return rec, out_host.numpy().copy()


def bptt_subset_gradients(dev, M: int = 64):
    """Gradients of the BPTT recipe on M worlds (H = 250, C = 25) in both MLP
    operand modes, kept for the comparison with the FP64 oracle in the CPU leg."""
    from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
    from paper_2606_01478_b300.rollout import PolicyRollout, pack_policy
    rw = W.policy_bptt(M=M)
    out = {}
    for prec in ("hilo", "bf16"):
        sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt, device=dev)
        sim.set_params(rw.params)
        runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act, precision=prec)
        x0 = torch.tensor(rw.x0, dtype=torch.float32, device=dev)
        wb = torch.tensor(pack_policy(rw.weights), dtype=torch.float32, device=dev).to(torch.bfloat16)
        p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device=dev).contiguous()
        loss, dW, dx0 = runner.grad(x0, wb, p_ref)
        out[prec] = (float(loss.item()), dW.cpu().numpy().astype(np.float64),
                     dx0.cpu().numpy().astype(np.float64))
    return rw, out


def gradient_error_vs_fp64(rw, gpu: dict) -> dict:
    """Relative errors of the GPU loss and gradients (norm-wise over dW and over
    dx0) against the FP64 oracle's adjoint, from the float32 inputs the GPU got."""
    from oracle import policy as po
    x0 = rw.x0.astype(np.float32).astype(np.float64)
    p_ref = rw.p_ref.astype(np.float32).astype(np.float64)
    L, _, dW_ref, dx_ref = po.rollout_grad(x0, rw.weights, p_ref, rw.params, rw.dt, rw.H, rw.w_act)
    g = po.pack(dW_ref)
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return {"worlds": int(rw.M), "H": int(rw.H), "C": int(rw.C),
            **{prec: {"loss": abs(v[0] - L) / abs(L), "dW": rel(v[1], g), "dx0": rel(v[2][:, :17], dx_ref[:, :17])}
               for prec, v in gpu.items()},
            "bar": 1e-3, "reference": "FP64 oracle adjoint from the same float32 inputs"}


def measure_single_drone(dev, reps: int = 5):
    """One drone under the position controller to a hover setpoint, Euler at
    500 Hz, 1000 steps in one launch -- one thread's chain of 1000 dependent steps, so
    latency bound.  Returns the record and the final state (its error against the FP64
    oracle is taken in the CPU leg)."""
    from paper_2606_01478_b300 import Sim
    wl = W.position_hold_single()
    sim = Sim(wl.M, wl.N, int(wl.model_of_world[0]), wl.integrator, wl.dt, ctrl=wl.ctrl,
              max_cmd_blocks=wl.cmd.shape[0], device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0 = torch.tensor(wl.x0, dtype=torch.float32, device=dev)
    cmd = torch.tensor(wl.cmd, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    times = []
    for r in range(reps + 1):
        sim.set_state(x0)
        sim.set_commands(cmd, wl.hold)
        _flush_l2(dev)
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(wl.steps, wl.steps)
        e1.record(stream)
        e1.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    final = sim.get_state().cpu().numpy()
    assert sim.status() == 0
    ms = statistics.median(times)
    return {"workload": "single_1x1_fp_euler_position_1000", "ms_per_rollout": ms,
            "us_per_step": ms * 1e3 / wl.steps, "value": wl.M * wl.N * wl.steps / (ms / 1e3),
            "unit": UNIT, "launches": 1,
            "note": "one drone: one thread's dependent chain, latency bound"}, final


def measure_swarm_scale(dev, reps: int = 3) -> dict:
    """The headline's step (first-principles, RK4, attitude interface, lag rotors) on
    2^20 drones, one fused launch of K = 100 steps.  The 16384 drones of the headline
    are 512 warps, one per busy SM sub-partition, so its time is one warp's
    instruction chain; here every sub-partition holds many warps and the kernel runs
    at its issue rate: the fused step's own fraction of the FP32 peak."""
    from paper_2606_01478_b300 import CTRL_ATTITUDE, FIRST_PRINCIPLES, RK4, Sim
    from paper_2606_01478_b300 import autotune
    wl = W.attitude_swarm_rk4(M=1 << 20, steps=100, K=100)
    sim = Sim(wl.M, wl.N, FIRST_PRINCIPLES, RK4, wl.dt, ctrl=CTRL_ATTITUDE,
              max_cmd_blocks=wl.cmd.shape[0], device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0 = torch.tensor(wl.x0, dtype=torch.float32, device=dev)
    cmd = torch.tensor(wl.cmd, dtype=torch.float32, device=dev)
    sim.set_state(x0)
    sim.set_commands(cmd, wl.hold)
    tuned = autotune.tune_step(sim, wl.steps, Ks=(wl.K,), reps=1)
    stream = torch.cuda.current_stream(dev)
    times = []
    for r in range(reps + 1):
        sim.set_state(x0)
        sim.set_commands(cmd, wl.hold)
        _flush_l2(dev)
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(wl.steps, wl.K)
        e1.record(stream)
        e1.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    assert sim.status() == 0
    ms = statistics.median(times)
    units = wl.M * wl.steps
    pk, _ = peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    achieved = FLOP_PER_DRONE_STEP[("fp", "rk4", "attitude")] * units / (ms / 1e3) / 1e12
    return {"workload": wl.name, "value": units / (ms / 1e3), "unit": UNIT, "ms": ms, "K": wl.K,
            "launches": 1, "tpb": tuned["tpb"],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": _profiled_traffic("step_kernel", wl.name)}}


_FLUSH = {}


def _flush_l2(dev) -> None:
    """Write a 256 MiB buffer (twice the 126 MB L2) so the next timed run starts
    with cold caches."""
    buf = _FLUSH.get(str(dev))
    if buf is None:
        buf = _FLUSH[str(dev)] = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    buf.fill_(len(_FLUSH) & 0xFF)


def _time_ms(fn, reps: int, dev) -> float:
    """Median device time of fn() over reps runs (one untimed warm-up), the L2
    flushed before each run."""
    stream = torch.cuda.current_stream(dev)
    times = []
    for r in range(reps + 1):
        _flush_l2(dev)
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
    return statistics.median(times)


# MLP FLOPs of one policy evaluation (13 -> 64 -> 64 -> 4): 2 x 5184 multiply-adds.
MLP_FLOP = 2.0 * (13 * 64 + 64 * 64 + 64 * 4)


def measure_policy_bptt(dev, reps: int = 9) -> dict:
    """The BPTT workload (8192 drones, policy MLP in the loop, Euler at 500 Hz, H = 250,
    checkpoints every C = 25): forward rollout, forward + adjoint (BPTT), and
    plain forward stepping of the same drones without the policy."""
    from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
    from paper_2606_01478_b300.rollout import PolicyRollout, pack_policy
    rw = W.policy_bptt()
    sim = Sim(rw.M, 1, FIRST_PRINCIPLES, EULER, rw.dt, device=dev)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, rw.H, rw.C, rw.w_act)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device=dev)
    wb = torch.tensor(pack_policy(rw.weights), dtype=torch.float32, device=dev).to(torch.bfloat16)
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device=dev).contiguous()
    loss = torch.empty(1, device=dev)
    ms_fwd = _time_ms(lambda: runner.forward(x0, wb, p_ref, loss=loss), reps, dev)
    ms_grad = _time_ms(lambda: runner.grad(x0, wb, p_ref), reps, dev)
    # the plain-bf16 operand mode (precision for speed; its gradient error against
    # FP64 is measured by the tests)
    runner16 = PolicyRollout(sim, rw.H, rw.C, rw.w_act, precision="bf16")
    ms_fwd16 = _time_ms(lambda: runner16.forward(x0, wb, p_ref, loss=loss), reps, dev)
    ms_grad16 = _time_ms(lambda: runner16.grad(x0, wb, p_ref), reps, dev)
    # plain forward stepping of the same drones (attitude interface, hover commands)
    sim.set_state(x0)
    sim.set_commands(torch.zeros(1, rw.M, 4, device=dev), rw.H)
    ms_plain = _time_ms(lambda: sim.run(rw.H, rw.H), reps, dev)
    units = rw.M * rw.H
    pk, kind = peaks()
    bf16 = pk.get("bf16_tflops", 1800.0)
    # algorithmic tensor work of forward + backward: policy forward, input-adjoint
    # and weight-gradient contractions, 3 x 2 x 5184 flop per drone-step
    grad_flop = 3 * MLP_FLOP * units
    return {
        "workload": rw.name,
        "fwd": {"value": units / (ms_fwd / 1e3), "unit": UNIT, "ms": ms_fwd},
        "fwd_adjoint": {"value": units / (ms_grad / 1e3), "unit": UNIT, "ms": ms_grad,
                        "gradients_per_s": rw.M / (ms_grad / 1e3)},
        "bf16_operands": {"fwd_ms": ms_fwd16, "fwd_adjoint_ms": ms_grad16,
                          "fwd_adjoint_value": units / (ms_grad16 / 1e3), "unit": UNIT},
        "plain_forward_stepping": {"value": units / (ms_plain / 1e3), "unit": UNIT, "ms": ms_plain},
        "adjoint_over_plain": ms_grad / ms_plain,
        "roofline_fwd_adjoint": {"bound": "tensor", "achieved": grad_flop / (ms_grad / 1e3) / 1e12,
                                 "peak": bf16, "unit": "TFLOP/s",
                                 "frac": grad_flop / (ms_grad / 1e3) / 1e12 / bf16,
                                 "traffic": _profiled_traffic("rollout_bwd_kernel", rw.name),
                                 "note": "latency bound: 250 dependent steps, 128 CTAs of 64 drones; "
                                         "mma.sync bf16 with hi/lo split (2-3 MMAs per product)"},
    }


# FP32 work of one sampled RK4 step (flopcount.py): the step, the action decode
# every step, the noise's Box-Muller arithmetic and scaling, and the goal
# distance.  Obstacle terms of obstacles beyond a drone's reach (exact zeros,
# which the kernel skips) and Philox's integer rounds are not counted.
SAMPLE_FLOP_PER_STEP = float(flopcount.sampling_step()["flop"])


def measure_sampling(dev, reps: int = 3) -> dict:
    """The uneven sampling workload (512 worlds, log-uniform drone counts, 256 samples, 50 RK4
    steps): one persistent sampling launch per outer iteration, replayed from a
    CUDA graph with a fresh device seed each time; block size from the library's
    autotuner (sim_autotune, SIM_TUNE_SAMPLE)."""
    from paper_2606_01478_b300 import RK4, Sim
    wl = W.uneven_sampling_rk4()
    n = len(wl.x0)
    sim = Sim.batched(wl.n_per_world, np.zeros(wl.M, np.int32), RK4, wl.dt, device=dev)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device=dev))
    goals = torch.tensor(wl.goals, dtype=torch.float32, device=dev)
    seed = torch.tensor([wl.seed], dtype=torch.int64, device=dev)
    cost = torch.empty(n, wl.S, device=dev)
    from paper_2606_01478_b300 import autotune
    tuned = autotune.tune_sample(sim, wl.S, wl.H, seed, wl.sigma, goals, wl.obstacles, wl.w_obs, cost,
                                 tpbs=(64, 128, 256), reps=1)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream(dev)
    st.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            sim.sample_rollouts(wl.S, wl.H, seed, wl.sigma, goals, wl.obstacles, wl.w_obs,
                                cost=cost, stream=st)
    torch.cuda.current_stream(dev).wait_stream(st)

    def replay():
        seed.add_(1)
        g.replay()
    ms = _time_ms(replay, reps, dev)
    rng = np.random.default_rng(5)
    drones, samples = rng.integers(0, n, 64), rng.integers(0, wl.S, 64)
    cost_sample = (drones, samples, int(seed.item()),
                   cost[torch.as_tensor(drones, device=dev), torch.as_tensor(samples, device=dev)].cpu().numpy())
    units = n * wl.S * wl.H
    pk, _ = peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    achieved = SAMPLE_FLOP_PER_STEP * units / (ms / 1e3) / 1e12
    return {"workload": wl.name, "drones": n, "samples_per_drone": wl.S, "horizon": wl.H,
            "value": units / (ms / 1e3), "unit": UNIT, "ms_per_outer_iteration": ms,
            "rollouts_per_s": n * wl.S / (ms / 1e3), "tpb": tuned["tpb"],
            "autotune": {k: v for k, v in tuned.items() if k != "table"}, "_cost_sample": cost_sample,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": _profiled_traffic("sample_kernel", wl.name),
                         "flop_per_sample_step": SAMPLE_FLOP_PER_STEP}}


def _mppi_run(dev, wl, reps: int) -> dict:
    """Time MPPI iterations (sampling launch + update launch) of one workload."""
    from paper_2606_01478_b300 import RK4, Sim
    n = len(wl.x0)
    c = wl.cfg
    sim = Sim.batched(wl.n_per_world, np.zeros(len(wl.n_per_world), np.int32), RK4, wl.dt, device=dev)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device=dev))
    goals = torch.tensor(wl.goals, dtype=torch.float32, device=dev)
    seed = torch.tensor([wl.seed], dtype=torch.int64, device=dev)
    mean = torch.zeros(n, c["n_ctrl"], c["H"], 4, device=dev)
    plan = torch.empty(n, c["H"], 4, device=dev)
    cost = torch.empty(n, c["S"], device=dev)
    best = torch.empty(n, device=dev)

    def it():
        seed.add_(1)
        sim.mppi_iteration(c, seed, goals, wl.obstacles, mean, plan=plan, cost=cost, best_cost=best)
    ms = _time_ms(it, reps, dev)
    units = n * c["S"] * c["H"]
    return {"workload": wl.name, "ms_per_iteration": ms, "iterations_per_s": 1e3 / ms,
            "value": units / (ms / 1e3), "unit": UNIT, "trajectories_per_iteration": n * c["S"],
            "controllers": c["n_ctrl"], "elites_per_controller": c["n_elite"],
            "best_cost_mean": float(best.mean().item())}


def measure_mppi(dev, reps: int = 3) -> dict:
    """MPPI / iCEM control.  The paper's configuration: one drone, 500k sampled
    trajectories per control step in five independent controllers of 100 000,
    each keeping its top 1 % (1000 elites), a 25-step horizon at 50 Hz, RK4;
    one iteration = sampling launch + update launch (cluster path).  Beside it,
    64 drones x 8000 samples (the same 512k trajectories spread over drones;
    warp-path update)."""
    out = _mppi_run(dev, W.mppi_workload(n_drones=1, S=500_000), reps)
    out["paper_context"] = ("500k samples x 25 steps at 50 Hz, > 5e8 steps/s on an unnamed GPU; "
                            "a 50 Hz control loop leaves 20 ms per iteration")
    out["multi_drone"] = _mppi_run(dev, W.mppi_workload(), reps)
    return out


def measure_bptt_training(dev, reps: int = 3) -> dict:
    """The paper's BPTT tracking setup (16 environments, 40 steps per rollout,
    learning rate 4.6e-2, 100 000 timesteps = 156 iterations, its tracking
    reward and weights) with the policy at the recommended 50 Hz of the
    attitude interface (each action held for 10 physics steps at 500 Hz): each
    iteration is the rollout gradient (forward + adjoint kernels) and the Adam
    kernel; one iteration is captured in a CUDA graph and replayed 156 times."""
    from paper_2606_01478_b300 import EULER, FIRST_PRINCIPLES, Sim
    from paper_2606_01478_b300.rollout import TRACKING_REWARD, PolicyRollout, pack_policy
    from paper_2606_01478_b300.train import PolicyTrainer
    M, H, C, R, iters, lr = 16, 40, 10, 10, 156, 4.6e-2
    rw = W.policy_bptt(M=M, H=H, C=C, repeat=R)
    sim = Sim(M, 1, FIRST_PRINCIPLES, EULER, rw.dt, device=dev)
    sim.set_params(rw.params)
    runner = PolicyRollout(sim, H, C, rw.w_act, reward=TRACKING_REWARD, action_repeat=R)
    w0 = torch.tensor(pack_policy(rw.weights), dtype=torch.float32, device=dev)
    x0 = torch.tensor(rw.x0, dtype=torch.float32, device=dev)
    p_ref = torch.tensor(rw.p_ref, dtype=torch.float32, device=dev).contiguous()
    first = PolicyTrainer(runner, w0, lr)
    initial_loss = first.iteration(x0, p_ref).item()
    times, final_loss = [], None
    for r in range(reps + 1):
        trainer = PolicyTrainer(runner, w0, lr)
        g = trainer.capture(x0, p_ref)
        _flush_l2(dev)
        torch.cuda._sleep(1_000_000)
        stream = torch.cuda.current_stream(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(iters):
            g.replay()
        e1.record(stream)
        e1.synchronize()
        if r:
            times.append(e0.elapsed_time(e1))
        final_loss = trainer.loss.item()
    ms = statistics.median(times)
    return {"workload": f"bptt_train_{M}envs_H{H}_R{R}_{iters}iters_lr{lr}_tracking_reward", "ms_total": ms,
            "ms_per_iteration": ms / iters, "iterations": iters,
            "timesteps": M * H * iters, "physics_steps": M * H * R * iters,
            "mean_reward_per_step_first_iteration": -initial_loss / H,
            "mean_reward_per_step_last_iteration": -final_loss / H,
            "paper_context": "1.56 s to train the 10 s Lissajous tracker (100k timesteps) on a CPU"}


def measure_depth(dev, reps: int = 3) -> dict:
    """Depth images at the paper's scale (64 x 64 rays, 1024 environments, one
    camera per drone): the sampling workload's 32 obstacles as spheres plus 8 boxes and the
    ground; frames per second of one batched launch."""
    import math
    from paper_2606_01478_b300 import RK4, Sim
    rng = np.random.default_rng(1006)
    n = 1024
    wl4 = W.uneven_sampling_rk4(M=8)
    P = W.crazyflie_params()
    x = np.zeros((n, 20))
    x[:, 0:3] = rng.uniform([-1.5, -1.5, 0.5], [1.5, 1.5, 3.5], (n, 3))
    x[:, 3:7] = W.quat_from_rpy(rng.uniform([-0.3, -0.3, -np.pi], [0.3, 0.3, np.pi], (n, 3)))
    x[:, 13:17] = W.hover_rpm(P)
    sim = Sim(n, 1, 0, RK4, 1 / 500, device=dev)
    sim.set_params(P)
    sim.set_state(torch.tensor(x, dtype=torch.float32, device=dev))
    lo = rng.uniform([-3, -3, 0], [2, 2, 1.5], (8, 3))
    boxes = np.concatenate([lo, lo + rng.uniform(0.3, 1.0, (8, 3))], 1)
    out = torch.empty(n, 64, 64, device=dev)
    ms = _time_ms(lambda: sim.render_depth(64, 64, math.radians(90), math.radians(90), 10.0,
                                           wl4.obstacles, boxes, out=out), reps, dev)
    return {"workload": "depth_1024x64x64_32spheres_8boxes", "ms_per_batch": ms,
            "frames_per_s": n / (ms / 1e3), "rays_per_s": n * 64 * 64 / (ms / 1e3),
            "paper_context": "350k frames/s at 64x64 across 1024 environments (MJX ray casting)"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--tpb", type=int, default=0, help="threads per block (0 = library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the measurements beside the headline")
    ap.add_argument("--worlds", type=int, default=1000, help="worlds of --only mixed")
    ap.add_argument("--models", default="mixed", choices=["mixed", "fp", "abs"],
                    help="--only mixed: every world first-principles (fp), abstracted (abs) or alternating")
    ap.add_argument("--only", choices=["mixed", "attitude", "bptt", "sampling", "mppi", "training", "depth",
                                       "scale"],
                    default=None,
                    help="run one extra workload alone and print its record (for profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        fn = {"mixed": lambda d, reps: measure_mixed(d, reps, args.worlds, args.models),
              "attitude": lambda d, reps: measure_attitude_swarm(d, reps)[0],
              "bptt": measure_policy_bptt, "sampling": measure_sampling,
              "mppi": measure_mppi, "training": measure_bptt_training, "depth": measure_depth,
              "scale": measure_swarm_scale}[args.only]
        rec = fn(dev, reps=args.steps)
        rec = {k: v for k, v in rec.items() if not k.startswith("_")}  # GPU data kept for the CPU leg
        print(json.dumps({"only": args.only, "record": rec}), flush=True)
        return 0
    rank = int(os.environ.get("RANK", "0"))
    wl = W.mixed_swarm_euler(seed=1002 + 7919 * rank)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_b300(args, wl)


if __name__ == "__main__":
    sys.exit(main())
