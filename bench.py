"""Benchmark of the B300 drone physics step (one JSON line on stdout).

Default workload (the headline configuration): 16384 worlds x 1 drone,
first-principles model, attitude interface, RK4 at dt = 1/500 s, 1000 steps
fused as launches of K = 100.  One benchmark "step" is that whole rollout
(10 launches).  The metric is drone-steps per second.

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

import workloads as W  # noqa: E402

METRIC = "drone-steps/s (fwd, fused RK4, first-principles + attitude controller)"
UNIT = "drone-steps/s"
# FP32 arithmetic of one RK4 drone-step of the first-principles model under the
# attitude interface (FMA = 2 flop), counted term by term from the kernel's
# formulation: controller 93 + 4 derivatives x 78 + RK4 combination 221 +
# quaternion renormalisation 11 = 637 (command decode, amortised over 50-step
# holds, adds ~1.2).
FLOP_PER_DRONE_STEP = {("fp", "rk4", "attitude"): 637.0, ("fp", "euler", "attitude"): 216.0,
                       ("abs", "euler", "attitude"): 58.0}
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
    "sample_kernel": ("sample.cu", "stepcore.cuh", "physics.cuh", "common.cuh"),
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


def cpu_baseline(wl, budget_s: float = 12.0) -> dict:
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: all worlds, as many steps as fit about budget_s seconds."""
    dt1, _ = oracle_sample(wl, wl.M, 2)
    steps = int(max(4, min(wl.steps, budget_s / max(dt1 / 2, 1e-6))))
    secs, units = oracle_sample(wl, wl.M, steps)
    return {"value": units / secs, "unit": UNIT, "cores": torch.get_num_threads(),
            "cpu": _cpu_model(), "kind": "oracle",
            "sample": f"{wl.M} drones x {steps} of {wl.steps} steps (FP64 torch CPU oracle)"}


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


def mixed_error_vs_fp64(sample, gpu_rows) -> dict:
    """Final-state error of the mixed swarm's 200 steps against the FP64 oracle on 64
    sampled drones of each model, from the float32 inputs the GPU received (part of
    the CPU-baseline leg)."""
    import dataclasses
    from oracle import physics as ph
    wl = W.mixed_swarm_euler()
    f32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    wl32 = dataclasses.replace(wl, x0=f32(wl.x0), cmd=f32(wl.cmd))
    ref = ph.rollout_workload(wl32, drones=sample).numpy()
    err = np.abs(np.asarray(gpu_rows, np.float64) - ref)
    models = wl.model_of_world[np.asarray(sample) // wl.N]
    out = {"drones_per_model": 64, "steps": int(wl.steps),
           "reference": "FP64 oracle from the same float32 inputs"}
    for m, name, fields in ((0, "first_principles", STATE_FIELDS), (1, "abstracted", ABS_FIELDS)):
        e = err[models == m]
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


def run_reference(args, wl):
    dist, rank, ws = _dist()
    if rank != 0:
        return 0
    n_steps = 20
    for _ in range(args.warmup):
        oracle_sample(wl, wl.M, n_steps)
    secs, units = 0.0, 0
    for _ in range(args.steps):
        s, u = oracle_sample(wl, wl.M, n_steps)
        secs += s
        units += u
    value = units / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _config(wl, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(),
                         "cpu": _cpu_model(), "kind": "oracle",
                         "sample": f"{wl.M} drones x {n_steps} of {wl.steps} steps per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _config(wl, args):
    return {"workload": wl.name, "worlds": wl.M, "drones_per_world": wl.N,
            "model": "first-principles", "integrator": "rk4", "control": "attitude",
            "dt": wl.dt, "steps_per_rollout": wl.steps, "K_fused": wl.K,
            "parallelism": f"replicas x{args.gpus} (independent worlds)",
            "l2": "flushed (256 MiB write) before every timed iteration"}


# --------------------------------------------------------------------------- B300 arm


def run_b300(args, wl):
    from paper_2606_01478_b300 import Sim
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    sim = Sim(wl.M, wl.N, 0, wl.integrator, wl.dt, ctrl=wl.ctrl, max_cmd_blocks=wl.cmd.shape[0],
              device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0_dev = torch.tensor(wl.x0, dtype=torch.float32, device=dev).contiguous()
    cmd_dev = torch.tensor(wl.cmd, dtype=torch.float32, device=dev).contiguous()
    x0_host = torch.tensor(wl.x0, dtype=torch.float32).pin_memory()
    cmd_host = torch.tensor(wl.cmd, dtype=torch.float32).pin_memory()
    out_host = torch.empty_like(x0_host).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sim.set_state(x0_dev)
    sim.set_commands(cmd_dev, wl.hold)
    if args.tpb:
        sim.set_block_size(args.tpb)
        tuned = {"tpb": args.tpb, "K": wl.K, "source": "--tpb"}
    else:
        from paper_2606_01478_b300 import autotune
        tuned = autotune.tune_step(sim, wl.steps, tag="attitude_swarm", Ks=(wl.K,), reps=2)
        tuned = {k: v for k, v in tuned.items() if k != "table"}
    n_launch = (wl.steps + wl.K - 1) // wl.K

    def one_rollout(events):
        for j in range(n_launch):
            k = min(wl.K, wl.steps - j * wl.K)
            if events is not None:
                events[j][0].record(stream)
            sim.step(k)
            if events is not None:
                events[j][1].record(stream)

    def reset():
        sim.set_state(x0_dev)
        sim.set_commands(cmd_dev, wl.hold)

    for _ in range(args.warmup):
        reset()
        one_rollout(None)
    torch.cuda.synchronize()
    assert sim.status() == 0, "non-finite state during warm-up"

    # device-resident timing (inputs already in HBM): two events per rollout
    launches0 = sim.launches
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    _barrier(dist)
    torch.cuda.synchronize()
    per_iter_ms = []
    for it in range(args.steps):
        reset()
        flush.fill_(it & 0xFF)
        # keep the device busy while the host enqueues the rollout, so the
        # events time device execution and not host launch latency
        torch.cuda._sleep(1_000_000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_rollout(None)
        e1.record(stream)
        torch.cuda.synchronize()
        per_iter_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    _barrier(dist)
    clocks = sampler.stop()
    # the set_state launch of each reset is not part of the timed region
    gpu_launches = sim.launches - launches0 - args.steps * 1
    # per-launch durations of the step kernel (for the roofline), in a separate pass
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_launch)]
    launch_ms = []
    for it in range(args.steps):
        reset()
        flush.fill_(it & 0xFF)
        torch.cuda._sleep(1_000_000)
        one_rollout(ev)
        torch.cuda.synchronize()
        launch_ms += [e[0].elapsed_time(e[1]) for e in ev]
    total_ms = _max_over_ranks(dist, sum(per_iter_ms))
    units = wl.M * wl.steps * args.steps * ws
    value = units / (total_ms / 1e3)

    # end to end through the C-ABI with host buffers
    e2e_ms = []
    for it in range(args.steps):
        flush.fill_(it & 0xFF)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        sim.run_host(x0_host, cmd_host, wl.hold, wl.steps, wl.K, out=out_host)
        t1.record(stream)
        t1.synchronize()
        e2e_ms.append(t0.elapsed_time(t1))
    e2e_total = _max_over_ranks(dist, sum(e2e_ms))
    assert sim.status() == 0
    h2d = x0_host.numel() * 4 + cmd_host.numel() * 4
    d2h = out_host.numel() * 4

    if rank != 0:
        return 0
    pk, pk_kind = peaks()
    clk_max = pk.get("sm_max_mhz", 2032.0)
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * clk_max * 1e6 / 1e12
    flop = FLOP_PER_DRONE_STEP[("fp", "rk4", "attitude")]
    # average launch duration over the timed region: the rollout's launches run
    # back to back on one stream (chained, each scheduled while the previous one
    # drains), so rollout time / launches; the separate pass above times each
    # launch between its own events, which serialises the chain
    avg_launch_s = total_ms / (args.steps * n_launch) / 1e3
    achieved = flop * wl.M * wl.K / avg_launch_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "traffic": _profiled_traffic("step_kernel", wl.name),
            "kernel": "step_kernel<first-principles, RK4, attitude>",
            "flop_per_drone_step": flop,
            "launch_ms_timed_region": avg_launch_s * 1e3,
            "peak_basis": f"FP32 FMA: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x "
                          f"{clk_max:.0f} MHz (max SM clock, {pk_kind} peaks file)"}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (fp32_peak * clocks["sm_mhz"] / clk_max)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(wl, args),
        "e2e": {"value": units / (e2e_total / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": gpu_launches,
        "launch_ms": {"mean": statistics.mean(launch_ms), "min": min(launch_ms),
                      "max": max(launch_ms), "count": len(launch_ms)},
        "roofline": roof,
        "clocks": clocks,
    }
    line["config"]["tpb"] = tuned["tpb"]
    line["autotune"] = tuned
    sd_final = bptt_sub = None
    if not args.no_extra:
        sd, sd_final = measure_single_drone(dev)
        bptt_sub = bptt_subset_gradients(dev)
        line["extra"] = {"single_drone": sd, "mixed_swarm": measure_mixed_swarm(dev), "policy_bptt": measure_policy_bptt(dev),
                         "sampling": measure_sampling(dev), "mppi": measure_mppi(dev),
                         "bptt_training": measure_bptt_training(dev), "depth": measure_depth(dev),
                         "swarm_scale": measure_swarm_scale(dev)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
        line["error_vs_fp64"] = error_vs_fp64(wl, out_host.numpy())
        if sd_final is not None:
            line["extra"]["single_drone"]["error_vs_fp64"] = error_vs_fp64(W.position_hold_single(), sd_final, n_drones=1)
        if bptt_sub is not None:
            line["extra"]["policy_bptt"]["gradient_error_vs_fp64"] = gradient_error_vs_fp64(*bptt_sub)
        if "extra" in line:
            mx, sp = line["extra"]["mixed_swarm"], line["extra"]["sampling"]
            mx["error_vs_fp64"] = mixed_error_vs_fp64(*mx["_final_sample"])
            sp["cost_error_vs_fp64"] = sampling_error_vs_fp64(*sp["_cost_sample"])
    if "extra" in line:  # GPU results kept for the CPU leg, not part of the record
        line["extra"]["mixed_swarm"].pop("_final_sample", None)
        line["extra"]["sampling"].pop("_cost_sample", None)
    print(json.dumps(line), flush=True)
    return 0


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


def measure_mixed_swarm(dev, reps: int = 3) -> dict:
    """The mixed swarm (1000 worlds x 4000 drones, 50/50 first-principles / abstracted,
    Euler, 200 steps) in both modes: one fused launch of K = 200 (FP32-issue
    bound) and 200 launches of K = 1 (HBM bound)."""
    from paper_2606_01478_b300 import Sim
    from paper_2606_01478_b300 import autotune
    wl = W.mixed_swarm_euler()
    n = wl.M * wl.N
    sim = Sim.batched(np.full(wl.M, wl.N), wl.model_of_world, wl.integrator, wl.dt, ctrl=wl.ctrl,
                      max_cmd_blocks=wl.cmd.shape[0], device=dev)
    sim.set_params(wl.params, wl.param_set_of_world)
    x0 = torch.tensor(wl.x0, dtype=torch.float32, device=dev)
    cmd = torch.tensor(wl.cmd, dtype=torch.float32, device=dev)
    del wl.x0, wl.cmd
    sim.set_state(x0)
    sim.set_commands(cmd, wl.hold)
    tuned = autotune.tune_step(sim, wl.steps, tag="mixed_swarm", Ks=(1, 200), reps=1)
    stream = torch.cuda.current_stream(dev)
    n_fp = n // 2
    n_abs = n - n_fp
    out = {}
    for K in (wl.steps, 1):
        times = []
        for r in range(reps + 1):
            sim.set_state(x0)
            sim.set_commands(cmd, wl.hold)
            _flush_l2(dev)
            torch.cuda._sleep(1_000_000)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.run(wl.steps, K)
            e1.record(stream)
            e1.synchronize()
            if r:
                times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        units = n * wl.steps
        rec = {"value": units / (ms / 1e3), "unit": UNIT, "ms": ms, "K": K,
               "launches": (wl.steps + K - 1) // K, "tpb": tuned["tpb"]}
        if K == 1:
            byt = n_fp * BYTES_PER_DRONE_STEP["fp"] + n_abs * BYTES_PER_DRONE_STEP["abs"]
            pk, kind = peaks()
            achieved = byt * wl.steps / (ms / 1e3) / 1e9
            rec["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                               "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                               "traffic": _profiled_traffic("step_batched_single_kernel", wl.name + "_K1"),
                               "bytes_per_launch": byt,
                               "peak_basis": f"{kind} HBM copy bandwidth"}
        else:
            flop = (n_fp * FLOP_PER_DRONE_STEP[("fp", "euler", "attitude")]
                    + n_abs * FLOP_PER_DRONE_STEP[("abs", "euler", "attitude")])
            pk, kind = peaks()
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
            achieved = flop * wl.steps / (ms / 1e3) / 1e12
            rec["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak,
                               "unit": "TFLOP/s", "frac": achieved / peak,
                               "traffic": _profiled_traffic("step_batched_kernel", wl.name),
                               "note": "abstracted drones also issue 6 MUFU sin/cos per step"}
        out[f"fused_K{K}" if K > 1 else "single_step_K1"] = rec
    assert sim.status() == 0
    # 64 drones of each model, for the FP64 comparison of the CPU leg (the state
    # after the last run: 200 steps from x0)
    rng = np.random.default_rng(2)
    models = wl.model_of_world[np.arange(n) // wl.N]
    sample = np.concatenate([rng.choice(np.nonzero(models == m)[0], 64, replace=False) for m in (0, 1)])
    out["_final_sample"] = (sample, sim.get_state()[torch.as_tensor(sample, device=dev)].cpu().numpy())
    out["workload"] = "swarm_1000x4000_mixed_euler_attitude_200"
    out["autotune"] = {k: v for k, v in tuned.items() if k != "table"}
    return out


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
    tuned = autotune.tune_step(sim, wl.steps, tag="swarm_scale", Ks=(wl.K,), reps=1)
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


def measure_policy_bptt(dev, reps: int = 3) -> dict:
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


# FP32 work of one sampled RK4 step: the step (637), the per-step attitude
# decode (25), noise scaling and Box-Muller (15) and the goal distance (10).
# Obstacle tests are not counted: the kernel drops obstacles outside a drone's
# reach bound (exact zeros), leaving almost none; Philox integer work and MUFU
# calls are not counted either.  ncu measures 773 executed flop per sample-step.
SAMPLE_FLOP_PER_STEP = 637.0 + 25.0 + 15.0 + 10.0


def measure_sampling(dev, reps: int = 3) -> dict:
    """The uneven sampling workload (512 worlds, log-uniform drone counts, 256 samples, 50 RK4
    steps): one persistent sampling launch per outer iteration, replayed from a
    CUDA graph with a fresh device seed each time; block size autotuned."""
    from paper_2606_01478_b300 import RK4, Sim
    wl = W.uneven_sampling_rk4()
    n = len(wl.x0)
    sim = Sim.batched(wl.n_per_world, np.zeros(wl.M, np.int32), RK4, wl.dt, device=dev)
    sim.set_params(wl.params)
    sim.set_state(torch.tensor(wl.x0, dtype=torch.float32, device=dev))
    goals = torch.tensor(wl.goals, dtype=torch.float32, device=dev)
    seed = torch.tensor([wl.seed], dtype=torch.int64, device=dev)
    cost = torch.empty(n, wl.S, device=dev)
    best = None
    for tpb in (64, 128, 256):
        sim.set_block_size(tpb)
        ms = _time_ms(lambda: sim.sample_rollouts(wl.S, wl.H, seed, wl.sigma, goals, wl.obstacles,
                                                  wl.w_obs, cost=cost), 1, dev)
        if best is None or ms < best[1]:
            best = (tpb, ms)
    sim.set_block_size(best[0])
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
            "rollouts_per_s": n * wl.S / (ms / 1e3), "tpb": best[0], "_cost_sample": cost_sample,
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
    ap.add_argument("--only", choices=["mixed", "bptt", "sampling", "mppi", "training", "depth", "scale"],
                    default=None,
                    help="run one extra workload alone and print its record (for profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only:
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        fn = {"mixed": measure_mixed_swarm, "bptt": measure_policy_bptt, "sampling": measure_sampling,
              "mppi": measure_mppi, "training": measure_bptt_training, "depth": measure_depth,
              "scale": measure_swarm_scale}[args.only]
        print(json.dumps({"only": args.only, "record": fn(dev, reps=args.steps)}), flush=True)
        return 0
    rank = int(os.environ.get("RANK", "0"))
    wl = W.attitude_swarm_rk4(seed=1001 + 7919 * rank)
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_b300(args, wl)


if __name__ == "__main__":
    sys.exit(main())
