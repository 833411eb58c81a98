"""Seeded synthetic inputs for the batched drone physics step.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle.  It
holds input recipes only (platform parameters, initial states, command
schedules, policy weights, obstacle scenes) and none of the method's
arithmetic: no dynamics, controller, integrator, loss or cost is computed here.

Every generator takes an explicit seed (numpy ``default_rng``) and returns
plain numpy arrays in float64; the CUDA side converts them to float32 when it
uploads them, the oracle uses them as they are.

State vector (per drone, 20 numbers, the paper's x = [p, q, v, omega, Omega]
of the first-principles model plus 3 controller integrator states):

    first-principles: p(3) q(4, scalar-last x,y,z,w) v(3) omega(3, body) Omega(4, RPM) I(3)
    abstracted:       p(3) Psi(3, roll,pitch,yaw)   v(3) Psidot(3) f_sigma(1)   (7 unused = 0)

Commands (per drone, 4 numbers):
    attitude interface: a in [-1, 1]^4 = (roll, pitch, yaw, thrust), normalised
    position interface: (x, y, z, yaw) setpoint
    rotor-speed interface: Omega_cmd (RPM) per rotor
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.spatial.transform import Rotation

STATE_DIM = 20
CMD_DIM = 4
G = 9.81

# Names of the per-platform parameters, in the order of the packed float vector
# declared in include/crazyflow.h (SIM_P_*).  Values are SI units except rotor
# speeds, which are in RPM (kf in N/RPM^2, km in N*m/RPM^2).
PARAM_NAMES = (
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
NPARAMS = 48  # packed length


def crazyflie_params(**overrides) -> dict:
    """Crazyflie 2.x platform: mass 0.027 kg, J = diag(1.4e-5, 1.4e-5, 2.17e-5),
    arm 0.046 m, kf 3.16e-10 N/RPM^2, km 7.94e-12 N*m/RPM^2, first-order motor
    lag with time constant 0.03 s (the four-coefficient rotor model with
    cv_up = cv_down = 1/0.03 and cd_up = cd_down = 0).

    omega_max: per-rotor speed limit giving a total thrust-to-weight of 1.9.
    Gains and the action scaling are readings adopted here (the paper prints none).
    Abstracted-model coefficients: roll/pitch omega_n = 15 rad/s, zeta = 0.7;
    yaw omega_n = 6 rad/s, zeta = 1; c_tau = 1/0.03; c_f = 1.
    Rotor inertia J_p (kg m^2) and the non-quadratic coefficients of the thrust
    (kf0 N, kf1 N/RPM) and drag-torque (km1 N m/RPM) curves default to 0.
    """
    m, kf = 0.027, 3.16e-10
    p = dict(
        mass=m, Jx=1.4e-5, Jy=1.4e-5, Jz=2.17e-5, arm=0.046, kf=kf, km=7.94e-12,
        cv_up=1.0 / 0.03, cd_up=0.0, cv_down=1.0 / 0.03, cd_down=0.0,
        omega_max=math.sqrt(1.9 * m * G / (4.0 * kf)),
        Ca_x=0.0, Ca_y=0.0, Ca_z=0.0,
        KR_x=100.0, KR_y=100.0, KR_z=40.0, Kw_x=20.0, Kw_y=20.0, Kw_z=12.0,
        Kp_x=4.0, Kp_y=4.0, Kp_z=6.0, Kd_x=3.0, Kd_y=3.0, Kd_z=4.0,
        Ki_x=0.5, Ki_y=0.5, Ki_z=1.0,
        max_angle=math.pi / 6.0, thrust_scale=0.45, g=G,
        c1_r=-225.0, c1_p=-225.0, c1_y=-36.0,
        c2_r=-21.0, c2_p=-21.0, c2_y=-12.0,
        c3_r=225.0, c3_p=225.0, c3_y=36.0,
        c_tau=1.0 / 0.03, c_f=1.0,
        J_p=0.0, kf0=0.0, kf1=0.0, km1=0.0,
    )
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = float(v)
    return p


def hover_rpm(p: dict) -> float:
    """Rotor speed at which the four rotors carry the weight (initial condition)."""
    return math.sqrt(p["mass"] * p["g"] / (4.0 * p["kf"]))


def quat_from_rpy(rpy: np.ndarray) -> np.ndarray:
    """Scalar-last quaternions [x,y,z,w] for R = Rz(yaw) Ry(pitch) Rx(roll)."""
    rpy = np.asarray(rpy, dtype=np.float64).reshape(-1, 3)
    return Rotation.from_euler("ZYX", rpy[:, ::-1]).as_quat()


def fp_state(p_pos, rpy, vel, omega, rotor, integ=None) -> np.ndarray:
    """Pack first-principles states [n, 20] from components."""
    n = len(p_pos)
    x = np.zeros((n, STATE_DIM), dtype=np.float64)
    x[:, 0:3] = p_pos
    x[:, 3:7] = quat_from_rpy(rpy)
    x[:, 7:10] = vel
    x[:, 10:13] = omega
    x[:, 13:17] = rotor
    if integ is not None:
        x[:, 17:20] = integ
    return x


def abs_state(p_pos, rpy, vel, rpy_rate, f_sigma) -> np.ndarray:
    """Pack abstracted-model states [n, 20] (last 7 entries unused, zero)."""
    n = len(p_pos)
    x = np.zeros((n, STATE_DIM), dtype=np.float64)
    x[:, 0:3] = p_pos
    x[:, 3:6] = rpy
    x[:, 6:9] = vel
    x[:, 9:12] = rpy_rate
    x[:, 12] = f_sigma
    return x


@dataclass
class Workload:
    """One synthetic workload: everything both sides need to run it."""
    name: str
    M: int
    N: int                      # drones per world (uniform worlds)
    model: int                  # 0 first-principles, 1 abstracted, -1 mixed per world
    integrator: int             # 0 Euler, 1 RK4
    ctrl: int                   # 0 rotor speed, 1 attitude, 2 position
    dt: float
    steps: int
    K: int                      # steps fused per launch
    hold: int                   # steps each command block is held
    params: list                # list of param dicts (one per param set)
    param_set_of_world: np.ndarray  # [M] int32
    model_of_world: np.ndarray      # [M] int32
    x0: np.ndarray              # [M*N, 20]
    cmd: np.ndarray             # [n_blocks, M*N, 4]


# ---------------------------------------------------------------------------
# The five workloads.  Seeds are 1000 + config index.


def position_hold_single(seed: int = 1000) -> Workload:
    """1 world x 1 drone, first-principles, position PID to a hover setpoint at
    (0, 0, 1); hover at z = 1 m plus U(+-0.1 m) position, U(+-10 deg) attitude
    per roll/pitch/yaw axis and U(+-1 rad/s) body rates; Euler, dt = 1/500 s,
    1000 steps (fused in one launch)."""
    rng = np.random.default_rng(seed)
    P = crazyflie_params()
    pos = np.array([[0.0, 0.0, 1.0]]) + rng.uniform(-0.1, 0.1, (1, 3))
    rpy = rng.uniform(-np.deg2rad(10), np.deg2rad(10), (1, 3))
    w = rng.uniform(-1.0, 1.0, (1, 3))
    x0 = fp_state(pos, rpy, np.zeros((1, 3)), w, np.full((1, 4), hover_rpm(P)))
    cmd = np.array([[[0.0, 0.0, 1.0, 0.0]]])
    return Workload("single_1x1_fp_euler_position_1000", 1, 1, 0, 0, 2, 1.0 / 500, 1000, 1000,
                    1000, [P], np.zeros(1, np.int32), np.zeros(1, np.int32), x0, cmd)


def _attitude_commands(rng, n_blocks, n, lo=-0.5, hi=0.5):
    return rng.uniform(lo, hi, (n_blocks, n, 4))


def attitude_swarm_rk4(seed: int = 1001, M: int = 16384, steps: int = 1000, K: int = 100) -> Workload:
    """16384 worlds x 1 drone, first-principles, attitude interface, RK4 at
    dt = 1/500 s, 1000 steps as launches of K = 100 fused steps.  Initial state:
    position U(+-1 m) around (0,0,1), roll/pitch/yaw U(+-30 deg), velocity
    U(+-1 m/s), body rates U(+-2 rad/s), rotors at hover speed.  Commands:
    a ~ U[-0.5, 0.5]^4 per world, each held for 50 steps."""
    rng = np.random.default_rng(seed)
    P = crazyflie_params()
    n = M
    pos = np.array([0.0, 0.0, 1.0]) + rng.uniform(-1, 1, (n, 3))
    rpy = rng.uniform(-np.deg2rad(30), np.deg2rad(30), (n, 3))
    vel = rng.uniform(-1, 1, (n, 3))
    w = rng.uniform(-2, 2, (n, 3))
    x0 = fp_state(pos, rpy, vel, w, np.full((n, 4), hover_rpm(P)))
    hold = 50
    cmd = _attitude_commands(rng, (steps + hold - 1) // hold, n)
    return Workload(f"swarm_{M}x1_fp_rk4_attitude_{steps}", M, 1, 0, 1, 1, 1.0 / 500, steps, K,
                    hold, [P], np.zeros(M, np.int32), np.zeros(M, np.int32), x0, cmd)


def mixed_swarm_euler(seed: int = 1002, M: int = 1000, N: int = 4000, steps: int = 200, K: int = 200,
                      models_of: str = "mixed") -> Workload:
    """M worlds x N drones (default 1000 x 4000 = 4M), even worlds
    first-principles, odd worlds abstracted with each abstracted coefficient
    scaled by U(0.9, 1.1) per world; attitude interface; Euler at dt = 1/500 s,
    200 steps.  Initial states as in attitude_swarm_rk4 (abstracted: Psi from the same
    roll/pitch/yaw draw, Psidot = 0, f_sigma = m g); per-drone attitude
    commands U[-0.5, 0.5]^4 held for 50 steps.  models_of = "fp" or "abs"
    makes every world first-principles or abstracted instead (the same draws)."""
    rng = np.random.default_rng(seed)
    base = crazyflie_params()
    params, models = [], np.zeros(M, np.int32)
    for w in range(M):
        first = (w % 2 == 0) if models_of == "mixed" else models_of == "fp"
        if models_of == "abs" or not first:
            coeff = {k: rng.uniform(0.9, 1.1) for k in ("c1_r", "c1_p", "c1_y", "c2_r", "c2_p", "c2_y",
                                                          "c3_r", "c3_p", "c3_y", "c_tau", "c_f")}
        if first:
            params.append(dict(base))
        else:
            models[w] = 1
            q = dict(base)
            for k, f in coeff.items():
                q[k] = base[k] * f
            params.append(q)
    n = M * N
    pos = np.array([0.0, 0.0, 1.0]) + rng.uniform(-1, 1, (n, 3))
    rpy = rng.uniform(-np.deg2rad(30), np.deg2rad(30), (n, 3))
    vel = rng.uniform(-1, 1, (n, 3))
    w = rng.uniform(-2, 2, (n, 3))
    x0 = fp_state(pos, rpy, vel, w, np.full((n, 4), hover_rpm(base)))
    world_of = np.repeat(np.arange(M), N)
    is_abs = models[world_of] == 1
    xa = abs_state(pos[is_abs], rpy[is_abs], vel[is_abs], np.zeros((is_abs.sum(), 3)),
                   np.full(is_abs.sum(), base["mass"] * base["g"]))
    x0[is_abs] = xa
    hold = 50
    cmd = _attitude_commands(rng, (steps + hold - 1) // hold, n)
    kind = {"mixed": "mixed", "fp": "fp", "abs": "abs"}[models_of]
    return Workload(f"swarm_{M}x{N}_{kind}_euler_attitude_{steps}", M, N, -1, 0, 1, 1.0 / 500, steps,
                    K, hold, params, np.arange(M, dtype=np.int32), models, x0, cmd)


# ---------------------------------------------------------------------------
# Differentiable rollout (policy MLP 13 -> 64 -> 64 -> 4, tanh) inputs.

MLP_SIZES = (13, 64, 64, 4)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (round-to-nearest-even) and
    return them as float64 (exactly representable in both fp32 and fp64)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def policy_weights(seed: int) -> dict:
    """Xavier-uniform weights (last layer x 0.1), zero biases, rounded to bf16.
    Returned as float64 arrays W1 [64,13], b1 [64], W2 [64,64], b2 [64],
    W3 [4,64], b3 [4]."""
    rng = np.random.default_rng(seed)
    out = {}
    for li, (fi, fo) in enumerate(zip(MLP_SIZES[:-1], MLP_SIZES[1:]), start=1):
        lim = math.sqrt(6.0 / (fi + fo))
        W = rng.uniform(-lim, lim, (fo, fi))
        if li == 3:
            W = W * 0.1
        out[f"W{li}"] = bf16_round(W)
        out[f"b{li}"] = np.zeros(fo)
    return out


@dataclass
class RolloutWorkload:
    name: str
    M: int
    H: int
    C: int
    dt: float
    params: dict
    x0: np.ndarray          # [M, 20]
    p_ref: np.ndarray       # [H + 1, M, 3] reference position at t0 + k R dt
    weights: dict
    w_act: float
    repeat: int = 1         # R: physics steps per policy step


def figure8(t: np.ndarray, radius: float = 0.5, period: float = 4.0, height: float = 1.0):
    """Figure-8 target curve (lemniscate of Gerono) at z = height: position and
    velocity at times t.  x = r sin(w t), y = (r/2) sin(2 w t), w = 2 pi / period."""
    w = 2.0 * math.pi / period
    t = np.asarray(t, dtype=np.float64)
    pos = np.stack([radius * np.sin(w * t), 0.5 * radius * np.sin(2 * w * t),
                    np.full_like(t, height)], axis=-1)
    vel = np.stack([radius * w * np.cos(w * t), radius * w * np.cos(2 * w * t),
                    np.zeros_like(t)], axis=-1)
    return pos, vel


def policy_bptt(seed: int = 1003, M: int = 8192, H: int = 250, C: int = 25,
            repeat: int = 1) -> RolloutWorkload:
    """Differentiable rollout: M worlds x 1 drone, first-principles, attitude
    interface driven by the policy MLP 13 -> 64 -> 64 -> 4 (tanh, bf16
    weights), Euler at 500 Hz over H steps, checkpoint every C steps.  Target:
    figure-8 of radius 0.5 m and period 4 s at z = 1 m, sampled per world at
    t0 + k dt with t0 ~ U[0, 4) s.  Initial state: on the curve at t0 with
    U(+-0.05 m) position noise, the curve's velocity, identity attitude, zero
    body rates, rotors at hover speed.  repeat = R > 1: the policy acts every R
    physics steps (R = 10: a 50 Hz attitude policy), H counts policy steps and
    the reference is sampled at t0 + k R dt."""
    rng = np.random.default_rng(seed)
    P = crazyflie_params()
    dt = 1.0 / 500
    t0 = rng.uniform(0.0, 4.0, M)
    noise = rng.uniform(-0.05, 0.05, (M, 3))
    weights = policy_weights(seed + 7)
    p0, v0 = figure8(t0)
    x0 = fp_state(p0 + noise, np.zeros((M, 3)), v0, np.zeros((M, 3)),
                  np.full((M, 4), hover_rpm(P)))
    t = t0[None, :] + repeat * dt * np.arange(H + 1)[:, None]
    p_ref, _ = figure8(t)
    name = f"bptt_{M}x1_euler_H{H}_C{C}" + (f"_R{repeat}" if repeat > 1 else "")
    return RolloutWorkload(name, M, H, C, dt, P, x0, p_ref, weights, 1e-3, repeat)


# ---------------------------------------------------------------------------
# Uneven batched sampling rollouts.

@dataclass
class SamplingWorkload:
    name: str
    M: int
    n_per_world: np.ndarray   # [M] int64
    S: int
    H: int
    dt: float
    sigma: float
    seed: int                 # Philox key
    params: dict
    x0: np.ndarray            # [sum N, 20]
    goals: np.ndarray         # [M, 3]
    obstacles: np.ndarray     # [n_obs, 4] = centre xyz, radius
    w_obs: float


def uneven_sampling_rk4(seed: int = 1004, M: int = 512, S: int = 256, H: int = 50, n_max: int = 4000,
            n_obs: int = 32) -> SamplingWorkload:
    """512 worlds with drone counts N_w = clamp(round(exp(U(0, ln 4000))), 1, 4000);
    each drone expands S = 256 command sequences a = clip(0.2 * xi, -1, 1)
    (xi ~ N(0,1) from Philox4x32-10 keyed by the seed) over H = 50 RK4 steps at
    500 Hz.  Drones start at hover with positions U in [-1.5,1.5]^2 x [0.5,3.5];
    each world has a goal U in the same box; 32 spherical obstacles shared by
    all worlds, centres U in [-2,2]^2 x [0,4], radii U[0.1, 0.3]."""
    rng = np.random.default_rng(seed)
    P = crazyflie_params()
    n_w = np.clip(np.round(np.exp(rng.uniform(0.0, math.log(n_max), M))), 1, n_max).astype(np.int64)
    n = int(n_w.sum())
    lo, hi = np.array([-1.5, -1.5, 0.5]), np.array([1.5, 1.5, 3.5])
    pos = rng.uniform(lo, hi, (n, 3))
    x0 = fp_state(pos, np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3)),
                  np.full((n, 4), hover_rpm(P)))
    goals = rng.uniform(lo, hi, (M, 3))
    obs = np.zeros((n_obs, 4))
    obs[:, 0:3] = rng.uniform(np.array([-2.0, -2.0, 0.0]), np.array([2.0, 2.0, 4.0]), (n_obs, 3))
    obs[:, 3] = rng.uniform(0.1, 0.3, n_obs)
    key = int(rng.integers(0, 2**63))
    return SamplingWorkload(f"sampling_{M}w_uneven_S{S}_H{H}_rk4", M, n_w, S, H, 1.0 / 500, 0.2, key, P,
                            x0, goals, obs, 1000.0)


@dataclass
class BatchedWorkload:
    """Uneven / mixed batch: world w holds n_per_world[w] drones of model
    model_of_world[w]; drones are laid out world after world."""
    name: str
    n_per_world: np.ndarray     # [M] int64
    model_of_world: np.ndarray  # [M] int32
    integrator: int
    ctrl: int
    dt: float
    steps: int
    K: int
    hold: int
    params: list                # one parameter set per world
    x0: np.ndarray              # [sum N, 20]
    cmd: np.ndarray             # [n_blocks, sum N, 4]

    @property
    def M(self):
        return len(self.n_per_world)

    @property
    def ntot(self):
        return int(self.n_per_world.sum())

    def world_of_drone(self):
        return np.repeat(np.arange(self.M), self.n_per_world)


def batched_workload(seed: int, n_per_world, model_of_world, integrator: int = 0,
                     steps: int = 200, K: int = 200, hold: int = 50,
                     jitter: float = 0.1) -> BatchedWorkload:
    """Uneven/mixed batch with the mixed-swarm recipe: first-principles worlds use
    the Crazyflie set, abstracted worlds scale each abstracted coefficient by
    U(1 - jitter, 1 + jitter); initial states and attitude commands as in
    the mixed swarm (commands per drone, held `hold` steps)."""
    rng = np.random.default_rng(seed)
    n_w = np.asarray(n_per_world, dtype=np.int64)
    mw = np.asarray(model_of_world, dtype=np.int32)
    base = crazyflie_params()
    params = []
    for m in mw:
        q = dict(base)
        if m == 1:
            for k in ("c1_r", "c1_p", "c1_y", "c2_r", "c2_p", "c2_y", "c3_r", "c3_p", "c3_y",
                      "c_tau", "c_f"):
                q[k] = base[k] * rng.uniform(1 - jitter, 1 + jitter)
        params.append(q)
    n = int(n_w.sum())
    pos = np.array([0.0, 0.0, 1.0]) + rng.uniform(-1, 1, (n, 3))
    rpy = rng.uniform(-np.deg2rad(30), np.deg2rad(30), (n, 3))
    vel = rng.uniform(-1, 1, (n, 3))
    w = rng.uniform(-2, 2, (n, 3))
    x0 = fp_state(pos, rpy, vel, w, np.full((n, 4), hover_rpm(base)))
    is_abs = mw[np.repeat(np.arange(len(n_w)), n_w)] == 1
    if is_abs.any():
        x0[is_abs] = abs_state(pos[is_abs], rpy[is_abs], vel[is_abs],
                               np.zeros((is_abs.sum(), 3)),
                               np.full(is_abs.sum(), base["mass"] * base["g"]))
    cmd = _attitude_commands(rng, (steps + hold - 1) // hold, n)
    return BatchedWorkload(f"batched_{len(n_w)}w_{n}d", n_w, mw, integrator, 1, 1.0 / 500, steps,
                           K, hold, params, x0, cmd)


def log_uniform_counts(seed: int, M: int, n_max: int) -> np.ndarray:
    """N_w = clamp(round(exp(U(0, ln n_max))), 1, n_max) (the sampling workload's recipe)."""
    rng = np.random.default_rng(seed)
    return np.clip(np.round(np.exp(rng.uniform(0.0, math.log(n_max), M))), 1, n_max).astype(np.int64)


@dataclass
class MppiWorkload:
    name: str
    n_per_world: np.ndarray
    params: dict
    x0: np.ndarray           # [Ntot, 20]
    goals: np.ndarray        # [M, 3]
    obstacles: np.ndarray    # [n_obs, 4]
    dt: float
    cfg: dict                # S, H, n_ctrl, sigma, rho, n_elite, lam, w_obs
    seed: int


def mppi_workload(seed: int = 1005, n_drones: int = 64, S: int = 8000, n_ctrl: int = 5, H: int = 25,
                  dt: float = 1.0 / 50, n_obs: int = 32) -> MppiWorkload:
    """MPPI / iCEM control at the paper's scale: 64 drones (one world each)
    with 8000 samples each (512k sampled trajectories per iteration, as the
    paper's 500k), 5 parallel controllers, top 1 % elites, a 25-step horizon at
    50 Hz, RK4; drones at rest in [-1.5,1.5]^2 x [0.5,3.5], goals in the same
    box, 32 spherical obstacles as in the uneven sampling workload."""
    rng = np.random.default_rng(seed)
    P = crazyflie_params()
    lo, hi = np.array([-1.5, -1.5, 0.5]), np.array([1.5, 1.5, 3.5])
    pos = rng.uniform(lo, hi, (n_drones, 3))
    x0 = fp_state(pos, np.zeros((n_drones, 3)), np.zeros((n_drones, 3)), np.zeros((n_drones, 3)),
                  np.full((n_drones, 4), hover_rpm(P)))
    goals = rng.uniform(lo, hi, (n_drones, 3))
    obs = np.zeros((n_obs, 4))
    obs[:, 0:3] = rng.uniform(np.array([-2.0, -2.0, 0.0]), np.array([2.0, 2.0, 4.0]), (n_obs, 3))
    obs[:, 3] = rng.uniform(0.1, 0.3, n_obs)
    # top 1 % of each controller's samples (at least one): ceil(S_c / 100)
    n_elite = max(1, -(-(S // n_ctrl) // 100))
    cfg = dict(S=S, H=H, n_ctrl=n_ctrl, sigma=0.3, rho=0.7, n_elite=n_elite, lam=0.05, w_obs=1000.0)
    return MppiWorkload(f"mppi_{n_drones}x{S}_C{n_ctrl}_H{H}_50Hz", np.ones(n_drones, np.int64), P,
                        x0, goals, obs, dt, cfg, int(rng.integers(0, 2**62)))
