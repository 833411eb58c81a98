"""FP64 oracle: drone dynamics, controllers and the Euler / RK4 step.

TEST INFRASTRUCTURE ONLY (see the package header).  Every function works on a
batch of drones (leading dimension B); parameters are a dict of [B] float64
tensors built by ``param_batch``.

Paper passages followed (Materials and Methods of arXiv 2606.01478):
  * rigid body, Eqs. 1-4 (First Principles Modeling): p' = v,
    q' = 1/2 q (x) [w; 0], m v' = f_sum, J w' = t_sum - w x J w
  * per-rotor thrust and drag counter-torque, "second-order polynomial" in the
    rotor speed (text before Eq. 5): f_i = kf W_i^2 + kf1 W_i + kf0,
    t_i = km W_i^2 + km1 W_i (the benchmark workloads use kf1 = kf0 = km1 = 0)
  * gyroscopic and reaction torques of the rotors, Eq. 5 (garbled in the
    paper; read from the rotors' angular momentum h = J_p (2 pi / 60)
    sum_i sigma_i W_i e_z with spin direction sigma_i = -s_i: tau_gyro = -w x h,
    tau_react = -dh/dt, whose z row is Eq. 5's third row)
  * X-configuration mixing (text after Eq. 5) with the yaw sign pattern
    (-, +, -, +) of Eq. 5's third row
  * linear body-frame drag f_a = C_a v_B (text after Eq. 5)
  * asymmetric rotor dynamics, Eq. 6 (tie W_cmd = W takes the first branch)
  * state x = [p, q, v, w, W], input u = W_cmd (text after Eq. 6)
  * abstracted model, Eqs. 7-10 (Abstracted Physics Modeling)
  * four control interfaces of the Mellinger stack (text after Eq. 6); the
    paper prints no controller equations or gains.

Parity status:
  deriv_fp, deriv_abs, rotor_wrench, motor_rate, step (Euler/RK4): pinned by
    closed forms (hover fixed point, free fall, torque-free symmetric top,
    energy / angular-momentum conservation, motor step response, linear
    abstracted response, RK4 order) in tests/test_oracle_physics.py.
  mixer: pinned by reproducing the requested wrench through rotor_wrench.
  attitude_command, attitude_torque, position_command: parity unpinned against
    the paper (the controller reading adopted here); pinned by the hover fixed
    point, the small-angle linearisation of the attitude error and closed-loop
    convergence.
"""
from __future__ import annotations

import math

import torch

from .rotation import euler_to_rot, quat_mul, quat_to_rot, vee

F64 = torch.float64

FIRST_PRINCIPLES, ABSTRACTED, ABSTRACTED_NOTHRUST = 0, 1, 2
EULER, RK4 = 0, 1
CTRL_ROTOR_SPEED, CTRL_ATTITUDE, CTRL_POSITION, CTRL_TORQUE = 0, 1, 2, 3

# X configuration (body x forward, y left, z up).  Rotor i sits at
# (sx_i a, sy_i a, 0) with a = arm / sqrt(2); its drag counter-torque about
# body z has sign s_i (Eq. 5, third row: -, +, -, +).
ROTOR_SX = (1.0, -1.0, -1.0, 1.0)
ROTOR_SY = (-1.0, -1.0, 1.0, 1.0)
ROTOR_YAW = (-1.0, 1.0, -1.0, 1.0)
RPM_TO_RAD_S = 2.0 * math.pi / 60.0


def param_batch(params: list, set_of_drone) -> dict:
    """Per-drone parameter tensors: params is a list of dicts (one per
    parameter set), set_of_drone [B] indexes into it."""
    idx = torch.as_tensor(set_of_drone, dtype=torch.long)
    out = {}
    for k in params[0]:
        col = torch.tensor([float(p[k]) for p in params], dtype=F64)
        out[k] = col[idx]
    return out


def _v3(P, a, b, c):
    return torch.stack([P[a], P[b], P[c]], dim=-1)


def rotor_positions(P) -> torch.Tensor:
    """[B, 4, 3] rotor positions in the body frame."""
    a = P["arm"] / math.sqrt(2.0)
    sx = torch.tensor(ROTOR_SX, dtype=F64)
    sy = torch.tensor(ROTOR_SY, dtype=F64)
    x = a[:, None] * sx[None, :]
    y = a[:, None] * sy[None, :]
    return torch.stack([x, y, torch.zeros_like(x)], dim=-1)


def rotor_thrust(W: torch.Tensor, P) -> torch.Tensor:
    """Per-rotor thrust kf W^2 + kf1 W + kf0 [B, 4]."""
    return P["kf"][:, None] * W * W + P["kf1"][:, None] * W + P["kf0"][:, None]


def rotor_wrench(W: torch.Tensor, P) -> tuple[torch.Tensor, torch.Tensor]:
    """Collective thrust T [B] and body torque tau [B, 3] of rotor speeds W [B, 4]
    (RPM): thrust f_i along body z at r_i, drag counter-torque
    km W_i^2 + km1 W_i with sign s_i about body z."""
    f = rotor_thrust(W, P)
    F = torch.zeros(W.shape + (3,), dtype=F64)
    F[..., 2] = f
    tau = torch.linalg.cross(rotor_positions(P), F, dim=-1).sum(dim=1)
    yaw = torch.tensor(ROTOR_YAW, dtype=F64)
    drag = P["km"][:, None] * W * W + P["km1"][:, None] * W
    tau[:, 2] = tau[:, 2] + (drag * yaw).sum(dim=1)
    return f.sum(dim=1), tau


def rotor_momentum(W: torch.Tensor, P) -> torch.Tensor:
    """z component of the rotors' angular momentum in the body frame [B]:
    J_p (2 pi / 60) sum_i sigma_i W_i with spin direction sigma_i = -s_i."""
    yaw = torch.tensor(ROTOR_YAW, dtype=F64)
    return -P["J_p"] * RPM_TO_RAD_S * (W * yaw).sum(dim=1)


def motor_rate(W: torch.Tensor, Wc: torch.Tensor, P) -> torch.Tensor:
    """Eq. 6: W' = c_v (Wc - W) + c_d (Wc^2 - W^2), coefficients (cv_up, cd_up)
    where Wc >= W, else (cv_down, cd_down)."""
    up = P["cv_up"][:, None] * (Wc - W) + P["cd_up"][:, None] * (Wc * Wc - W * W)
    dn = P["cv_down"][:, None] * (Wc - W) + P["cd_down"][:, None] * (Wc * Wc - W * W)
    return torch.where(Wc >= W, up, dn)


def _has_drag(P) -> bool:
    return bool((P["Ca_x"] != 0).any() or (P["Ca_y"] != 0).any() or (P["Ca_z"] != 0).any())


def deriv_fp(x: torch.Tensor, Wc: torch.Tensor, P) -> torch.Tensor:
    """First-principles derivative (Eqs. 1-4, 6) of x = [p, q, v, w, W] [B, 17]
    for held rotor-speed commands Wc [B, 4].  Gravity g acts along -z; the
    linear drag term is evaluated only when some C_a entry is non-zero (it is
    identically zero otherwise)."""
    p, q, v, w, W = x[:, 0:3], x[:, 3:7], x[:, 7:10], x[:, 10:13], x[:, 13:17]
    R = quat_to_rot(q)
    T, tau = rotor_wrench(W, P)
    f_body = torch.zeros_like(v)
    f_body[:, 2] = T
    if _has_drag(P):
        v_body = (R.transpose(-1, -2) @ v[..., None])[..., 0]
        f_body = f_body + _v3(P, "Ca_x", "Ca_y", "Ca_z") * v_body
    f_world = (R @ f_body[..., None])[..., 0]
    g = torch.zeros_like(v)
    g[:, 2] = P["g"]
    v_dot = f_world / P["mass"][:, None] - g
    J = torch.diag_embed(_v3(P, "Jx", "Jy", "Jz"))
    Jw = (J @ w[..., None])[..., 0]
    W_dot = motor_rate(W, Wc, P)
    if bool((P["J_p"] != 0).any()):
        # rotor angular momentum h e_z: gyroscopic -w x h and reaction -dh/dt
        h = torch.zeros_like(w)
        h[:, 2] = rotor_momentum(W, P)
        dh = torch.zeros_like(w)
        dh[:, 2] = rotor_momentum(W_dot, P)
        tau = tau - torch.linalg.cross(w, h, dim=-1) - dh
    w_dot = torch.linalg.solve(J, tau - torch.linalg.cross(w, Jw, dim=-1))
    q_dot = 0.5 * quat_mul(q, torch.cat([w, torch.zeros_like(w[:, :1])], dim=-1))
    return torch.cat([v, q_dot, v_dot, w_dot, W_dot], dim=-1)


def deriv_abs_nothrust(x: torch.Tensor, u: torch.Tensor, P) -> torch.Tensor:
    """Abstracted model without thrust dynamics and drag (last sentence of
    Abstracted Physics Modeling): m v' = f_g + R(Psi) e_z c_f f_cmd, with the
    attitude channels of Eq. 10; the f_sum slot does not evolve (the stepper
    sets it to f_cmd)."""
    psi, v, psid = x[:, 3:6], x[:, 6:9], x[:, 9:12]
    R = euler_to_rot(psi)
    g = torch.zeros_like(v)
    g[:, 2] = P["g"]
    v_dot = R[:, :, 2] * (P["c_f"] * u[:, 3] / P["mass"])[:, None] - g
    psi_dd = (_v3(P, "c1_r", "c1_p", "c1_y") * psi + _v3(P, "c2_r", "c2_p", "c2_y") * psid
              + _v3(P, "c3_r", "c3_p", "c3_y") * u[:, 0:3])
    return torch.cat([v, psid, v_dot, psi_dd, torch.zeros_like(x[:, 12:13])], dim=-1)


def deriv_abs(x: torch.Tensor, u: torch.Tensor, P) -> torch.Tensor:
    """Abstracted model (Eqs. 7-10) of x = [p, Psi, v, Psi', f_sum] [B, 13] for
    u = [Psi_cmd (3), f_cmd] [B, 4]:
        p' = v
        m v' = f_g + R(Psi) e_z c_f f_sum + R(Psi) C_a R(Psi)^T v
        f_sum' = c_tau (f_cmd - f_sum)
        Psi'' = c1 Psi + c2 Psi' + c3 Psi_cmd   (per axis)."""
    p, psi, v, psid, fs = x[:, 0:3], x[:, 3:6], x[:, 6:9], x[:, 9:12], x[:, 12]
    R = euler_to_rot(psi)
    f_body = torch.zeros_like(v)
    f_body[:, 2] = P["c_f"] * fs
    if _has_drag(P):
        v_body = (R.transpose(-1, -2) @ v[..., None])[..., 0]
        f_body = f_body + _v3(P, "Ca_x", "Ca_y", "Ca_z") * v_body
    g = torch.zeros_like(v)
    g[:, 2] = P["g"]
    v_dot = (R @ f_body[..., None])[..., 0] / P["mass"][:, None] - g
    fs_dot = P["c_tau"] * (u[:, 3] - fs)
    psi_dd = (_v3(P, "c1_r", "c1_p", "c1_y") * psi + _v3(P, "c2_r", "c2_p", "c2_y") * psid
              + _v3(P, "c3_r", "c3_p", "c3_y") * u[:, 0:3])
    return torch.cat([v, psid, v_dot, psi_dd, fs_dot[:, None]], dim=-1)


# ---------------------------------------------------------------------------
# Controller (the reading of the Mellinger stack adopted here; see module header)


def attitude_command(a: torch.Tensor, P) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Normalised action a in [-1, 1]^4 (clipped) -> desired roll/pitch/yaw
    (a_1..3 * max_angle), R_d = Rz Ry Rx of those angles, and collective thrust
    T_d = m g (1 + thrust_scale a_4)."""
    a = a.clamp(-1.0, 1.0)
    ang = a[:, 0:3] * P["max_angle"][:, None]
    Td = P["mass"] * P["g"] * (1.0 + P["thrust_scale"] * a[:, 3])
    return ang, euler_to_rot(ang), Td


def position_command(x: torch.Tensor, sp: torch.Tensor, I: torch.Tensor, P, dt: float):
    """Position PID (geometric, Mellinger-style) to setpoint sp = (x, y, z, yaw):
        e_p = sp - p,  a_d = Kp e_p + Ki I - Kd v + g e_z,
        T_d = m a_d . (R e_z),  z_d = a_d / |a_d|,
        y_d = z_d x (cos yaw, sin yaw, 0) normalised,  x_d = y_d x z_d,
        I <- I + e_p dt  (explicit Euler at controller time)."""
    p, q, v = x[:, 0:3], x[:, 3:7], x[:, 7:10]
    R = quat_to_rot(q)
    e_p = sp[:, 0:3] - p
    g = torch.zeros_like(p)
    g[:, 2] = P["g"]
    a_d = (_v3(P, "Kp_x", "Kp_y", "Kp_z") * e_p + _v3(P, "Ki_x", "Ki_y", "Ki_z") * I
           - _v3(P, "Kd_x", "Kd_y", "Kd_z") * v + g)
    Td = P["mass"] * (a_d * R[:, :, 2]).sum(dim=-1)
    z_d = a_d / torch.linalg.vector_norm(a_d, dim=-1, keepdim=True)
    yaw = sp[:, 3]
    x_c = torch.stack([torch.cos(yaw), torch.sin(yaw), torch.zeros_like(yaw)], dim=-1)
    y_d = torch.linalg.cross(z_d, x_c, dim=-1)
    y_d = y_d / torch.linalg.vector_norm(y_d, dim=-1, keepdim=True)
    x_d = torch.linalg.cross(y_d, z_d, dim=-1)
    Rd = torch.stack([x_d, y_d, z_d], dim=-1)
    return Rd, Td, I + e_p * dt


def attitude_torque(R: torch.Tensor, w: torch.Tensor, Rd: torch.Tensor, P) -> torch.Tensor:
    """Geometric attitude PD on SO(3) with zero desired rate:
        e_R = 1/2 vee(R_d^T R - R^T R_d),  tau = J (-K_R e_R - K_w w)."""
    e_R = 0.5 * vee(Rd.transpose(-1, -2) @ R - R.transpose(-1, -2) @ Rd)
    J = _v3(P, "Jx", "Jy", "Jz")
    return J * (-_v3(P, "KR_x", "KR_y", "KR_z") * e_R - _v3(P, "Kw_x", "Kw_y", "Kw_z") * w)


def mixing_matrix(P) -> torch.Tensor:
    """A [B, 4, 4] with [T, tau_x, tau_y, tau_z] = A f for per-rotor thrusts f:
    columns (1, y_i, -x_i, s_i km / kf)."""
    r = rotor_positions(P)
    yaw = torch.tensor(ROTOR_YAW, dtype=F64)
    rows = [torch.ones_like(r[..., 0]), r[..., 1], -r[..., 0],
            (P["km"] / P["kf"])[:, None] * yaw[None, :]]
    return torch.stack(rows, dim=1)


def mixer(Td: torch.Tensor, tau: torch.Tensor, P) -> torch.Tensor:
    """Per-rotor thrusts f = A^-1 [T_d, tau] clipped to [f(0), f(W_max)], then
    the rotor-speed commands that produce them: the root W >= 0 of
    kf W^2 + kf1 W + kf0 = f (W = sqrt(f / kf) for a pure quadratic).  The yaw
    row of A uses the quadratic coefficients' ratio km / kf."""
    wrench = torch.cat([Td[:, None], tau], dim=-1)
    f = torch.linalg.solve(mixing_matrix(P), wrench)
    wmax = P["omega_max"]
    fmin = P["kf0"]
    fmax = P["kf"] * wmax * wmax + P["kf1"] * wmax + P["kf0"]
    f = torch.minimum(torch.maximum(f, fmin[:, None]), fmax[:, None])
    kf, kf1 = P["kf"][:, None], P["kf1"][:, None]
    disc = torch.clamp(kf1 * kf1 + 4.0 * kf * (f - P["kf0"][:, None]), min=0.0)
    return (torch.sqrt(disc) - kf1) / (2.0 * kf)


def control(x20: torch.Tensor, u: torch.Tensor, P, ctrl: int, dt: float):
    """Controller for the first-principles model: returns (W_cmd [B,4], I' [B,3])."""
    x = x20[:, :17]
    I = x20[:, 17:20]
    if ctrl == CTRL_ROTOR_SPEED:
        Wc = torch.minimum(torch.clamp(u, min=0.0), P["omega_max"][:, None])
        return Wc, I
    if ctrl == CTRL_TORQUE:
        return mixer(u[:, 0], u[:, 1:4], P), I
    if ctrl == CTRL_ATTITUDE:
        _, Rd, Td = attitude_command(u, P)
        I_new = I
    elif ctrl == CTRL_POSITION:
        Rd, Td, I_new = position_command(x, u, I, P, dt)
    else:
        raise ValueError(ctrl)
    R = quat_to_rot(x[:, 3:7])
    tau = attitude_torque(R, x[:, 10:13], Rd, P)
    return mixer(Td, tau, P), I_new


def integrate(f, x: torch.Tensor, dt: float, integrator: int) -> torch.Tensor:
    """Explicit Euler x + dt f(x), or classic RK4 with the input held over the
    four stages."""
    if integrator == EULER:
        return x + dt * f(x)
    k1 = f(x)
    k2 = f(x + 0.5 * dt * k1)
    k3 = f(x + 0.5 * dt * k2)
    k4 = f(x + dt * k3)
    return x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


def step(x20: torch.Tensor, u: torch.Tensor, P, dt: float, integrator: int, ctrl: int,
         model: int) -> torch.Tensor:
    """One simulation step of a batch of drones of one model: controller (held
    over the step), derivative, integrator; the first-principles quaternion is
    renormalised once at the end of the step."""
    if model == FIRST_PRINCIPLES:
        Wc, I_new = control(x20, u, P, ctrl, dt)
        x = integrate(lambda s: deriv_fp(s, Wc, P), x20[:, :17], dt, integrator)
        q = x[:, 3:7] / torch.linalg.vector_norm(x[:, 3:7], dim=-1, keepdim=True)
        return torch.cat([x[:, 0:3], q, x[:, 7:17], I_new], dim=-1)
    if model in (ABSTRACTED, ABSTRACTED_NOTHRUST):
        if ctrl != CTRL_ATTITUDE:
            raise ValueError("the abstracted model takes attitude commands")
        ang, _, Td = attitude_command(u, P)
        ua = torch.cat([ang, Td[:, None]], dim=-1)
        if model == ABSTRACTED:
            x = integrate(lambda s: deriv_abs(s, ua, P), x20[:, :13], dt, integrator)
        else:
            x = integrate(lambda s: deriv_abs_nothrust(s, ua, P), x20[:, :13], dt, integrator)
            x = torch.cat([x[:, :12], Td[:, None]], dim=-1)  # f_sum follows f_cmd at once
        return torch.cat([x, x20[:, 13:20]], dim=-1)
    raise ValueError(model)


def rollout(x0, cmd, hold: int, steps: int, params: list, set_of_drone, model_of_drone,
            dt: float, integrator: int, ctrl: int, record_every: int = 0):
    """Run `steps` steps of a batch whose drones may mix models.  cmd is
    [n_blocks, B, 4]; step k uses block min(k // hold, n_blocks - 1).
    Returns the final [B, 20] state (and, if record_every > 0, the states
    after every record_every steps)."""
    x = torch.as_tensor(x0, dtype=F64).clone()
    cmd = torch.as_tensor(cmd, dtype=F64)
    P_all = param_batch(params, set_of_drone)
    models = torch.as_tensor(model_of_drone, dtype=torch.long)
    groups = [(m, torch.nonzero(models == m)[:, 0])
              for m in (FIRST_PRINCIPLES, ABSTRACTED, ABSTRACTED_NOTHRUST)]
    groups = [(m, idx) for m, idx in groups if idx.numel() > 0]
    Pg = {m: {k: v[idx] for k, v in P_all.items()} for m, idx in groups}
    trace = []
    for k in range(steps):
        b = min(k // hold, cmd.shape[0] - 1)
        for m, idx in groups:
            x[idx] = step(x[idx], cmd[b][idx], Pg[m], dt, integrator, ctrl, m)
        if record_every and (k + 1) % record_every == 0:
            trace.append(x.clone())
    return (x, trace) if record_every else x


def rollout_workload(wl, steps: int | None = None, drones=None):
    """Oracle rollout of a ``workloads.Workload`` (optionally a subset of drones,
    which is exact because drones do not interact)."""
    n = wl.M * wl.N
    idx = torch.arange(n) if drones is None else torch.as_tensor(drones, dtype=torch.long)
    world = idx // wl.N
    set_of = torch.as_tensor(wl.param_set_of_world, dtype=torch.long)[world]
    model_of = torch.as_tensor(wl.model_of_world, dtype=torch.long)[world]
    x0 = torch.as_tensor(wl.x0, dtype=F64)[idx]
    cmd = torch.as_tensor(wl.cmd, dtype=F64)[:, idx]
    return rollout(x0, cmd, wl.hold, wl.steps if steps is None else steps, wl.params, set_of,
                   model_of, wl.dt, wl.integrator, wl.ctrl)
