"""Pins of the FP64 oracle's dynamics, controller and integrators against
closed forms, conservation laws and special cases (no test here re-types the
oracle's own formulas)."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import workloads as W
from oracle import physics as ph
from oracle.rotation import quat_to_rot

F64 = torch.float64
DT = 1.0 / 500


def _P(n, **over):
    return ph.param_batch([W.crazyflie_params(**over)], [0] * n)


def _hover_state(n, P):
    x = torch.zeros(n, 20, dtype=F64)
    x[:, 0:3] = torch.randn(n, 3, dtype=F64)
    x[:, 6] = 1.0
    x[:, 13:17] = W.hover_rpm(W.crazyflie_params())
    return x


# --------------------------------------------------------------------------- hover


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_hover_is_a_fixed_point(integrator):
    """From hover (q = I, v = w = 0, W = W_h) with a zero action, each rotor
    carries m g / 4 and the state does not move (to rounding) for 1000 steps."""
    n = 4
    P = _P(n)
    x0 = _hover_state(n, P)
    T, tau = ph.rotor_wrench(x0[:, 13:17], P)
    p = W.crazyflie_params()
    np.testing.assert_allclose(T.numpy() / 4, p["mass"] * p["g"] / 4, rtol=1e-15)
    assert tau.abs().max() < 1e-18
    x = x0.clone()
    u = torch.zeros(n, 4, dtype=F64)
    for _ in range(1000):
        x = ph.step(x, u, P, DT, integrator, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
    assert (x - x0).abs()[:, :13].max() < 1e-12
    assert ((x - x0)[:, 13:17].abs() / 14476.0).max() < 1e-12


def test_position_controller_hover_fixed_point():
    n = 3
    P = _P(n)
    x = _hover_state(n, P)
    sp = torch.cat([x[:, 0:3], torch.zeros(n, 1, dtype=F64)], -1)
    x0 = x.clone()
    for _ in range(500):
        x = ph.step(x, sp, P, DT, ph.EULER, ph.CTRL_POSITION, ph.FIRST_PRINCIPLES)
    assert (x - x0)[:, :13].abs().max() < 1e-12


# --------------------------------------------------------------------------- translation


def _free_fall(integrator, n_steps):
    n = 5
    P = _P(n)
    rng = np.random.default_rng(0)
    x = torch.zeros(n, 20, dtype=F64)
    x[:, 0:3] = torch.tensor(rng.uniform(-1, 1, (n, 3)))
    x[:, 3:7] = torch.tensor(Rotation.random(n, random_state=1).as_quat())
    x[:, 7:10] = torch.tensor(rng.uniform(-2, 2, (n, 3)))
    x0 = x.clone()
    u = torch.zeros(n, 4, dtype=F64)  # rotor-speed interface, rotors stopped
    for _ in range(n_steps):
        x = ph.step(x, u, P, DT, integrator, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
    return x0, x


def test_free_fall_euler_closed_form():
    """Explicit Euler on p' = v, v' = -g e_z gives exactly
    p_n = p0 + n dt v0 - g dt^2 n (n - 1) / 2 e_z and v_n = v0 - n dt g e_z."""
    n = 300
    x0, x = _free_fall(ph.EULER, n)
    g = 9.81
    ez = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    p = x0[:, 0:3] + n * DT * x0[:, 7:10] - 0.5 * g * DT * DT * n * (n - 1) * ez
    v = x0[:, 7:10] - n * DT * g * ez
    assert torch.allclose(x[:, 0:3], p, atol=1e-12)
    assert torch.allclose(x[:, 7:10], v, atol=1e-12)


def test_free_fall_rk4_exact_parabola():
    """RK4 integrates the quadratic free-fall trajectory exactly."""
    n = 300
    x0, x = _free_fall(ph.RK4, n)
    t = n * DT
    ez = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    p = x0[:, 0:3] + t * x0[:, 7:10] - 0.5 * 9.81 * t * t * ez
    assert torch.allclose(x[:, 0:3], p, atol=1e-12)
    # no torque, no rotation: attitude unchanged
    assert torch.allclose(x[:, 3:7], x0[:, 3:7], atol=1e-14)


# --------------------------------------------------------------------------- rotation


def _tumble(J, w0, n_steps, dt, integrator=ph.RK4):
    n = w0.shape[0]
    P = _P(n, Jx=J[0], Jy=J[1], Jz=J[2])
    x = torch.zeros(n, 20, dtype=F64)
    x[:, 3:7] = torch.tensor(Rotation.random(n, random_state=7).as_quat())
    x[:, 10:13] = w0
    u = torch.zeros(n, 4, dtype=F64)
    traj = [x.clone()]
    for _ in range(n_steps):
        x = ph.step(x, u, P, dt, integrator, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
        traj.append(x.clone())
    return traj


def test_torque_free_symmetric_top_closed_form():
    """J_x = J_y (as the Crazyflie's inertia): w_z is constant and (w_x, w_y)
    rotates at lambda = (J_z - J_x) / J_x * w_z (Euler's equations)."""
    J = (1.4e-5, 1.4e-5, 2.17e-5)
    w0 = torch.tensor([[1.0, -0.5, 3.0], [-2.0, 0.3, -5.0], [0.2, 0.1, 8.0]], dtype=F64)
    n = 500
    traj = _tumble(J, w0, n, DT)
    t = n * DT
    lam = (J[2] - J[0]) / J[0] * w0[:, 2]
    c, s = torch.cos(lam * t), torch.sin(lam * t)
    wx = c * w0[:, 0] - s * w0[:, 1]
    wy = s * w0[:, 0] + c * w0[:, 1]
    w = traj[-1][:, 10:13]
    assert torch.allclose(w[:, 0], wx, atol=1e-9)
    assert torch.allclose(w[:, 1], wy, atol=1e-9)
    assert torch.allclose(w[:, 2], w0[:, 2], atol=1e-13)


def _energy_momentum(x, J):
    w = x[:, 10:13]
    Jv = torch.tensor(J, dtype=F64)
    E = 0.5 * (Jv * w * w).sum(-1)
    L = (quat_to_rot(x[:, 3:7]) @ (Jv * w)[..., None])[..., 0]
    return E, L


def test_asymmetric_tumbling_conserves_energy_and_momentum():
    """Torque-free asymmetric body: kinetic energy 1/2 w^T J w and the world
    angular momentum R J w are invariants; RK4 drift is small and falls by about
    2^4 per halving of dt."""
    J = (1.0e-5, 1.6e-5, 2.3e-5)
    w0 = torch.tensor([[3.0, 0.2, -1.0], [0.1, 4.0, 0.5]], dtype=F64)
    drifts = []
    for dt in (1 / 250, 1 / 500, 1 / 1000):
        traj = _tumble(J, w0, int(round(1.0 / dt)), dt)
        E0, L0 = _energy_momentum(traj[0], J)
        E1, L1 = _energy_momentum(traj[-1], J)
        drifts.append(((E1 - E0).abs() / E0).max().item()
                      + ((L1 - L0).norm(dim=-1) / L0.norm(dim=-1)).max().item())
    assert drifts[1] < 1e-7
    for a, b in zip(drifts[:-1], drifts[1:]):
        assert 10.0 < a / b < 24.0


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_quaternion_stays_unit(integrator):
    wl = W.attitude_swarm_rk4(M=64, steps=40)
    x = torch.tensor(wl.x0, dtype=F64)
    P = ph.param_batch(wl.params, [0] * 64)
    cmd = torch.tensor(wl.cmd, dtype=F64)
    for k in range(40):
        x = ph.step(x, cmd[k // 50], P, DT, integrator, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
        assert ((x[:, 3:7].norm(dim=-1) - 1).abs().max()) < 1e-14


def test_quaternion_derivative_is_tangent():
    """q' = 1/2 q (x) [w, 0] is orthogonal to q."""
    n = 16
    P = _P(n)
    x = torch.zeros(n, 17, dtype=F64)
    x[:, 3:7] = torch.tensor(Rotation.random(n, random_state=3).as_quat())
    x[:, 10:13] = torch.randn(n, 3, dtype=F64)
    d = ph.deriv_fp(x, torch.zeros(n, 4, dtype=F64), P)
    assert (d[:, 3:7] * x[:, 3:7]).sum(-1).abs().max() < 1e-15


# --------------------------------------------------------------------------- motors


def _motor_run(integrator, W0, Wc, n_steps, **over):
    n = W0.shape[0]
    P = _P(n, **over)
    x = torch.zeros(n, 20, dtype=F64)
    x[:, 6] = 1.0
    x[:, 13:17] = W0
    for _ in range(n_steps):
        x = ph.step(x, Wc, P, DT, integrator, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
    return x[:, 13:17]


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_motor_first_order_lag_closed_form(integrator):
    """With W' = (W_cmd - W) / tau, Euler gives W_n = W_c + (W_0 - W_c)(1 - h)^n and
    RK4 the degree-4 Taylor polynomial of exp(-h) per step, h = dt / tau."""
    W0 = torch.tensor([[10000.0, 15000.0, 12000.0, 2000.0]], dtype=F64)
    Wc = torch.tensor([[14000.0, 9000.0, 12000.0, 19000.0]], dtype=F64)
    n = 100
    h = DT / 0.03
    f = 1 - h if integrator == ph.EULER else 1 - h + h**2 / 2 - h**3 / 6 + h**4 / 24
    Wn = _motor_run(integrator, W0, Wc, n)
    ref = Wc + (W0 - Wc) * f**n
    assert torch.allclose(Wn, ref, rtol=1e-13, atol=1e-9)


def test_motor_asymmetric_branches():
    """Eq. 6: spin-up uses (cv_up, cd_up), spin-down (cv_down, cd_down).  With
    cd = 0 each branch is a first-order lag with its own rate; rotors commanded
    above their speed follow the up-rate and the others the down-rate."""
    W0 = torch.tensor([[10000.0, 15000.0, 10000.0, 15000.0]], dtype=F64)
    Wc = torch.tensor([[14000.0, 11000.0, 14000.0, 11000.0]], dtype=F64)
    cu, cdn = 50.0, 12.0
    n = 60
    Wn = _motor_run(ph.EULER, W0, Wc, n, cv_up=cu, cv_down=cdn)
    fu, fd = (1 - DT * cu) ** n, (1 - DT * cdn) ** n
    ref = Wc + (W0 - Wc) * torch.tensor([fu, fd, fu, fd], dtype=F64)
    assert torch.allclose(Wn, ref, rtol=1e-13)


def test_motor_quadratic_drag_braking():
    """Pure quadratic term (cv = 0, cd > 0) towards W_cmd = 0: W' = -cd W^2 has
    the solution W(t) = W0 / (1 + cd W0 t); RK4 follows it to O(dt^4)."""
    W0 = torch.tensor([[12000.0, 8000.0, 16000.0, 4000.0]], dtype=F64)
    cd = 2e-4
    n = 250
    Wn = _motor_run(ph.RK4, W0, torch.zeros(1, 4, dtype=F64), n, cv_up=0.0, cv_down=0.0,
                    cd_up=cd, cd_down=cd)
    t = n * DT
    assert torch.allclose(Wn, W0 / (1 + cd * W0 * t), rtol=1e-6)


# --------------------------------------------------------------------------- mixer / controller


def test_mixer_reproduces_requested_wrench():
    """rotor_wrench(mixer(T, tau)) == (T, tau) whenever no rotor saturates:
    the mixer's linear solve and the rotor cross products are independent
    formulations of the X-configuration geometry."""
    n = 50
    P = _P(n)
    p = W.crazyflie_params()
    rng = np.random.default_rng(11)
    T = torch.tensor(p["mass"] * p["g"] * rng.uniform(0.8, 1.3, n))
    tau = torch.tensor(rng.uniform(-1, 1, (n, 3)) * np.array([2e-4, 2e-4, 2e-4]))
    Wc = ph.mixer(T, tau, P)
    T2, tau2 = ph.rotor_wrench(Wc, P)
    assert torch.allclose(T2, T, rtol=1e-13)
    assert torch.allclose(tau2, tau, atol=1e-17)


def test_mixer_saturation():
    n = 2
    P = _P(n)
    p = W.crazyflie_params()
    T = torch.tensor([10.0, -1.0], dtype=F64)  # far above max, below zero
    Wc = ph.mixer(T, torch.zeros(n, 3, dtype=F64), P)
    assert torch.allclose(Wc[0], torch.full((4,), p["omega_max"], dtype=F64))
    assert torch.equal(Wc[1], torch.zeros(4, dtype=F64))


def test_attitude_error_small_angle_linearisation():
    """For R = R_d exp([th]x) with small th, e_R = th + O(th^2) and the PD torque
    opposes the error."""
    n = 20
    P = _P(n)
    Rd = torch.tensor(Rotation.random(n, random_state=9).as_matrix())
    th = torch.tensor(np.random.default_rng(2).normal(0, 1e-4, (n, 3)))
    R = Rd @ torch.tensor(Rotation.from_rotvec(th.numpy()).as_matrix())
    tau = ph.attitude_torque(R, torch.zeros(n, 3, dtype=F64), Rd, P)
    p = W.crazyflie_params()
    e_R = -tau / torch.tensor([p["Jx"] * p["KR_x"], p["Jy"] * p["KR_y"], p["Jz"] * p["KR_z"]])
    assert torch.allclose(e_R, th, atol=1e-7)


def test_attitude_loop_tracks_commanded_angles():
    """Closed loop (attitude interface, RK4): from random tilts within 30 deg and
    rates within 2 rad/s, the attitude converges to R_d of the command."""
    wl = W.attitude_swarm_rk4(M=32, steps=1)
    x = torch.tensor(wl.x0, dtype=F64)
    x[:, 7:10] = 0
    P = ph.param_batch(wl.params, [0] * 32)
    a = torch.tensor(np.random.default_rng(4).uniform(-0.5, 0.5, (32, 4)))
    a[:, 3] = 0.0
    for _ in range(1500):
        x = ph.step(x, a, P, DT, ph.RK4, ph.CTRL_ATTITUDE, ph.FIRST_PRINCIPLES)
    _, Rd, _ = ph.attitude_command(a, P)
    R = quat_to_rot(x[:, 3:7])
    assert (R - Rd).abs().max() < 1e-6
    assert x[:, 10:13].abs().max() < 1e-5


def test_position_loop_converges_single_drone():
    """Single-drone closed loop (position PID + attitude PD, Euler 500 Hz): after
    10 s the drone holds the (0, 0, 1) setpoint."""
    wl = W.position_hold_single()
    sp = torch.tensor([0.0, 0.0, 1.0], dtype=F64)
    e0 = (torch.tensor(wl.x0[0, 0:3]) - sp).norm()
    x5 = ph.rollout_workload(wl, steps=2500)
    wl.x0 = x5.numpy()
    x10 = ph.rollout_workload(wl, steps=2500)
    e5, e10 = (x5[0, 0:3] - sp).norm(), (x10[0, 0:3] - sp).norm()
    assert e10 < 5e-3 and e10 < 0.6 * e5 and e5 < 0.5 * e0
    assert x10[0, 7:13].abs().max() < 1e-3


# --------------------------------------------------------------------------- abstracted


def _abs_params(n, **over):
    return ph.param_batch([W.crazyflie_params(**over)], [0] * n)


def test_abstracted_euler_is_the_linear_recurrence():
    """With constant inputs the attitude and thrust channels are linear; Euler
    gives x_{n+1} = (I + dt A) x_n + dt B u exactly (checked with a matrix
    power), per axis and for f_sum."""
    n_st = 200
    P = _abs_params(1)
    p = W.crazyflie_params()
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 3:6] = torch.tensor([0.1, -0.2, 0.3])
    x[0, 9:12] = torch.tensor([0.5, 0.0, -0.4])
    x[0, 12] = 0.2
    a = torch.tensor([[0.3, -0.4, 0.8, 0.25]], dtype=F64)
    xs = x.clone()
    for _ in range(n_st):
        xs = ph.step(xs, a, P, DT, ph.EULER, ph.CTRL_ATTITUDE, ph.ABSTRACTED)
    for ax, (c1, c2, c3) in enumerate([("c1_r", "c2_r", "c3_r"), ("c1_p", "c2_p", "c3_p"),
                                       ("c1_y", "c2_y", "c3_y")]):
        A = np.array([[0.0, 1.0], [p[c1], p[c2]]])
        Bu = np.array([0.0, p[c3] * a[0, ax].item() * p["max_angle"]])
        Mx = np.eye(2) + DT * A
        z = np.array([x[0, 3 + ax].item(), x[0, 9 + ax].item()])
        ref = np.linalg.matrix_power(Mx, n_st) @ z + np.linalg.solve(
            np.eye(2) - Mx, (np.eye(2) - np.linalg.matrix_power(Mx, n_st)) @ (DT * Bu))
        np.testing.assert_allclose([xs[0, 3 + ax].item(), xs[0, 9 + ax].item()], ref, rtol=1e-11,
                                   atol=1e-13)
    fc = p["mass"] * p["g"] * (1 + p["thrust_scale"] * 0.25)
    ref_f = fc + (0.2 - fc) * (1 - DT * p["c_tau"]) ** n_st
    assert abs(xs[0, 12].item() - ref_f) < 1e-12


def test_abstracted_steady_state_and_hover():
    """Steady state Psi* = -c3 / c1 * Psi_cmd and f_sum -> f_cmd; from level
    attitude with f_sum = m g / c_f the point mass hovers."""
    P = _abs_params(1)
    p = W.crazyflie_params()
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 12] = p["mass"] * p["g"]
    x0 = x.clone()
    for _ in range(300):
        x = ph.step(x, torch.zeros(1, 4, dtype=F64), P, DT, ph.RK4, ph.CTRL_ATTITUDE, ph.ABSTRACTED)
    assert (x - x0).abs().max() < 1e-13
    a = torch.tensor([[0.2, -0.3, 0.6, 0.0]], dtype=F64)
    for _ in range(5000):
        x = ph.step(x, a, P, DT, ph.RK4, ph.CTRL_ATTITUDE, ph.ABSTRACTED)
    ang = a[0, :3] * p["max_angle"]
    c1 = torch.tensor([p["c1_r"], p["c1_p"], p["c1_y"]], dtype=F64)
    c3 = torch.tensor([p["c3_r"], p["c3_p"], p["c3_y"]], dtype=F64)
    assert torch.allclose(x[0, 3:6], -c3 / c1 * ang, atol=1e-10)


def test_abstracted_vertical_climb_closed_form():
    """Level attitude, constant thrust f_sum = f_cmd: vertical acceleration
    (c_f f - m g) / m, so z(t) = z0 + vz0 t + a t^2 / 2 (RK4 exact)."""
    P = _abs_params(1)
    p = W.crazyflie_params()
    a4 = 0.4
    fc = p["mass"] * p["g"] * (1 + p["thrust_scale"] * a4)
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 2], x[0, 8], x[0, 12] = 1.0, 0.3, fc
    n = 400
    for _ in range(n):
        x = ph.step(x, torch.tensor([[0.0, 0.0, 0.0, a4]], dtype=F64), P, DT, ph.RK4,
                    ph.CTRL_ATTITUDE, ph.ABSTRACTED)
    t = n * DT
    acc = (p["c_f"] * fc - p["mass"] * p["g"]) / p["mass"]
    assert abs(x[0, 2].item() - (1.0 + 0.3 * t + 0.5 * acc * t * t)) < 1e-11


def test_linear_drag_terminal_velocity():
    """Abstracted model, level hover thrust, drag C_a = -c I: horizontal velocity
    decays as v(t) = v0 exp(-c t / m)."""
    c = 0.01
    P = _abs_params(1, Ca_x=-c, Ca_y=-c, Ca_z=-c)
    p = W.crazyflie_params()
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 6], x[0, 12] = 1.5, p["mass"] * p["g"]
    n = 500
    for _ in range(n):
        x = ph.step(x, torch.zeros(1, 4, dtype=F64), P, DT, ph.RK4, ph.CTRL_ATTITUDE, ph.ABSTRACTED)
    assert abs(x[0, 6].item() - 1.5 * math.exp(-c * n * DT / p["mass"])) < 1e-9


def test_first_principles_drag_is_body_frame():
    """First-principles drag acts in the body frame: with yaw = 90 deg and
    C_a = diag(-cx, -cy, 0), a world-x velocity is damped by the body-y
    coefficient."""
    P = _P(1, Ca_x=-0.01, Ca_y=-0.03, Ca_z=0.0)
    p = W.crazyflie_params()
    x = torch.zeros(1, 17, dtype=F64)
    x[0, 3:7] = torch.tensor(Rotation.from_euler("z", 90, degrees=True).as_quat())
    x[0, 7] = 2.0
    d = ph.deriv_fp(x, torch.zeros(1, 4, dtype=F64), P)
    assert abs(d[0, 7].item() - (-0.03 * 2.0 / p["mass"])) < 1e-12


# --------------------------------------------------------------------------- RK4 order


def test_rk4_fourth_order_convergence():
    """Smooth case (rotor-speed interface, constant commands, equal motor
    coefficients): the error at t = 0.1 s against a dt/64 reference falls by
    about 16 per halving of dt."""
    n = 4
    P = _P(n)
    rng = np.random.default_rng(21)
    x = torch.zeros(n, 20, dtype=F64)
    x[:, 0:3] = torch.tensor(rng.uniform(-1, 1, (n, 3)))
    x[:, 3:7] = torch.tensor(Rotation.random(n, random_state=5).as_quat())
    x[:, 7:10] = torch.tensor(rng.uniform(-1, 1, (n, 3)))
    x[:, 10:13] = torch.tensor(rng.uniform(-3, 3, (n, 3)))
    x[:, 13:17] = torch.tensor(rng.uniform(12000, 17000, (n, 4)))
    u = torch.tensor(rng.uniform(12000, 17000, (n, 4)))
    T = 0.1

    def run(dt):
        xs = x.clone()
        for _ in range(int(round(T / dt))):
            xs = ph.step(xs, u, P, dt, ph.RK4, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
        return xs

    ref = run(1 / 32000)
    errs = []
    for dt in (1 / 250, 1 / 500, 1 / 1000):
        e = run(dt) - ref
        errs.append(max(e[:, 0:13].abs().max().item(), (e[:, 13:17].abs().max() / 1e4).item()))
    for a, b in zip(errs[:-1], errs[1:]):
        assert 12.0 < a / b < 20.0, errs
