"""Pins of the oracle's rotor extensions and extra interfaces: rotor inertia
(gyroscopic + reaction torques) conserving total angular momentum, the
polynomial thrust curve's inversion, the torque interface, and the abstracted
variant without thrust dynamics."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import workloads as W
from oracle import physics as ph
from oracle.rotation import quat_to_rot

F64 = torch.float64


def _P(n, **over):
    return ph.param_batch([W.crazyflie_params(**over)], [0] * n)


def _momentum(x, P, J):
    """World-frame total angular momentum R (J w + h e_z)."""
    w = x[:, 10:13]
    Lb = torch.tensor(J, dtype=F64) * w
    Lb[:, 2] = Lb[:, 2] + ph.rotor_momentum(x[:, 13:17], P)
    return (quat_to_rot(x[:, 3:7]) @ Lb[..., None])[..., 0]


def test_rotor_inertia_conserves_total_angular_momentum():
    """With no rotor wrench (kf = km = 0) the gyroscopic and reaction torques
    are internal: R (J w + h e_z) is invariant while the rotors spin up and down
    at different rates; RK4's drift falls ~16x per halving of dt."""
    J = (1.4e-5, 1.6e-5, 2.17e-5)
    n = 3
    P = _P(n, Jx=J[0], Jy=J[1], Jz=J[2], J_p=6e-8, kf=0.0, km=0.0)
    rng = np.random.default_rng(0)
    x0 = torch.zeros(n, 20, dtype=F64)
    x0[:, 3:7] = torch.tensor(Rotation.random(n, random_state=2).as_quat())
    x0[:, 10:13] = torch.tensor(rng.uniform(-3, 3, (n, 3)))
    x0[:, 13:17] = torch.tensor(rng.uniform(8000, 16000, (n, 4)))
    u = torch.tensor(rng.uniform(6000, 19000, (n, 4)))
    drifts = []
    for dt in (1 / 250, 1 / 500, 1 / 1000):
        x = x0.clone()
        L0 = _momentum(x, P, J)
        for _ in range(int(round(0.4 / dt))):
            x = ph.step(x, u, P, dt, ph.RK4, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
        L1 = _momentum(x, P, J)
        drifts.append(((L1 - L0).norm(dim=-1) / L0.norm(dim=-1)).max().item())
        # the rotors did change speed, so the reaction torque was exercised
        assert (x[:, 13:17] - x0[:, 13:17]).abs().max() > 1000
    assert drifts[1] < 1e-8
    for a, b in zip(drifts[:-1], drifts[1:]):
        assert 10.0 < a / b < 24.0


def test_rotor_spin_up_turns_the_body_the_other_way():
    """From rest, one rotor accelerating (spin direction sigma = -s) gives the
    body the opposite yaw momentum: J_z w_z = -(h - h0) exactly (z-axis only)."""
    P = _P(1, J_p=6e-8, kf=0.0, km=0.0)
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 6] = 1.0
    x[0, 13:17] = 10000.0
    u = torch.tensor([[18000.0, 10000.0, 10000.0, 10000.0]], dtype=F64)
    h0 = ph.rotor_momentum(x[:, 13:17], P)
    for _ in range(100):
        x = ph.step(x, u, P, 1 / 500, ph.RK4, ph.CTRL_ROTOR_SPEED, ph.FIRST_PRINCIPLES)
    h = ph.rotor_momentum(x[:, 13:17], P)
    assert abs(x[0, 12].item() * 2.17e-5 + (h - h0).item()) < 1e-12
    # rotor 1 has yaw sign s = -1, i.e. spins along +z: the body turns along -z
    assert x[0, 12].item() < 0
    assert x[0, 10:12].abs().max() < 1e-15


def test_polynomial_thrust_inversion():
    """thrust(mixer(T, 0)) = T / 4 per rotor for a thrust curve with linear and
    constant terms (the quadratic root against the forward polynomial), and the
    hover fixed point survives."""
    n = 6
    P = _P(n, kf1=2e-7, kf0=-0.004)
    p = W.crazyflie_params(kf1=2e-7, kf0=-0.004)
    T = torch.tensor(p["mass"] * p["g"] * np.linspace(0.6, 1.6, n))
    Wc = ph.mixer(T, torch.zeros(n, 3, dtype=F64), P)
    f = ph.rotor_thrust(Wc, P)
    assert torch.allclose(f, (T / 4)[:, None].expand(n, 4), rtol=1e-12)
    x = torch.zeros(2, 20, dtype=F64)
    x[:, 2] = 1.0
    x[:, 6] = 1.0
    P2 = _P(2, kf1=2e-7, kf0=-0.004)
    x[:, 13:17] = ph.mixer(torch.full((2,), p["mass"] * p["g"], dtype=F64),
                           torch.zeros(2, 3, dtype=F64), P2)
    x0 = x.clone()
    for _ in range(500):
        x = ph.step(x, torch.zeros(2, 4, dtype=F64), P2, 1 / 500, ph.RK4, ph.CTRL_ATTITUDE,
                    ph.FIRST_PRINCIPLES)
    assert (x - x0)[:, :13].abs().max() < 1e-12


def test_torque_interface_reproduces_the_wrench():
    n = 20
    P = _P(n)
    p = W.crazyflie_params()
    rng = np.random.default_rng(3)
    T = p["mass"] * p["g"] * rng.uniform(0.8, 1.2, n)
    tau = rng.uniform(-1, 1, (n, 3)) * 2e-4
    u = torch.tensor(np.concatenate([T[:, None], tau], 1))
    Wc, _ = ph.control(torch.zeros(n, 20, dtype=F64), u, P, ph.CTRL_TORQUE, 0.002)
    T2, tau2 = ph.rotor_wrench(Wc, P)
    assert torch.allclose(T2, torch.tensor(T), rtol=1e-13)
    assert torch.allclose(tau2, torch.tensor(tau), atol=1e-17)


@pytest.mark.parametrize("integrator", [ph.EULER, ph.RK4])
def test_abstracted_without_thrust_dynamics(integrator):
    """Level attitude and a constant command: z follows the parabola of
    acceleration c_f f_cmd / m - g (RK4 exactly, Euler its exact discrete form);
    the f_sum slot holds f_cmd; the attitude channels equal the full
    abstracted model's."""
    p = W.crazyflie_params()
    P = _P(1)
    a4 = 0.3
    fc = p["mass"] * p["g"] * (1 + p["thrust_scale"] * a4)
    x = torch.zeros(1, 20, dtype=F64)
    x[0, 2], x[0, 8] = 1.0, 0.2
    n, dt = 300, 1 / 500
    u = torch.tensor([[0.0, 0.0, 0.0, a4]], dtype=F64)
    for _ in range(n):
        x = ph.step(x, u, P, dt, integrator, ph.CTRL_ATTITUDE, ph.ABSTRACTED_NOTHRUST)
    acc = p["c_f"] * fc / p["mass"] - p["g"]
    t = n * dt
    z = 1.0 + 0.2 * t + (0.5 * acc * t * t if integrator == ph.RK4 else 0.5 * acc * dt * dt * n * (n - 1))
    assert abs(x[0, 2].item() - z) < 1e-12
    assert x[0, 12].item() == fc
    ua = torch.tensor([[0.4, -0.3, 0.5, 0.1]], dtype=F64)
    xa = torch.zeros(1, 20, dtype=F64)
    xa[0, 12] = p["mass"] * p["g"]
    xb = xa.clone()
    for _ in range(50):
        xa = ph.step(xa, ua, P, dt, integrator, ph.CTRL_ATTITUDE, ph.ABSTRACTED)
        xb = ph.step(xb, ua, P, dt, integrator, ph.CTRL_ATTITUDE, ph.ABSTRACTED_NOTHRUST)
    assert torch.equal(xa[:, 3:6], xb[:, 3:6]) and torch.equal(xa[:, 9:12], xb[:, 9:12])
