"""Algorithmic FP32 work of one drone-step, counted by running a plain scalar
restatement of the step on an op-counting number type.

The restatement follows the method's formulas as stated (First Principles
Modeling, Eqs. 1-6; Abstracted Physics Modeling, Eqs. 7-10; the attitude
interface's controller and mixer; explicit Euler and classic RK4 with the
controller output held over the stages; the quaternion renormalised once per
step), for the configuration every benchmark workload uses: pure quadratic
rotor curves (kf W^2, km W^2), first-order-lag rotors (Eq. 6 with equal up and
down coefficients and no quadratic term), no linear drag and no rotor inertia.
Terms that are identically zero in that configuration are not evaluated.
Everything that depends on parameters alone (1/m, 1/J, the mixer's inverse
matrix, m g, products of gains) is a host-side constant: operations between
plain Python floats are not counted; operations that touch a per-drone value
are.  Each formula is evaluated as written: the controller and every
derivative evaluation compute R(q) afresh; nothing is shared across them.

Counted per drone-step (``count(...)``):
  flop  additions, subtractions, multiplications and divisions (1 each; a
        fused multiply-add in executed code is its multiply and its add, 2)
  mufu  sqrt, sin, cos, exp, log (special-function unit)
  cmp   comparisons, min / max and clipping (not floating-point arithmetic)

The attitude command decode (angles, desired rotation, thrust) runs once per
command block and is amortised over the block's `hold` steps.  The restated
step returns the same state as the FP64 oracle's step (checked in
tests/test_flopcount.py), so the count is of the method's arithmetic and not of
a simplified model.  Run ``python flopcount.py`` for the table.
"""
from __future__ import annotations

import math

# --------------------------------------------------------------------------- counting scalar


class Tally:
    def __init__(self):
        self.flop = 0
        self.mufu = 0
        self.cmp = 0


_T = Tally()


def _v(x):
    return x.v if isinstance(x, Num) else x


class Num:
    """A per-drone float64 value whose arithmetic is tallied in the active Tally."""
    __slots__ = ("v",)

    def __init__(self, v: float):
        self.v = float(v)

    def _op(self, o, f):
        _T.flop += 1
        return Num(f(self.v, _v(o)))

    def __add__(self, o):
        return self._op(o, lambda a, b: a + b)

    def __radd__(self, o):
        return self._op(o, lambda a, b: b + a)

    def __sub__(self, o):
        return self._op(o, lambda a, b: a - b)

    def __rsub__(self, o):
        return self._op(o, lambda a, b: b - a)

    def __mul__(self, o):
        return self._op(o, lambda a, b: a * b)

    def __rmul__(self, o):
        return self._op(o, lambda a, b: b * a)

    def __truediv__(self, o):
        return self._op(o, lambda a, b: a / b)

    def __rtruediv__(self, o):
        return self._op(o, lambda a, b: b / a)

    def __neg__(self):  # a sign flip folds into the consuming instruction
        return Num(-self.v)

    def __ge__(self, o):
        _T.cmp += 1
        return self.v >= _v(o)


def sqrt(x):
    _T.mufu += 1
    return Num(math.sqrt(_v(x)))


def sin(x):
    _T.mufu += 1
    return Num(math.sin(_v(x)))


def cos(x):
    _T.mufu += 1
    return Num(math.cos(_v(x)))


def clip(x, lo, hi):
    _T.cmp += 2
    return Num(min(max(_v(x), lo), hi))


# --------------------------------------------------------------------------- the restated step

# X configuration: rotor i at (sx_i a, sy_i a), drag counter-torque sign s_i.
SX = (1.0, -1.0, -1.0, 1.0)
SY = (-1.0, -1.0, 1.0, 1.0)
SYAW = (-1.0, 1.0, -1.0, 1.0)


def quat_to_rot(q):
    x, y, z, w = q
    ww, xx, yy, zz = w * w, x * x, y * y, z * z
    xy, wz, xz, wy, yz, wx = x * y, w * z, x * z, w * y, y * z, w * x
    return ((ww + xx - yy - zz, 2.0 * (xy - wz), 2.0 * (xz + wy)),
            (2.0 * (xy + wz), ww - xx + yy - zz, 2.0 * (yz - wx)),
            (2.0 * (xz - wy), 2.0 * (yz + wx), ww - xx - yy + zz))


def euler_to_rot(r, p, y):
    """Rz(y) Ry(p) Rx(r)."""
    cr, sr, cp, sp, cy, sy = cos(r), sin(r), cos(p), sin(p), cos(y), sin(y)
    csp, ssp = cy * sp, sy * sp
    return ((cy * cp, csp * sr - sy * cr, csp * cr + sy * sr),
            (sy * cp, ssp * sr + cy * cr, ssp * cr - cy * sr),
            (-sp, cp * sr, cp * cr))


def mixer_inverse(P) -> list:
    """Host constant: the inverse of the wrench map [T, tx, ty, tz] = A f."""
    import numpy as np
    a = P["arm"] / math.sqrt(2.0)
    A = np.array([[1.0] * 4, [s * a for s in SY], [-s * a for s in SX],
                  [s * P["km"] / P["kf"] for s in SYAW]])
    return np.linalg.inv(A).tolist()


def decode(a, P):
    """Attitude command: angles a * max_angle, R_d = Rz Ry Rx, T_d = m g (1 + s a4)."""
    a = [clip(ai, -1.0, 1.0) for ai in a]
    ang = [a[j] * P["max_angle"] for j in range(3)]
    Rd = euler_to_rot(*ang)
    Td = (1.0 + P["thrust_scale"] * a[3]) * (P["mass"] * P["g"])
    return ang, Rd, Td


def attitude_controller(x, Rd, Td, P, Ainv):
    """Geometric attitude PD, mixer and rotor-speed commands."""
    R = quat_to_rot(x[3:7])
    # M = R_d^T R; e_R = 1/2 vee(M - M^T) needs its six off-diagonal entries
    M = {}
    for i, j in ((2, 1), (1, 2), (0, 2), (2, 0), (1, 0), (0, 1)):
        M[i, j] = Rd[0][i] * R[0][j] + Rd[1][i] * R[1][j] + Rd[2][i] * R[2][j]
    eR = (0.5 * (M[2, 1] - M[1, 2]), 0.5 * (M[0, 2] - M[2, 0]), 0.5 * (M[1, 0] - M[0, 1]))
    w = x[10:13]
    KR = (P["KR_x"], P["KR_y"], P["KR_z"])
    Kw = (P["Kw_x"], P["Kw_y"], P["Kw_z"])
    J = (P["Jx"], P["Jy"], P["Jz"])
    tau = [(-KR[k] * eR[k] - Kw[k] * w[k]) * J[k] for k in range(3)]
    wrench = [Td] + tau
    fmax = P["kf"] * P["omega_max"] ** 2
    Wc = []
    for i in range(4):
        f = Ainv[i][0] * wrench[0] + Ainv[i][1] * wrench[1] + Ainv[i][2] * wrench[2] + Ainv[i][3] * wrench[3]
        f = clip(f, 0.0, fmax)
        Wc.append(sqrt(f * (1.0 / P["kf"])))
    return Wc


def deriv_fp(x, Wc, P):
    """Eqs. 1-4 and the lag form of Eq. 6 (no drag, no rotor inertia)."""
    q, v, w, W = x[3:7], x[7:10], x[10:13], x[13:17]
    R = quat_to_rot(q)
    W2 = [Wi * Wi for Wi in W]
    f = [P["kf"] * W2i for W2i in W2]
    T = f[0] + f[1] + f[2] + f[3]
    a = P["arm"] / math.sqrt(2.0)
    tx = (-f[0] - f[1] + f[2] + f[3]) * a
    ty = -(f[0] - f[1] - f[2] + f[3]) * a
    tz = (-W2[0] + W2[1] - W2[2] + W2[3]) * P["km"]
    Tm = T * (1.0 / P["mass"])
    v_dot = (R[0][2] * Tm, R[1][2] * Tm, R[2][2] * Tm - P["g"])
    J = (P["Jx"], P["Jy"], P["Jz"])
    Jw = (J[0] * w[0], J[1] * w[1], J[2] * w[2])
    c = (w[1] * Jw[2] - w[2] * Jw[1], w[2] * Jw[0] - w[0] * Jw[2], w[0] * Jw[1] - w[1] * Jw[0])
    w_dot = ((tx - c[0]) * (1.0 / J[0]), (ty - c[1]) * (1.0 / J[1]), (tz - c[2]) * (1.0 / J[2]))
    qx, qy, qz, qw = q
    wx, wy, wz = w
    q_dot = (0.5 * (qw * wx + qy * wz - qz * wy), 0.5 * (qw * wy - qx * wz + qz * wx),
             0.5 * (qw * wz + qx * wy - qy * wx), 0.5 * (-qx * wx - qy * wy - qz * wz))
    cv = P["cv_up"]
    W_dot = [cv * (Wc[i] - W[i]) for i in range(4)]
    return list(v) + list(q_dot) + list(v_dot) + list(w_dot) + W_dot


def deriv_abs(x, ang, Td, P):
    """Eqs. 7-10 (no drag): only the third column of R(Psi) enters."""
    r, p, y = x[3:6]
    cr, sr, cp, sp, cy, sy = cos(r), sin(r), cos(p), sin(p), cos(y), sin(y)
    col = ((cy * sp) * cr + sy * sr, (sy * sp) * cr - cy * sr, cp * cr)
    fm = x[12] * (P["c_f"] / P["mass"])
    v_dot = (col[0] * fm, col[1] * fm, col[2] * fm - P["g"])
    c1 = (P["c1_r"], P["c1_p"], P["c1_y"])
    c2 = (P["c2_r"], P["c2_p"], P["c2_y"])
    c3 = (P["c3_r"], P["c3_p"], P["c3_y"])
    psi_dd = [c1[k] * x[3 + k] + c2[k] * x[9 + k] + c3[k] * ang[k] for k in range(3)]
    fs_dot = P["c_tau"] * (Td - x[12])
    return list(x[6:9]) + list(x[9:12]) + list(v_dot) + psi_dd + [fs_dot]


def integrate(f, x, dt, rk4: bool):
    if not rk4:
        k = f(x)
        return [x[i] + dt * k[i] for i in range(len(x))]
    h = 0.5 * dt
    k1 = f(x)
    k2 = f([x[i] + h * k1[i] for i in range(len(x))])
    k3 = f([x[i] + h * k2[i] for i in range(len(x))])
    k4 = f([x[i] + dt * k3[i] for i in range(len(x))])
    c = dt / 6.0
    return [x[i] + c * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) for i in range(len(x))]


def renormalise(q):
    n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
    return [qi / n for qi in q]


def step_fp(x20, a, P, dt, rk4, Ainv, decoded=None):
    """One first-principles step under the attitude interface; x20 = p q v w W I."""
    _, Rd, Td = decode(a, P) if decoded is None else decoded
    x = x20[:17]
    Wc = attitude_controller(x, Rd, Td, P, Ainv)
    y = integrate(lambda s: deriv_fp(s, Wc, P), x, dt, rk4)
    return y[0:3] + renormalise(y[3:7]) + y[7:17] + list(x20[17:20])


def step_abs(x20, a, P, dt, rk4, decoded=None):
    """One abstracted-model step under the attitude interface."""
    ang, _, Td = decode(a, P) if decoded is None else decoded
    y = integrate(lambda s: deriv_abs(s, ang, Td, P), x20[:13], dt, rk4)
    return y + list(x20[13:20])


# --------------------------------------------------------------------------- counts


def _count(fn) -> dict:
    global _T
    saved, _T = _T, Tally()
    try:
        fn()
        return {"flop": _T.flop, "mufu": _T.mufu, "cmp": _T.cmp}
    finally:
        _T = saved


def _sample_state(model: str):
    """A representative in-flight state (branch decisions do not change counts)."""
    if model == "fp":
        q = [0.1, -0.05, 0.2, 0.0]
        q[3] = math.sqrt(1.0 - sum(c * c for c in q[:3]))
        return [Num(v) for v in [0.1, -0.2, 1.0] + q + [0.3, -0.1, 0.2, 0.5, -0.4, 0.1]
                + [14000.0, 14500.0, 14200.0, 14800.0] + [0.0, 0.0, 0.0]]
    return [Num(v) for v in [0.1, -0.2, 1.0, 0.1, -0.05, 0.3, 0.2, 0.1, -0.3, 0.4, -0.2, 0.1, 0.26]
            + [0.0] * 7]


def count(model: str, integrator: str, hold: int = 50, params=None) -> dict:
    """Per-drone-step counts for model "fp" or "abs", integrator "euler" or
    "rk4", attitude interface, commands held for `hold` steps."""
    import workloads as W
    P = W.crazyflie_params() if params is None else params
    rk4 = integrator == "rk4"
    dt = 1.0 / 500
    a = [Num(0.2), Num(-0.3), Num(0.1), Num(0.25)]
    x = _sample_state(model)
    Ainv = mixer_inverse(P)
    dec = decode(a, P)
    c_dec = _count(lambda: decode(a, P))
    if model == "fp":
        c_step = _count(lambda: step_fp(x, a, P, dt, rk4, Ainv, decoded=dec))
    else:
        c_step = _count(lambda: step_abs(x, a, P, dt, rk4, decoded=dec))
    out = {k: c_step[k] + c_dec[k] / hold for k in c_step}
    out["decode_per_block"] = c_dec
    out["step_without_decode"] = c_step
    return out


# The benchmark workloads' steps (attitude interface, commands held 50 steps).
def table() -> dict:
    return {(m, i): count(m, i) for m, i in (("fp", "rk4"), ("fp", "euler"), ("abs", "euler"),
                                             ("abs", "rk4"))}


def sampling_step() -> dict:
    """One sampled RK4 step of the MPPI rollouts: the action decode every step,
    the noise (Box-Muller on two Philox word pairs: 2 log, 2 sqrt, 2 sin/cos
    pairs and their scaling), the action clip(nominal + sigma xi), the step and
    the goal distance.  Obstacle terms of obstacles beyond a drone's reach are
    exact zeros and are not counted (the kernel skips them); Philox's integer
    rounds are not floating-point work."""
    import workloads as W
    P = W.crazyflie_params()
    x = _sample_state("fp")
    Ainv = mixer_inverse(P)
    xi = [Num(0.3), Num(-1.1), Num(0.7), Num(0.05)]
    g = (0.5, 0.5, 1.5)

    def one():
        # Box-Muller: r = sqrt(-2 ln u1), angle 2 pi u2 - pi, z = -r cos, -r sin (per pair)
        for _ in range(2):
            u2 = Num(0.7)
            _T.mufu += 1  # ln u1
            ln_u1 = Num(math.log(0.3))
            r = sqrt(-2.0 * ln_u1)
            ang = 2.0 * math.pi * u2 - math.pi
            c, s = cos(ang), sin(ang)
            _ = (-r * c, -r * s)
        act = [clip(0.0 + 0.2 * xi[j], -1.0, 1.0) for j in range(4)]
        y = step_fp(x, act, P, 1.0 / 500, True, Ainv)
        ex, ey, ez = y[0] - g[0], y[1] - g[1], y[2] - g[2]
        _ = sqrt(ex * ex + ey * ey + ez * ez)
    return _count(one)


if __name__ == "__main__":
    for (m, i), c in table().items():
        print(f"{m:3s} {i:5s} attitude: {c['flop']:.1f} flop, {c['mufu']:.2f} MUFU, {c['cmp']:.1f} cmp "
              f"per drone-step (step {c['step_without_decode']}, decode {c['decode_per_block']} per block)")
    print("sampling rk4 step:", sampling_step())
