// One drone step shared by the fused step kernels and the sampling kernel:
// controller (held over the step) -> derivative -> Euler or RK4 -> quaternion
// renormalisation.
#pragma once

#include "physics.cuh"

namespace cf {

// Controller state held between command-block changes.
struct CtrlHold {
  float qd[4];       // attitude interface: twice the desired quaternion (attitude_command_q)
  float Td;
  float Wc[4];       // rotor-speed interface: clipped commands
  float4 sp;         // position interface: setpoint
  float syaw, cyaw;  // position interface: yaw sine/cosine
  float u[4];        // abstracted model input
  float cu[4];       // abstracted model: its command terms (abstracted_command)
};

template <int MODEL, int CTRL>
__device__ __forceinline__ void decode_command(float4 c, const DevParams& P, CtrlHold& h) {
  if constexpr (MODEL != SIM_FIRST_PRINCIPLES) {
    abstracted_command<MODEL == SIM_ABSTRACTED>(c, P, h.u, h.cu);
  } else if constexpr (CTRL == SIM_CTRL_TORQUE) {
    h.Td = c.x;
    h.sp = c;  // body torque in (y, z, w)
  } else if constexpr (CTRL == SIM_CTRL_ATTITUDE) {
    attitude_command_q(c, P, h.qd, h.Td);
  } else if constexpr (CTRL == SIM_CTRL_POSITION) {
    h.sp = c;
    __sincosf(c.w, &h.syaw, &h.cyaw);
  } else {
    h.Wc[0] = clampf(c.x, 0.f, P.omega_max);
    h.Wc[1] = clampf(c.y, 0.f, P.omega_max);
    h.Wc[2] = clampf(c.z, 0.f, P.omega_max);
    h.Wc[3] = clampf(c.w, 0.f, P.omega_max);
  }
}

// Lag-rotor step form (first-principles model with MOTOR_LAG): rotor commands
// are carried as rates u = cv W_cmd, the derivative returns 2 q' (deriv_fp_rate)
// and the integrator takes half coefficients for q.  Under RK4 the rotor
// speeds, whose ODE W' = u - cv W is linear with u held, take the RK4 update in
// closed form: W + k1 (1 - P4(-h)) / cv, P4 the degree-4 Taylor polynomial of
// exp, h = cv dt -- equal to the four-stage combination in exact arithmetic.
template <int MODEL, int MOTOR>
constexpr bool lag_step_form() {
  return MODEL == SIM_FIRST_PRINCIPLES && MOTOR == MOTOR_LAG;
}

// Explicit Euler step of the abstracted model without drag (Eqs. 7-10), s + dt
// f(s), with the step size folded into the linear terms (equal in exact
// arithmetic; cu as for deriv_abs):
//   p' = p + dt v,   Psi' = Psi + dt Psidot,
//   v' = v + (dt c_f f / m) R(Psi) e3 - dt g e3,
//   Psidot' = (dt c1) Psi + (1 + dt c2) Psidot + dt cu_Psi,
//   f' = (1 - dt c_tau) f + dt cu_f.
// Every right-hand side reads the state at the start of the step.  Element pairs
// go through the packed FP32 instructions (each lane rounded as its scalar form).
__device__ __forceinline__ void euler_abs(float* s, const float cu[4], const DevParams& P, float dt) {
  float sr, cr, sp, cp, sy, cy;
  __sincosf(s[3], &sr, &cr);
  __sincosf(s[4], &sp, &cp);
  __sincosf(s[5], &sy, &cy);
  // third column of Rz Ry Rx
  const float r02 = fmaf(cy * sp, cr, sy * sr);
  const float r12 = fmaf(sy * sp, cr, -cy * sr);
  const float r22 = cp * cr;
  const float fmd = (dt * P.cf_inv_m) * s[12];
  const float2 dt2 = make_float2(dt, dt);
  const float x3 = s[3];
  const float2 x45 = make_float2(s[4], s[5]);
  const float2 p01 = __ffma2_rn(dt2, make_float2(s[6], s[7]), make_float2(s[0], s[1]));
  const float2 p23 = __ffma2_rn(dt2, make_float2(s[8], s[9]), make_float2(s[2], s[3]));
  const float2 p45 = __ffma2_rn(dt2, make_float2(s[10], s[11]), x45);
  const float2 v01 = __ffma2_rn(make_float2(fmd, fmd), make_float2(r02, r12), make_float2(s[6], s[7]));
  // vertical: thrust and gravity nearly cancel near hover, so their sum is formed
  // (one rounding) before it is added to v
  const float v2 = s[8] + fmaf(fmd, r22, -dt * P.g);
  const float w0 = fmaf(dt * P.c1_r, x3, fmaf(fmaf(dt, P.c2_r, 1.f), s[9], dt * cu[0]));
  const float2 w12 = __ffma2_rn(make_float2(dt * P.c1_p, dt * P.c1_y), x45,
                                __ffma2_rn(make_float2(fmaf(dt, P.c2_p, 1.f), fmaf(dt, P.c2_y, 1.f)),
                                           make_float2(s[10], s[11]),
                                           make_float2(dt * cu[1], dt * cu[2])));
  const float f = fmaf(fmaf(-dt, P.c_tau, 1.f), s[12], dt * cu[3]);
  s[0] = p01.x;
  s[1] = p01.y;
  s[2] = p23.x;
  s[3] = p23.y;
  s[4] = p45.x;
  s[5] = p45.y;
  s[6] = v01.x;
  s[7] = v01.y;
  s[8] = v2;
  s[9] = w0;
  s[10] = w12.x;
  s[11] = w12.y;
  s[12] = f;
}

// Explicit Euler step of the first-principles model (Eqs. 1-6) under the attitude
// interface with lag rotors, s + dt f(s), with the step size folded into the
// constant of each term (equal in exact arithmetic; constants as in
// deriv_fp_rate and attitude_mixer_rate_e):
//   dt u_i = sqrt(clip(dt^2 f_i))    the step-form mixer on dt^2-scaled gains
//   W' = (1 - dt cv) W + dt u,       v' = v + (dt kf / m) S R e3 - dt g e3,
//   q' = q + q (x) [dt w / 2, 0],    w' = w + dt J^-1 (tau - w x J w),
// then the quaternion renormalisation.  Every right-hand side reads the state at
// the start of the step.  SYM_XY as for deriv_fp_rate.
template <bool SYM_XY>
__device__ __forceinline__ void euler_fp_lag_attitude(float* s, const CtrlHold& h, const DevParams& P,
                                                      float dt) {
  const float qx = s[3], qy = s[4], qz = s[5], qw = s[6];
  const float wx = s[10], wy = s[11], wz = s[12];
  // controller and mixer: 2 e_R from quaternions, dt u from dt^2-scaled gains
  float ex, ey, ez;
  attitude_error2_q(s, h.qd, ex, ey, ez);
  const float d2 = dt * dt;
  // products that feed an addition are rounded on their own (__fmul_rn), so that
  // no launch shape contracts them differently (fused and single-step launches
  // give the same state bit for bit)
  const float A = __fmul_rn(d2 * P.cA, h.Td);
  const float X = -fmaf(d2 * P.cRx, ex, (d2 * P.cwx) * wx);
  const float Y = -fmaf(d2 * P.cRy, ey, (d2 * P.cwy) * wy);
  const float Z = -fmaf(d2 * P.cRz, ez, (d2 * P.cwz) * wz);
  const float um = d2 * P.u2max;
  const float du0 = sqrt_approx(clampf((A - X) - (Y + Z), 0.f, um));
  const float du1 = sqrt_approx(clampf((A - X) + (Y + Z), 0.f, um));
  const float du2 = sqrt_approx(clampf((A + X) + (Y - Z), 0.f, um));
  const float du3 = sqrt_approx(clampf((A + X) - (Y - Z), 0.f, um));
  // rotor-square sums of the wrench (deriv_fp_rate)
  const float W0 = s[13], W1 = s[14], W2 = s[15], W3 = s[16];
  const float s0 = W0 * W0, s2 = W2 * W2;
  const float a01 = fmaf(W1, W1, s0), a23 = fmaf(W3, W3, s2), S = a01 + a23;
  const float e10 = fmaf(W1, W1, -s0), e32 = fmaf(W3, W3, -s2);
  // translation
  const float Tmd = (dt * P.kfm) * S, Tm2d = (dt * P.kfm2) * S;
  // scalar multiply-adds: as packed pairs (operands in aligned register pairs) they
  // measured slower
  const float p0 = fmaf(dt, s[7], s[0]), p1 = fmaf(dt, s[8], s[1]), p2 = fmaf(dt, s[9], s[2]);
  const float v0 = fmaf(Tm2d, fmaf(qx, qz, qw * qy), s[7]);
  const float v1 = fmaf(Tm2d, fmaf(qy, qz, -qw * qx), s[8]);
  // vertical: thrust and gravity summed first, as for the abstracted model
  const float v2 = s[9] + fmaf(Tmd, fmaf(qw, qw, __fmul_rn(qz, qz)) - fmaf(qx, qx, __fmul_rn(qy, qy)),
                               -dt * P.g);
  // attitude: q (x) [h, 0] with h = dt w / 2
  const float hd = 0.5f * dt;
  const float hx = hd * wx, hy = hd * wy, hz = hd * wz;
  const float nqx = fmaf(qw, hx, fmaf(qy, hz, fmaf(-qz, hy, qx)));
  const float nqy = fmaf(qw, hy, fmaf(qz, hx, fmaf(-qx, hz, qy)));
  const float nqz = fmaf(qw, hz, fmaf(qx, hy, fmaf(-qy, hx, qz)));
  const float nqw = fmaf(-qx, hx, fmaf(-qy, hy, fmaf(-qz, hz, qw)));
  // body rates: roll (s2 + s3) - (s0 + s1), pitch e10 - e32, yaw e10 + e32
  float nwx, nwy, nwz;
  if constexpr (SYM_XY) {
    const float t = (dt * P.cJx) * wz;
    nwx = fmaf(dt * P.kfaJx, a23 - a01, fmaf(t, wy, wx));
    nwy = fmaf(dt * P.kfaJy, e10 - e32, fmaf(-t, wx, wy));
    nwz = fmaf(dt * P.kmJz, e10 + e32, wz);
  } else {
    nwx = fmaf(dt * P.kfaJx, a23 - a01, fmaf((dt * P.cJx) * wy, wz, wx));
    nwy = fmaf(dt * P.kfaJy, e10 - e32, fmaf((dt * P.cJy) * wz, wx, wy));
    nwz = fmaf(dt * P.kmJz, e10 + e32, fmaf((dt * P.cJz) * wx, wy, wz));
  }
  // rotors (ncv = -cv)
  const float ar = fmaf(dt, P.ncv, 1.f);
  const float nW0 = fmaf(ar, W0, du0), nW1 = fmaf(ar, W1, du1);
  const float nW2 = fmaf(ar, W2, du2), nW3 = fmaf(ar, W3, du3);
  const float in = rsqrt_approx(fmaf(nqx, nqx, fmaf(nqy, nqy, fmaf(nqz, nqz, nqw * nqw))));
  s[0] = p0;
  s[1] = p1;
  s[2] = p2;
  s[3] = nqx * in;
  s[4] = nqy * in;
  s[5] = nqz * in;
  s[6] = nqw * in;
  s[7] = v0;
  s[8] = v1;
  s[9] = v2;
  s[10] = nwx;
  s[11] = nwy;
  s[12] = nwz;
  s[13] = nW0;
  s[14] = nW1;
  s[15] = nW2;
  s[16] = nW3;
}

// SYM_XY (lag step form only): Jx = Jy, the yaw rate's gyroscopic term left out.
template <int MODEL, int INTEG, int CTRL, int MOTOR, bool SYM_XY = false>
__device__ __forceinline__ void one_step(float* s, const CtrlHold& h, const DevParams& P, bool drag,
                                         float dt) {
  if constexpr (INTEG == SIM_EULER && MODEL == SIM_ABSTRACTED) {
    if (MOTOR == MOTOR_LAG || !drag) {  // drag exists only with general motors
      euler_abs(s, h.cu, P, dt);
      return;
    }
  }
  constexpr bool LSF = lag_step_form<MODEL, MOTOR>();
  if constexpr (INTEG == SIM_EULER && LSF && CTRL == SIM_CTRL_ATTITUDE) {
    euler_fp_lag_attitude<SYM_XY>(s, h, P, dt);
    return;
  }
  constexpr int D = (MODEL == SIM_FIRST_PRINCIPLES) ? 17 : 13;
  float Wc[4];  // rotor-speed commands (rates cv W_cmd in the lag step form)
  float ep[3] = {0.f, 0.f, 0.f};
  // R(q) of the state at the start of the step: the position controller's
  // matrices; the first derivative stage reads its third column.  The attitude
  // interface forms its error from quaternions instead and every stage takes the
  // thrust direction from q.
  float R[9];
  constexpr bool NEED_R = MODEL == SIM_FIRST_PRINCIPLES && CTRL == SIM_CTRL_POSITION;
  if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
    if constexpr (NEED_R) quat_rot(s[3], s[4], s[5], s[6], R);
    if constexpr (CTRL == SIM_CTRL_ROTOR_SPEED) {
#pragma unroll
      for (int r = 0; r < 4; ++r) Wc[r] = LSF ? -P.ncv * h.Wc[r] : h.Wc[r];
    } else if constexpr (CTRL == SIM_CTRL_TORQUE) {
      if constexpr (LSF) {
        mixer_rate(h.Td, h.sp.y * P.cXt, h.sp.z * P.cXt, h.sp.w * P.cZt, P, Wc);
      } else {
        mixer<MOTOR>(h.Td, h.sp.y, h.sp.z, h.sp.w, P, Wc);
      }
    } else if constexpr (CTRL == SIM_CTRL_ATTITUDE) {
      float ex, ey, ez;
      attitude_error2_q(s, h.qd, ex, ey, ez);
      if constexpr (LSF) {
        attitude_mixer_rate_e(ex, ey, ez, h.Td, s[10], s[11], s[12], P, Wc);
      } else {
        float tx, ty, tz;
        attitude_torque_e(ex, ey, ez, s[10], s[11], s[12], P, tx, ty, tz);
        mixer<MOTOR>(h.Td, tx, ty, tz, P, Wc);
      }
    } else {
      float Rd[9], Td;
      position_command(s, R, h.sp, h.syaw, h.cyaw, P, Rd, Td, ep);
      if constexpr (LSF) {
        attitude_mixer_rate(R, Rd, Td, s[10], s[11], s[12], P, Wc);
      } else {
        float tx, ty, tz;
        attitude_torque(R, Rd, s[10], s[11], s[12], P, tx, ty, tz);
        mixer<MOTOR>(Td, tx, ty, tz, P, Wc);
      }
    }
  }
  auto deriv = [&](const float* x, float* d, const float* Rx) {
    if constexpr (LSF) {
      deriv_fp_rate<SYM_XY>(x, Wc, P, d, Rx);
    } else if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
      deriv_fp<MOTOR>(x, Wc, P, drag, d, Rx);
    } else if constexpr (MODEL == SIM_ABSTRACTED) {
      deriv_abs<MOTOR>(x, h.cu, P, drag, d);
    } else {
      deriv_abs_nothrust(x, h.cu, P, d);
    }
  };
  const float* R0 = NEED_R ? R : nullptr;
  // integrator coefficient c for element j (halved for q in the lag step form).
  // The element-wise arithmetic is scalar: as packed FP32 pairs (__ffma2_rn) it
  // measured slower under RK4.
  auto co = [&](int j, float c) { return (LSF && j >= 3 && j <= 6) ? 0.5f * c : c; };
  if constexpr (INTEG == SIM_EULER) {
    float d[D];
    deriv(s, d, R0);
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = fmaf(co(j, dt), d[j], s[j]);
  } else {
    // classic RK4; in the lag step form the rotor speeds (13..16) take the
    // closed-form update and need no stage accumulator
    constexpr int NA = LSF ? 13 : D;  // elements with an RK4 accumulator
    float k[D], acc[D], xs[D], k1W[4];
    const float h2 = 0.5f * dt, h6 = dt * (1.f / 6.f);
    deriv(s, k, R0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      if (j < NA) acc[j] = k[j];
      xs[j] = fmaf(co(j, h2), k[j], s[j]);
    }
    if constexpr (LSF) {
#pragma unroll
      for (int r = 0; r < 4; ++r) k1W[r] = k[13 + r];
    }
#pragma unroll
    for (int st = 0; st < 2; ++st) {
      deriv(xs, k, nullptr);
      const float c = st == 0 ? h2 : dt;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        if (j < NA) acc[j] = fmaf(2.f, k[j], acc[j]);
        xs[j] = fmaf(co(j, c), k[j], s[j]);
      }
    }
    deriv(xs, k, nullptr);
#pragma unroll
    for (int j = 0; j < NA; ++j) s[j] = fmaf(co(j, h6), acc[j] + k[j], s[j]);
    if constexpr (LSF) {
      // (1 - P4(-h)) / cv = dt (1 - h/2 + h^2/6 - h^3/24), h = cv dt
      const float hc = -P.ncv * dt;
      const float c4 = dt * fmaf(hc, fmaf(hc, fmaf(hc, -1.f / 24.f, 1.f / 6.f), -0.5f), 1.f);
#pragma unroll
      for (int r = 0; r < 4; ++r) s[13 + r] = fmaf(c4, k1W[r], s[13 + r]);
    }
  }
  if constexpr (MODEL == SIM_ABSTRACTED_NOTHRUST) s[12] = h.u[3];  // f_sum follows f_cmd at once
  if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
    const float in = rsqrt_approx(fmaf(s[3], s[3], fmaf(s[4], s[4], fmaf(s[5], s[5], s[6] * s[6]))));
    s[3] *= in;
    s[4] *= in;
    s[5] *= in;
    s[6] *= in;
    if constexpr (CTRL == SIM_CTRL_POSITION) {
      s[17] = fmaf(dt, ep[0], s[17]);
      s[18] = fmaf(dt, ep[1], s[18]);
      s[19] = fmaf(dt, ep[2], s[19]);
    }
  }
}

}  // namespace cf
