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
  const float v2 = fmaf(fmd, r22, fmaf(-dt, P.g, s[8]));
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
  constexpr int D = (MODEL == SIM_FIRST_PRINCIPLES) ? 17 : 13;
  constexpr bool LSF = lag_step_form<MODEL, MOTOR>();
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
  // integrator coefficient c for element j (halved for q in the lag step form)
  auto co = [&](int j, float c) { return (LSF && j >= 3 && j <= 6) ? 0.5f * c : c; };
  // Element-wise integrator arithmetic runs on element pairs (2i, 2i + 1) with the
  // packed FP32 instructions (two lanes per instruction, each lane rounded as its
  // scalar counterpart); D is odd, so element D - 1 is scalar.
  constexpr int DP = D - 1;
  auto c2 = [&](int j, float c) { return make_float2(co(j, c), co(j + 1, c)); };
  auto pr = [](const float* a, int j) { return make_float2(a[j], a[j + 1]); };
  auto put = [](float* a, int j, float2 v) {
    a[j] = v.x;
    a[j + 1] = v.y;
  };
  if constexpr (INTEG == SIM_EULER) {
    float d[D];
    deriv(s, d, R0);
#pragma unroll
    for (int j = 0; j < DP; j += 2) put(s, j, __ffma2_rn(c2(j, dt), pr(d, j), pr(s, j)));
    s[DP] = fmaf(dt, d[DP], s[DP]);
  } else {
    // classic RK4; in the lag step form the rotor speeds (13..16) take the
    // closed-form update and need no stage accumulator
    constexpr int NA = LSF ? 13 : D;  // elements with an RK4 accumulator
    float k[D], acc[D], xs[D], k1W[4];
    const float h2 = 0.5f * dt, h6 = dt * (1.f / 6.f);
    const float2 two = make_float2(2.f, 2.f);
    deriv(s, k, R0);
#pragma unroll
    for (int j = 0; j < DP; j += 2) {
      put(acc, j, pr(k, j));
      put(xs, j, __ffma2_rn(c2(j, h2), pr(k, j), pr(s, j)));
    }
    acc[DP] = k[DP];
    xs[DP] = fmaf(h2, k[DP], s[DP]);
    if constexpr (LSF) {
#pragma unroll
      for (int r = 0; r < 4; ++r) k1W[r] = k[13 + r];
    }
#pragma unroll
    for (int st = 0; st < 2; ++st) {
      deriv(xs, k, nullptr);
      const float c = st == 0 ? h2 : dt;
#pragma unroll
      for (int j = 0; j < DP; j += 2) {
        if (j < NA) put(acc, j, __ffma2_rn(two, pr(k, j), pr(acc, j)));
        put(xs, j, __ffma2_rn(c2(j, c), pr(k, j), pr(s, j)));
      }
      if (DP < NA) acc[DP] = fmaf(2.f, k[DP], acc[DP]);
      xs[DP] = fmaf(c, k[DP], s[DP]);
    }
    deriv(xs, k, nullptr);
    if constexpr (LSF) {
#pragma unroll
      for (int j = 0; j < 12; j += 2)
        put(s, j, __ffma2_rn(c2(j, h6), __fadd2_rn(pr(acc, j), pr(k, j)), pr(s, j)));
      s[12] = fmaf(h6, acc[12] + k[12], s[12]);
      // (1 - P4(-h)) / cv = dt (1 - h/2 + h^2/6 - h^3/24), h = cv dt
      const float hc = -P.ncv * dt;
      const float c4 = dt * fmaf(hc, fmaf(hc, fmaf(hc, -1.f / 24.f, 1.f / 6.f), -0.5f), 1.f);
      s[13] = fmaf(c4, k1W[0], s[13]);
      put(s, 14, __ffma2_rn(make_float2(c4, c4), make_float2(k1W[1], k1W[2]), pr(s, 14)));
      s[16] = fmaf(c4, k1W[3], s[16]);
    } else {
#pragma unroll
      for (int j = 0; j < DP; j += 2)
        put(s, j, __ffma2_rn(c2(j, h6), __fadd2_rn(pr(acc, j), pr(k, j)), pr(s, j)));
      s[DP] = fmaf(h6, acc[DP] + k[DP], s[DP]);
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
