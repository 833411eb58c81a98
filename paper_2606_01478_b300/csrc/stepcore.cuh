// One drone step shared by the fused step kernels and the sampling kernel:
// controller (held over the step) -> derivative -> Euler or RK4 -> quaternion
// renormalisation.
#pragma once

#include "physics.cuh"

namespace cf {

// Controller state held between command-block changes.
struct CtrlHold {
  float Rd[9];
  float Td;
  float Wc[4];       // rotor-speed interface: clipped commands
  float4 sp;         // position interface: setpoint
  float syaw, cyaw;  // position interface: yaw sine/cosine
  float u[4];        // abstracted model input
};

template <int MODEL, int CTRL>
__device__ __forceinline__ void decode_command(float4 c, const DevParams& P, CtrlHold& h) {
  if constexpr (MODEL != SIM_FIRST_PRINCIPLES) {
    abstracted_command(c, P, h.u);
  } else if constexpr (CTRL == SIM_CTRL_TORQUE) {
    h.Td = c.x;
    h.sp = c;  // body torque in (y, z, w)
  } else if constexpr (CTRL == SIM_CTRL_ATTITUDE) {
    attitude_command(c, P, h.Rd, h.Td);
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

template <int MODEL, int INTEG, int CTRL, int MOTOR>
__device__ __forceinline__ void one_step(float* s, const CtrlHold& h, const DevParams& P, bool drag,
                                         float dt) {
  constexpr int D = (MODEL == SIM_FIRST_PRINCIPLES) ? 17 : 13;
  float Wc[4];
  float ep[3] = {0.f, 0.f, 0.f};
  float R[9];  // R(q) of the state at the start of the step (controller and first stage)
  if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
    quat_rot(s[3], s[4], s[5], s[6], R);
    if constexpr (CTRL == SIM_CTRL_ROTOR_SPEED) {
#pragma unroll
      for (int r = 0; r < 4; ++r) Wc[r] = h.Wc[r];
    } else if constexpr (CTRL == SIM_CTRL_TORQUE) {
      mixer<MOTOR>(h.Td, h.sp.y, h.sp.z, h.sp.w, P, Wc);
    } else {
      float tx, ty, tz;
      if constexpr (CTRL == SIM_CTRL_POSITION) {
        float Rd[9], Td;
        position_command(s, R, h.sp, h.syaw, h.cyaw, P, Rd, Td, ep);
        attitude_torque(R, Rd, s[10], s[11], s[12], P, tx, ty, tz);
        mixer<MOTOR>(Td, tx, ty, tz, P, Wc);
      } else {
        attitude_torque(R, h.Rd, s[10], s[11], s[12], P, tx, ty, tz);
        mixer<MOTOR>(h.Td, tx, ty, tz, P, Wc);
      }
    }
  }
  auto deriv = [&](const float* x, float* d, const float* Rx) {
    if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
      deriv_fp<MOTOR>(x, Wc, P, drag, d, Rx);
    } else if constexpr (MODEL == SIM_ABSTRACTED) {
      deriv_abs<MOTOR>(x, h.u, P, drag, d);
    } else {
      deriv_abs_nothrust(x, h.u, P, d);
    }
  };
  const float* R0 = (MODEL == SIM_FIRST_PRINCIPLES) ? R : nullptr;
  if constexpr (INTEG == SIM_EULER) {
    float d[D];
    deriv(s, d, R0);
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = fmaf(dt, d[j], s[j]);
  } else {
    float k[D], acc[D], xs[D];
    const float h2 = 0.5f * dt, h6 = dt * (1.f / 6.f);
    deriv(s, k, R0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      acc[j] = k[j];
      xs[j] = fmaf(h2, k[j], s[j]);
    }
    deriv(xs, k, nullptr);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      acc[j] = fmaf(2.f, k[j], acc[j]);
      xs[j] = fmaf(h2, k[j], s[j]);
    }
    deriv(xs, k, nullptr);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      acc[j] = fmaf(2.f, k[j], acc[j]);
      xs[j] = fmaf(dt, k[j], s[j]);
    }
    deriv(xs, k, nullptr);
#pragma unroll
    for (int j = 0; j < D; ++j) s[j] = fmaf(h6, acc[j] + k[j], s[j]);
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
