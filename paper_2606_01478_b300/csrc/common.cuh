// Device-side definitions shared by the kernels of the B300 drone step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "crazyflow.h"

namespace cf {

// Constants derived on the host (double precision, then rounded to float) from
// one user parameter vector (enum sim_param_index).  Kernels read either a
// by-value copy (kernel parameter space, so arithmetic takes the constants
// directly as constant-bank operands) or a per-world array in global memory.
struct DevParams {
  // rigid body (Eqs. 1-4): 1/m, gravity, 1/J and the Euler coupling terms
  // (Jy-Jz)/Jx, (Jz-Jx)/Jy, (Jx-Jy)/Jz of J^-1 (tau - w x J w)
  float inv_m, g, mass;
  float inv_Jx, inv_Jy, inv_Jz;
  float cJx, cJy, cJz;
  // rotors: thrust kf W^2, torque arm factor kf * arm / sqrt(2), drag torque km W^2
  float kf, kfa, km;
  // rotor dynamics, Eq. 6
  float cv_up, cd_up, cv_down, cd_down;
  // body-frame linear drag diagonal (text after Eq. 5)
  float Ca_x, Ca_y, Ca_z;
  // attitude PD: 0.5 * K_R * J (the 1/2 of e_R folded in) and K_w * J
  float KRJh_x, KRJh_y, KRJh_z;
  float KwJ_x, KwJ_y, KwJ_z;
  // position PID
  float Kp_x, Kp_y, Kp_z, Kd_x, Kd_y, Kd_z, Ki_x, Ki_y, Ki_z;
  // action map: angle = a * max_angle, T = m g + (m g thrust_scale) a4;
  // half_max_angle = max_angle / 2 (half angles of the desired quaternion)
  float max_angle, half_max_angle, mg, ts_mg;
  // mixer f_i = T/4 +- tau_x mix_a +- tau_y mix_a +- tau_z mix_k, clip [0, fmax],
  // W_cmd = sqrt(f * inv_kf)
  float mix_a, mix_k, inv_kf, fmax, omega_max;
  // abstracted model, Eqs. 8-10 (per axis roll, pitch, yaw)
  float c1_r, c1_p, c1_y, c2_r, c2_p, c2_y, c3_r, c3_p, c3_y, c_tau, cf_inv_m;
  // general rotor curves and inertia (used by the general rotor path only):
  // thrust kf W^2 + kf1 W + kf0, drag torque km W^2 + km1 W; the mixer clips
  // thrust to [kf0, fmax] and inverts W = (sqrt(kf1^2 + 4 kf (f - kf0)) - kf1) / (2 kf);
  // rotor angular momentum about z: -Jpc sum_i s_i W_i (Jpc = J_p 2 pi / 60)
  float kf0, kf1, km1, kf1sq, four_kf, inv_2kf, Jpc;
  // lag-rotor step form (one_step with MOTOR_LAG): rotor commands enter as
  // rates u = cv W_cmd, so W' = u - cv W; constants folded so that
  //   accel = (kf/m) sum W^2 along R e_z,  w' = (kfa/J) (W^2 combination) + ...,
  //   u_i = sqrt(clip(cA T + (+-X) + (+-Y) + (+-Z), 0, u2max)) with
  //   X = cRx e_Rx + cwx w_x etc. (attitude PD times mixer times cv^2 / kf) or
  //   X = cXt tau_x (torque interface)
  float kfm, kfm2, kfaJx, kfaJy, kmJz, ncv, cA, cRx, cRy, cRz, cwx, cwy, cwz, cXt, cZt, u2max;
  int flags;
};

// PF_GENERAL_MOTOR selects the general kernel variants (MOTOR_GENERAL): polynomial
// rotor curves, asymmetric or quadratic rotor dynamics, rotor inertia, or drag
// (PF_DRAG implies it).  The lag-rotor variants (MOTOR_LAG) have none of these.
// PF_ASYM_XY marks Jx != Jy: without it the yaw rate's gyroscopic term
// (Jx - Jy) wx wy / Jz is zero, and the lag-rotor variants can leave it out.
enum : int { PF_DRAG = 1, PF_GENERAL_MOTOR = 2, PF_ASYM_XY = 4 };

// Arguments of the step kernels (by value).
struct StepArgs {
  float4* planes;               // [5][n] float4, plane j = state slots 4j..4j+3
  const float4* cmd;            // [n_blocks][n] float4
  const DevParams* params;      // per parameter set (global memory)
  const int32_t* set_of_world;  // [M]
  uint32_t* status;             // device status word
  // uneven batches, fused launches: [0] the next tile to hand out, [1] warps done;
  // zero between launches (the grid's last warp resets both)
  uint32_t* tile_ctr;
  int n;                        // drones
  int N;                        // drones per world (uniform batches)
  int n_blocks, hold, t0, K;
  float dt;
};

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
  return fminf(fmaxf(x, lo), hi);
}

}  // namespace cf
