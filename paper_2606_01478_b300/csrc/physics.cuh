// Device functions of one drone step (one drone per thread, state in registers).
//
// State slots (SIM_STATE_DIM = 20):
//   first-principles: 0-2 p, 3-6 q (x,y,z,w), 7-9 v, 10-12 omega (body),
//                     13-16 Omega (RPM), 17-19 position-controller integrator
//   abstracted:       0-2 p, 3-5 Psi, 6-8 v, 9-11 Psidot, 12 f_sigma
#pragma once

#include "common.cuh"

namespace cf {

enum : int { MOTOR_LAG = 0, MOTOR_GENERAL = 1 };

// Rotation matrix (body -> world) of a scalar-last quaternion, quadratic form
// R = (w^2 - |v|^2) I + 2 v v^T + 2 w [v]x applied to q as stored.
__device__ __forceinline__ void quat_rot(float qx, float qy, float qz, float qw, float R[9]) {
  const float xx = qx * qx, yy = qy * qy, zz = qz * qz, ww = qw * qw;
  const float xy = qx * qy, xz = qx * qz, yz = qy * qz;
  const float wx = qw * qx, wy = qw * qy, wz = qw * qz;
  R[0] = (ww + xx) - (yy + zz);
  R[1] = 2.f * (xy - wz);
  R[2] = 2.f * (xz + wy);
  R[3] = 2.f * (xy + wz);
  R[4] = (ww + yy) - (xx + zz);
  R[5] = 2.f * (yz - wx);
  R[6] = 2.f * (xz - wy);
  R[7] = 2.f * (yz + wx);
  R[8] = (ww + zz) - (xx + yy);
}

// R = Rz(yaw) Ry(pitch) Rx(roll) from sines/cosines.
__device__ __forceinline__ void euler_rot(float sr, float cr, float sp, float cp, float sy, float cy,
                                          float R[9]) {
  R[0] = cy * cp;
  R[1] = cy * sp * sr - sy * cr;
  R[2] = cy * sp * cr + sy * sr;
  R[3] = sy * cp;
  R[4] = sy * sp * sr + cy * cr;
  R[5] = sy * sp * cr - cy * sr;
  R[6] = -sp;
  R[7] = cp * sr;
  R[8] = cp * cr;
}

// Eq. 6 rotor dynamics.  LAG: cv_up = cv_down, cd = 0 (first-order lag).
// GENERAL: W' = (Wc - W) (c_v + c_d (Wc + W)) with (c_v, c_d) picked by Wc >= W,
// which equals c_v (Wc - W) + c_d (Wc^2 - W^2).
template <int MOTOR>
__device__ __forceinline__ float motor_rate(float W, float Wc, const DevParams& P) {
  const float e = Wc - W;
  if constexpr (MOTOR == MOTOR_LAG) {
    return P.cv_up * e;
  } else {
    const bool up = Wc >= W;
    const float cv = up ? P.cv_up : P.cv_down;
    const float cd = up ? P.cd_up : P.cd_down;
    return e * fmaf(cd, Wc + W, cv);
  }
}

// First-principles derivative (Eqs. 1-4 with the rotor wrench and Eq. 6) of
// x[0..16] for held rotor commands Wc.  Rotor i at (sx_i a, sy_i a) with
// sx = (+,-,-,+), sy = (-,-,+,+), yaw sign s = (-,+,-,+).
// Rc: optional R(q) of this very x (row-major 9), e.g. from the controller.
template <int MOTOR>
__device__ __forceinline__ void deriv_fp(const float* x, const float Wc[4], const DevParams& P,
                                         bool drag, float* d, const float* Rc = nullptr) {
  const float qx = x[3], qy = x[4], qz = x[5], qw = x[6];
  const float wx = x[10], wy = x[11], wz = x[12];
  const float s0 = x[13] * x[13], s1 = x[14] * x[14], s2 = x[15] * x[15], s3 = x[16] * x[16];
  float T, tx, ty, tz;
  if constexpr (MOTOR == MOTOR_LAG) {
    T = P.kf * ((s0 + s1) + (s2 + s3));
    tx = P.kfa * ((s2 + s3) - (s0 + s1));
    ty = P.kfa * ((s1 + s2) - (s0 + s3));
    tz = P.km * ((s1 + s3) - (s0 + s2));
  } else {
    // polynomial curves: thrust kf W^2 + kf1 W + kf0, drag torque km W^2 + km1 W
    float f[4], t[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float Wr = x[13 + r];
      f[r] = fmaf(P.kf, Wr * Wr, fmaf(P.kf1, Wr, P.kf0));
      t[r] = fmaf(P.km, Wr * Wr, P.km1 * Wr);
    }
    const float fa = P.kfa * P.inv_kf;  // the rotor arm a = kfa / kf
    T = (f[0] + f[1]) + (f[2] + f[3]);
    tx = fa * ((f[2] + f[3]) - (f[0] + f[1]));
    ty = fa * ((f[1] + f[2]) - (f[0] + f[3]));
    tz = (t[1] + t[3]) - (t[0] + t[2]);
  }
  // thrust along the third column of R(q)
  const float Tm = T * P.inv_m;
  const float r02 = Rc ? Rc[2] : 2.f * fmaf(qx, qz, qw * qy);
  const float r12 = Rc ? Rc[5] : 2.f * fmaf(qy, qz, -qw * qx);
  const float r22 = Rc ? Rc[8] : (qw * qw + qz * qz) - (qx * qx + qy * qy);
  float ax = Tm * r02, ay = Tm * r12, az = fmaf(Tm, r22, -P.g);
  if (MOTOR != MOTOR_LAG && drag) {
    float R[9];
    if (Rc) {
#pragma unroll
      for (int j = 0; j < 9; ++j) R[j] = Rc[j];
    } else {
      quat_rot(qx, qy, qz, qw, R);
    }
    const float vx = x[7], vy = x[8], vz = x[9];
    const float bx = P.Ca_x * P.inv_m * (R[0] * vx + R[3] * vy + R[6] * vz);
    const float by = P.Ca_y * P.inv_m * (R[1] * vx + R[4] * vy + R[7] * vz);
    const float bz = P.Ca_z * P.inv_m * (R[2] * vx + R[5] * vy + R[8] * vz);
    ax += R[0] * bx + R[1] * by + R[2] * bz;
    ay += R[3] * bx + R[4] * by + R[5] * bz;
    az += R[6] * bx + R[7] * by + R[8] * bz;
  }
  d[0] = x[7];
  d[1] = x[8];
  d[2] = x[9];
  // q' = 1/2 q (x) [w, 0]
  d[3] = 0.5f * (fmaf(qw, wx, qy * wz) - qz * wy);
  d[4] = 0.5f * (fmaf(qw, wy, qz * wx) - qx * wz);
  d[5] = 0.5f * (fmaf(qw, wz, qx * wy) - qy * wx);
  d[6] = -0.5f * (fmaf(qx, wx, qy * wy) + qz * wz);
  d[7] = ax;
  d[8] = ay;
  d[9] = az;
#pragma unroll
  for (int r = 0; r < 4; ++r) d[13 + r] = motor_rate<MOTOR>(x[13 + r], Wc[r], P);
  if constexpr (MOTOR != MOTOR_LAG) {
    // rotor angular momentum h e_z, h = -Jpc sum s_i W_i: gyroscopic -w x h and
    // reaction -dh/dt (Eq. 5)
    const float h = -P.Jpc * ((x[14] + x[16]) - (x[13] + x[15]));
    const float dh = -P.Jpc * ((d[14] + d[16]) - (d[13] + d[15]));
    tx = fmaf(-wy, h, tx);
    ty = fmaf(wx, h, ty);
    tz -= dh;
  }
  // w' = J^-1 tau - J^-1 (w x J w)
  d[10] = fmaf(tx, P.inv_Jx, P.cJx * wy * wz);
  d[11] = fmaf(ty, P.inv_Jy, P.cJy * wz * wx);
  d[12] = fmaf(tz, P.inv_Jz, P.cJz * wx * wy);
}

// First-principles derivative in the lag-rotor step form (MOTOR_LAG, no drag):
// the same Eqs. 1-6 as deriv_fp, with the rotor commands given as rates
// u_i = cv W_cmd,i (so W_i' = u_i - cv W_i) and the quaternion rate returned
// doubled, d[3..6] = q (x) [w, 0] = 2 q' (the integrator folds the 1/2 into its
// coefficients).  Constants kf/m, kfa/J, km/J are folded (DevParams).
// SYM_XY: Jx = Jy, where the yaw rate's gyroscopic term (Jx - Jy) wx wy / Jz is
// zero and is left out, and the roll and pitch terms share their factor.
template <bool SYM_XY = false>
__device__ __forceinline__ void deriv_fp_rate(const float* x, const float u[4], const DevParams& P,
                                              float* d, const float* Rc = nullptr) {
  const float qx = x[3], qy = x[4], qz = x[5], qw = x[6];
  const float wx = x[10], wy = x[11], wz = x[12];
  // squared rotor speeds s_i = W_i^2 in the sums the wrench takes: s0 + s1,
  // s2 + s3, s1 - s0 and s3 - s2 (two products, four multiply-adds)
  const float W0 = x[13], W1 = x[14], W2 = x[15], W3 = x[16];
  const float s0 = W0 * W0, s2 = W2 * W2;
  const float a01 = fmaf(W1, W1, s0), a23 = fmaf(W3, W3, s2), S = a01 + a23;
  const float e10 = fmaf(W1, W1, -s0), e32 = fmaf(W3, W3, -s2);
  const float Tm = P.kfm * S;  // collective thrust / m
  float ax, ay, az;
  if (Rc) {
    ax = Tm * Rc[2];
    ay = Tm * Rc[5];
    az = fmaf(Tm, Rc[8], -P.g);
  } else {
    // third column of R(q): 2 (xz + wy), 2 (yz - wx), w^2 - x^2 - y^2 + z^2
    const float Tm2 = P.kfm2 * S;
    ax = Tm2 * fmaf(qx, qz, qw * qy);
    ay = Tm2 * fmaf(qy, qz, -qw * qx);
    az = fmaf(Tm, (qw * qw + qz * qz) - (qx * qx + qy * qy), -P.g);
  }
  d[0] = x[7];
  d[1] = x[8];
  d[2] = x[9];
  d[3] = fmaf(qw, wx, qy * wz) - qz * wy;
  d[4] = fmaf(qw, wy, qz * wx) - qx * wz;
  d[5] = fmaf(qw, wz, qx * wy) - qy * wx;
  d[6] = -(fmaf(qx, wx, qy * wy) + qz * wz);
  d[7] = ax;
  d[8] = ay;
  d[9] = az;
  // w' = J^-1 tau - J^-1 (w x J w), rotor torques as in deriv_fp
  // roll (s2 + s3) - (s0 + s1), pitch (s1 + s2) - (s0 + s3) = e10 - e32,
  // yaw (s1 + s3) - (s0 + s2) = e10 + e32
  if constexpr (SYM_XY) {
    // Jx = Jy: cJy = -cJx exactly (the same quotient negated), cJz = 0
    const float t = P.cJx * wz;
    d[10] = fmaf(P.kfaJx, a23 - a01, t * wy);
    d[11] = fmaf(P.kfaJy, e10 - e32, -t * wx);
    d[12] = P.kmJz * (e10 + e32);
  } else {
    d[10] = fmaf(P.kfaJx, a23 - a01, P.cJx * wy * wz);
    d[11] = fmaf(P.kfaJy, e10 - e32, P.cJy * wz * wx);
    d[12] = fmaf(P.kmJz, e10 + e32, P.cJz * wx * wy);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) d[13 + r] = fmaf(P.ncv, x[13 + r], u[r]);
}

// Abstracted derivative (Eqs. 7-10) of x[0..12] for u = (Psi_cmd, f_cmd).  The
// drag term exists only in the general variant (MOTOR_GENERAL).
// cu = (c3_r Psi_cmd,r, c3_p Psi_cmd,p, c3_y Psi_cmd,y, c_tau f_cmd): the command
// terms, constant while a command is held (abstracted_command).
template <int MOTOR>
__device__ __forceinline__ void deriv_abs(const float* x, const float cu[4], const DevParams& P,
                                          bool drag, float* d) {
  float sr, cr, sp, cp, sy, cy;
  __sincosf(x[3], &sr, &cr);
  __sincosf(x[4], &sp, &cp);
  __sincosf(x[5], &sy, &cy);
  // third column of Rz Ry Rx
  const float r02 = fmaf(cy * sp, cr, sy * sr);
  const float r12 = fmaf(sy * sp, cr, -cy * sr);
  const float r22 = cp * cr;
  const float fm = P.cf_inv_m * x[12];
  float ax = fm * r02, ay = fm * r12, az = fmaf(fm, r22, -P.g);
  if (MOTOR != MOTOR_LAG && drag) {
    float R[9];
    euler_rot(sr, cr, sp, cp, sy, cy, R);
    const float vx = x[6], vy = x[7], vz = x[8];
    const float bx = P.Ca_x * P.inv_m * (R[0] * vx + R[3] * vy + R[6] * vz);
    const float by = P.Ca_y * P.inv_m * (R[1] * vx + R[4] * vy + R[7] * vz);
    const float bz = P.Ca_z * P.inv_m * (R[2] * vx + R[5] * vy + R[8] * vz);
    ax += R[0] * bx + R[1] * by + R[2] * bz;
    ay += R[3] * bx + R[4] * by + R[5] * bz;
    az += R[6] * bx + R[7] * by + R[8] * bz;
  }
  d[0] = x[6];
  d[1] = x[7];
  d[2] = x[8];
  d[3] = x[9];
  d[4] = x[10];
  d[5] = x[11];
  d[6] = ax;
  d[7] = ay;
  d[8] = az;
  d[9] = fmaf(P.c1_r, x[3], fmaf(P.c2_r, x[9], cu[0]));
  d[10] = fmaf(P.c1_p, x[4], fmaf(P.c2_p, x[10], cu[1]));
  d[11] = fmaf(P.c1_y, x[5], fmaf(P.c2_y, x[11], cu[2]));
  d[12] = fmaf(-P.c_tau, x[12], cu[3]);  // c_tau (f_cmd - f)
}

// Abstracted model without thrust dynamics and drag (last sentence of Abstracted
// Physics Modeling): thrust c_f f_cmd acts at once; f_sum does not evolve.
// cu as for deriv_abs, with cu[3] = c_f f_cmd / m (the thrust follows its command).
__device__ __forceinline__ void deriv_abs_nothrust(const float* x, const float cu[4],
                                                   const DevParams& P, float* d) {
  float sr, cr, sp, cp, sy, cy;
  __sincosf(x[3], &sr, &cr);
  __sincosf(x[4], &sp, &cp);
  __sincosf(x[5], &sy, &cy);
  const float fm = cu[3];
  d[0] = x[6];
  d[1] = x[7];
  d[2] = x[8];
  d[3] = x[9];
  d[4] = x[10];
  d[5] = x[11];
  d[6] = fm * fmaf(cy * sp, cr, sy * sr);
  d[7] = fm * fmaf(sy * sp, cr, -cy * sr);
  d[8] = fmaf(fm, cp * cr, -P.g);
  d[9] = fmaf(P.c1_r, x[3], fmaf(P.c2_r, x[9], cu[0]));
  d[10] = fmaf(P.c1_p, x[4], fmaf(P.c2_p, x[10], cu[1]));
  d[11] = fmaf(P.c1_y, x[5], fmaf(P.c2_y, x[11], cu[2]));
  d[12] = 0.f;
}

// ---------------------------------------------------------------- controller

// Attitude action a -> desired rotation Rd and collective thrust Td.
__device__ __forceinline__ void attitude_command(float4 a, const DevParams& P, float Rd[9],
                                                 float& Td) {
  const float ar = clampf(a.x, -1.f, 1.f) * P.max_angle;
  const float ap = clampf(a.y, -1.f, 1.f) * P.max_angle;
  const float ay = clampf(a.z, -1.f, 1.f) * P.max_angle;
  float sr, cr, sp, cp, sy, cy;
  __sincosf(ar, &sr, &cr);
  __sincosf(ap, &sp, &cp);
  __sincosf(ay, &sy, &cy);
  euler_rot(sr, cr, sp, cp, sy, cy, Rd);
  Td = fmaf(P.ts_mg, clampf(a.w, -1.f, 1.f), P.mg);
}

// Attitude action a -> twice the desired unit quaternion qd (scalar last) and the
// collective thrust Td.  qd is the rotation of Rd = Rz(yaw) Ry(pitch) Rx(roll)
// (attitude_command), composed from half angles: qd = qz(yaw) (x) qy(pitch) (x)
// qx(roll).  The factor 2 makes attitude_error2_q's product the vee of the
// matrix form without another multiply.
__device__ __forceinline__ void attitude_command_q(float4 a, const DevParams& P, float qd[4],
                                                   float& Td) {
  const float hr = clampf(a.x, -1.f, 1.f) * P.half_max_angle;
  const float hp = clampf(a.y, -1.f, 1.f) * P.half_max_angle;
  const float hy = clampf(a.z, -1.f, 1.f) * P.half_max_angle;
  float sr, cr, sp, cp, sy, cy;
  __sincosf(hr, &sr, &cr);
  __sincosf(hp, &sp, &cp);
  __sincosf(hy, &sy, &cy);
  const float cp2 = cp + cp, sp2 = sp + sp;
  const float a_ = cp2 * cy, b_ = sp2 * sy, c_ = sp2 * cy, d_ = cp2 * sy;
  qd[0] = fmaf(sr, a_, -cr * b_);
  qd[1] = fmaf(cr, c_, sr * d_);
  qd[2] = fmaf(cr, d_, -sr * c_);
  qd[3] = fmaf(cr, a_, sr * b_);
  Td = fmaf(P.ts_mg, clampf(a.w, -1.f, 1.f), P.mg);
}

// 2 e_R = vee(Rd^T R - R^T Rd) from quaternions: with qe = qd* (x) q,
// Rd^T R = R(qe) and vee(R(qe) - R(qe)^T) = 4 qe_w qe_v for the quadratic form
// of R (any norm of q); with qd2 = 2 qd (attitude_command_q) that is
// (qd2* (x) q)_w (qd2* (x) q)_v.  x = the state (q in slots 3-6).
__device__ __forceinline__ void attitude_error2_q(const float* x, const float qd2[4], float& ex,
                                                  float& ey, float& ez) {
  const float qx = x[3], qy = x[4], qz = x[5], qw = x[6];
  const float dx = qd2[0], dy = qd2[1], dz = qd2[2], dw = qd2[3];
  // qd* (x) q = (dw qv - qw dv - dv x qv, dw qw + dv . qv)
  const float vx = fmaf(dw, qx, fmaf(-qw, dx, fmaf(-dy, qz, dz * qy)));
  const float vy = fmaf(dw, qy, fmaf(-qw, dy, fmaf(-dz, qx, dx * qz)));
  const float vz = fmaf(dw, qz, fmaf(-qw, dz, fmaf(-dx, qy, dy * qx)));
  const float w = fmaf(dw, qw, fmaf(dx, qx, fmaf(dy, qy, dz * qz)));
  ex = w * vx;
  ey = w * vy;
  ez = w * vz;
}

// Abstracted-model input u = (Psi_cmd, f_cmd) from an attitude action, and the
// derivative's command terms cu (deriv_abs with THRUST_LAG, deriv_abs_nothrust
// without).
template <bool THRUST_LAG>
__device__ __forceinline__ void abstracted_command(float4 a, const DevParams& P, float u[4],
                                                   float cu[4]) {
  u[0] = clampf(a.x, -1.f, 1.f) * P.max_angle;
  u[1] = clampf(a.y, -1.f, 1.f) * P.max_angle;
  u[2] = clampf(a.z, -1.f, 1.f) * P.max_angle;
  u[3] = fmaf(P.ts_mg, clampf(a.w, -1.f, 1.f), P.mg);
  // the derivative's command terms (Eqs. 8-10), constant while the command is held
  cu[0] = P.c3_r * u[0];
  cu[1] = P.c3_p * u[1];
  cu[2] = P.c3_y * u[2];
  cu[3] = THRUST_LAG ? P.c_tau * u[3] : P.cf_inv_m * u[3];
}

// 2 e_R = vee(Rd^T R - R^T Rd); only the off-diagonal entries of Rd^T R are formed.
__device__ __forceinline__ void attitude_error2(const float R[9], const float Rd[9], float& ex,
                                                float& ey, float& ez) {
#define CF_M(i, j) fmaf(Rd[i], R[j], fmaf(Rd[3 + i], R[3 + j], Rd[6 + i] * R[6 + j]))
  ex = CF_M(2, 1) - CF_M(1, 2);
  ey = CF_M(0, 2) - CF_M(2, 0);
  ez = CF_M(1, 0) - CF_M(0, 1);
#undef CF_M
}

// Geometric attitude PD, tau = -K_R J e_R - K_w J w, given 2 e_R.
__device__ __forceinline__ void attitude_torque_e(float ex, float ey, float ez, float wx, float wy,
                                                  float wz, const DevParams& P, float& tx,
                                                  float& ty, float& tz) {
  tx = -fmaf(P.KRJh_x, ex, P.KwJ_x * wx);
  ty = -fmaf(P.KRJh_y, ey, P.KwJ_y * wy);
  tz = -fmaf(P.KRJh_z, ez, P.KwJ_z * wz);
}

// The same with e_R = 1/2 vee(Rd^T R - R^T Rd) from the matrices.
__device__ __forceinline__ void attitude_torque(const float R[9], const float Rd[9], float wx,
                                                float wy, float wz, const DevParams& P,
                                                float& tx, float& ty, float& tz) {
  float ex, ey, ez;
  attitude_error2(R, Rd, ex, ey, ez);
  attitude_torque_e(ex, ey, ez, wx, wy, wz, P, tx, ty, tz);
}

// X-configuration mixer: per-rotor thrusts from (T, tau), clipped to the
// thrust curve's range, converted to rotor-speed commands (pure quadratic:
// sqrt(f / kf); general: the root of kf W^2 + kf1 W + kf0 = f).
template <int MOTOR = MOTOR_LAG>
__device__ __forceinline__ void mixer(float T, float tx, float ty, float tz, const DevParams& P,
                                      float Wc[4]) {
  const float A = 0.25f * T, X = tx * P.mix_a, Y = ty * P.mix_a, Z = tz * P.mix_k;
  float f[4];
  f[0] = (A - X) - (Y + Z);
  f[1] = (A - X) + (Y + Z);
  f[2] = (A + X) + (Y - Z);
  f[3] = (A + X) - (Y - Z);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if constexpr (MOTOR == MOTOR_LAG) {
      Wc[r] = sqrt_approx(clampf(f[r], 0.f, P.fmax) * P.inv_kf);
    } else {
      const float fc = clampf(f[r], P.kf0, P.fmax);
      const float disc = fmaxf(fmaf(P.four_kf, fc - P.kf0, P.kf1sq), 0.f);
      Wc[r] = (sqrt_approx(disc) - P.kf1) * P.inv_2kf;
    }
  }
}

// Lag-rotor mixer in the step form: rotor command rates u_i = cv W_cmd,i.  X, Y,
// Z are the mixer's torque terms tau_x mix_a, tau_y mix_a, tau_z mix_k scaled by
// cv^2 / kf (as is cA = cv^2 / (4 kf)), so u_i^2 = cv^2 f_i / kf with the same
// X-configuration signs and thrust clip [0, kf W_max^2] as mixer.
__device__ __forceinline__ void mixer_rate(float T, float X, float Y, float Z, const DevParams& P,
                                           float u[4]) {
  const float A = P.cA * T;
  float f[4];
  f[0] = (A - X) - (Y + Z);
  f[1] = (A - X) + (Y + Z);
  f[2] = (A + X) + (Y - Z);
  f[3] = (A + X) - (Y - Z);
#pragma unroll
  for (int r = 0; r < 4; ++r) u[r] = sqrt_approx(clampf(f[r], 0.f, P.u2max));
}

// Attitude PD followed by the step-form mixer (lag rotors), given 2 e_R: the PD
// gains, mixer factors and cv^2 / kf are folded into cR*, cw* (DevParams).
__device__ __forceinline__ void attitude_mixer_rate_e(float ex, float ey, float ez, float T,
                                                      float wx, float wy, float wz,
                                                      const DevParams& P, float u[4]) {
  mixer_rate(T, -fmaf(P.cRx, ex, P.cwx * wx), -fmaf(P.cRy, ey, P.cwy * wy),
             -fmaf(P.cRz, ez, P.cwz * wz), P, u);
}

__device__ __forceinline__ void attitude_mixer_rate(const float R[9], const float Rd[9], float T,
                                                    float wx, float wy, float wz,
                                                    const DevParams& P, float u[4]) {
  float ex, ey, ez;
  attitude_error2(R, Rd, ex, ey, ez);
  attitude_mixer_rate_e(ex, ey, ez, T, wx, wy, wz, P, u);
}

// Position PID (geometric): setpoint sp = (x, y, z, yaw) with (sin, cos) of
// yaw precomputed; returns Rd, Td and the integrator increment e_p.
__device__ __forceinline__ void position_command(const float* x, const float R[9], float4 sp,
                                                 float syaw, float cyaw, const DevParams& P,
                                                 float Rd[9], float& Td, float ep[3]) {
  ep[0] = sp.x - x[0];
  ep[1] = sp.y - x[1];
  ep[2] = sp.z - x[2];
  const float adx = fmaf(P.Kp_x, ep[0], fmaf(P.Ki_x, x[17], -P.Kd_x * x[7]));
  const float ady = fmaf(P.Kp_y, ep[1], fmaf(P.Ki_y, x[18], -P.Kd_y * x[8]));
  const float adz = fmaf(P.Kp_z, ep[2], fmaf(P.Ki_z, x[19], -P.Kd_z * x[9])) + P.g;
  Td = P.mass * fmaf(adx, R[2], fmaf(ady, R[5], adz * R[8]));
  const float inz = rsqrt_approx(fmaf(adx, adx, fmaf(ady, ady, adz * adz)));
  const float zx = adx * inz, zy = ady * inz, zz = adz * inz;
  // y_d = z_d x (cos yaw, sin yaw, 0), normalised
  float yx = -zz * syaw, yy = zz * cyaw, yz = fmaf(zx, syaw, -zy * cyaw);
  const float iny = rsqrt_approx(fmaf(yx, yx, fmaf(yy, yy, yz * yz)));
  yx *= iny;
  yy *= iny;
  yz *= iny;
  // x_d = y_d x z_d
  const float xx = fmaf(yy, zz, -yz * zy), xy = fmaf(yz, zx, -yx * zz), xz = fmaf(yx, zy, -yy * zx);
  Rd[0] = xx; Rd[1] = yx; Rd[2] = zx;
  Rd[3] = xy; Rd[4] = yy; Rd[5] = zy;
  Rd[6] = xz; Rd[7] = yz; Rd[8] = zz;
}

}  // namespace cf
