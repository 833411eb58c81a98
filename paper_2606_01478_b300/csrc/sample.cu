// Batched sampling rollouts: the forward model of the paper's MPPI / iCEM
// controller (Results, Control in Cluttered Environments; Materials and
// Methods, Model Predictive Path Integral), which evaluates many sampled
// command sequences per control step with the full simulation.
//
// One rollout (drone d, sample s) per thread of a persistent grid.  Per step k:
//   xi = 4 normals: Philox4x32-10 (Salmon et al., SC'11) on counter
//        (id_lo, id_hi, k, 0), key = 64-bit seed, id = d * S + s; Box-Muller on
//        the top 23 bits of each word
//   a  = clip(nominal[w][k] + sigma xi, -1, 1)  (attitude interface)
//   one first-principles step (Euler or RK4) from the drone's current state
//   cost += |p - g_w| + w_obs sum_o max(0, r_o - |p - c_o|)
// The S samples of a drone are consecutive threads, so the drone's state,
// goal and parameters are broadcast loads; the obstacles live in kernel
// parameter space (constant bank).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "noise.cuh"
#include "stepcore.cuh"

namespace cf {
namespace sp {

struct Scene {
  float4 obs[SIM_MAX_OBSTACLES];  // centre xyz, radius
  float r2[SIM_MAX_OBSTACLES];    // radius^2
  int n_obs;
  float w_obs, sigma, dt;
  int S, H;
  int cull_steps;  // obstacle culling window (steps)
};

struct Args {
  const float4* planes;  // [5][n] drone states (read only)
  const int* offsets;    // [M + 1] first drone of each world (uneven batches) or null
  const float* goals;    // [M][3]
  const float* nominal;  // [M][H][4] or null (zero)
  const unsigned long long* seed;
  const DevParams* params;
  const int32_t* set_of_world;
  float* cost;  // [n][S]
  long long total;
  int n, M, N;
  // MPPI mode (n_ctrl > 0): nominal is [n][n_ctrl][H][4], sample s uses
  // controller s / S_c; noise eps_k = rho eps_{k-1} + rho_c xi_k (rho_c = sqrt(1 - rho^2))
  int n_ctrl, S_c;
  float rho, rho_c;
};

using noise::box_muller;
using noise::philox4x32_10;
using noise::philox_round_key;

// SYM: Jx = Jy in every parameter set (the lag step form then drops the yaw
// rate's zero gyroscopic term).
template <int INTEG, int MOTOR, bool WINDOWED, bool SYM>
__device__ __forceinline__ float rollout(const Args& a, const Scene& sc, const DevParams& P,
                                         long long r, int d, int smp, int w,
                                         const uint2* keys) {
  float s[20];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float4 v = a.planes[(size_t)j * a.n + d];
    s[4 * j] = v.x;
    s[4 * j + 1] = v.y;
    s[4 * j + 2] = v.z;
    s[4 * j + 3] = v.w;
  }
  const float gx = a.goals[3 * w], gy = a.goals[3 * w + 1], gz = a.goals[3 * w + 2];
  const bool drag = (P.flags & PF_DRAG) != 0;
  const uint32_t id_lo = (uint32_t)r, id_hi = (uint32_t)((unsigned long long)r >> 32);
  const float4* nom = nullptr;
  if (a.nominal) {
    const size_t row = a.n_ctrl > 0 ? (size_t)d * a.n_ctrl + smp / a.S_c : (size_t)w;
    nom = reinterpret_cast<const float4*>(a.nominal) + row * sc.H;
  }
  // Obstacles the drone cannot reach within a window of T = steps x dt contribute
  // exactly 0 to the penalties of those steps and are skipped.  Reach bound from
  // the state at the window's start: |v| T + A T^2 with
  // A >= |p''| = |(T_rotor/m) R e_z - g e_z| <= 4 kf W_max^2 / m + g, valid for
  // Euler and RK4 (both move p by at most T|v| + A T^2 / 2) when the rotor
  // speeds stay within [0, max(W_max, W)]: first-order-lag rotors with
  // dt * cv <= 1 and no drag.  Otherwise every obstacle is tested.  The
  // candidate set is rebuilt at the start of every window of sc.cull_steps
  // steps: over a long horizon the bound would cover the whole scene.
  const unsigned long long all = sc.n_obs >= 64 ? ~0ull : ((1ull << sc.n_obs) - 1ull);
  uint32_t cand_lo = (uint32_t)all, cand_hi = (uint32_t)(all >> 32);
  bool sparse = false;  // few candidates: visit the set bits; else test every obstacle
  auto cull = [&](int steps) {
    const float wmax = fmaxf(fmaxf(P.omega_max, fmaxf(s[13], s[14])), fmaxf(s[15], s[16]));
    const float acc = 4.f * P.kf * wmax * wmax * P.inv_m * 1.01f + P.g;
    const float T = steps * sc.dt;
    const float v0 = sqrtf(fmaf(s[7], s[7], fmaf(s[8], s[8], s[9] * s[9])));
    const float reach = fmaf(T, v0, acc * T * T) * 1.01f + 1e-3f;
    unsigned long long cand = 0ull;
    for (int o = 0; o < sc.n_obs; ++o) {
      const float4 ob = sc.obs[o];
      const float dx = s[0] - ob.x, dy = s[1] - ob.y, dz = s[2] - ob.z;
      const float lim = ob.w + reach;
      if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < lim * lim) cand |= 1ull << o;
    }
    cand_lo = (uint32_t)cand;
    cand_hi = (uint32_t)(cand >> 32);
    sparse = 3 * __popcll(cand) < sc.n_obs;
  };
  const bool cullable = MOTOR == MOTOR_LAG && !drag && sc.dt * P.cv_up <= 1.f;
  // When the warp's 32 lanes hold samples of one drone, the warp culls once for
  // all of them: the union of the lanes' candidate sets is bounded by the
  // sphere around lane 0's position whose radius is the largest distance of a
  // lane from it plus that lane's reach; every obstacle outside it lies outside
  // each lane's own bound (triangle inequality), and testing an obstacle a lane
  // cannot reach adds exactly zero, so the costs are those of per-sample culling.
  // Each lane tests one obstacle per pass; a ballot gathers the set.
  const unsigned FULL = 0xffffffffu;
  bool coop = false;
  if (cullable && __activemask() == FULL) coop = __all_sync(FULL, d == __shfl_sync(FULL, d, 0));
  auto cull_warp = [&](int steps) {
    const float wmax = fmaxf(fmaxf(P.omega_max, fmaxf(s[13], s[14])), fmaxf(s[15], s[16]));
    const float acc = 4.f * P.kf * wmax * wmax * P.inv_m * 1.01f + P.g;
    const float T = steps * sc.dt;
    const float v0 = sqrtf(fmaf(s[7], s[7], fmaf(s[8], s[8], s[9] * s[9])));
    const float reach = fmaf(T, v0, acc * T * T) * 1.01f + 1e-3f;
    const float cx = __shfl_sync(FULL, s[0], 0), cy = __shfl_sync(FULL, s[1], 0),
                cz = __shfl_sync(FULL, s[2], 0);
    const float ox = s[0] - cx, oy = s[1] - cy, oz = s[2] - cz;
    // non-negative floats order like their bit patterns
    const float rad = __uint_as_float(__reduce_max_sync(
        FULL, __float_as_uint(sqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz))) + reach)));
    const float R = rad * 1.0001f + 1e-4f;
    const int lane = threadIdx.x & 31;
    unsigned long long cand = 0ull;
    for (int base = 0; base < sc.n_obs; base += 32) {
      const int o = base + lane;
      bool in = false;
      if (o < sc.n_obs) {
        const float4 ob = sc.obs[o];
        const float dx = cx - ob.x, dy = cy - ob.y, dz = cz - ob.z;
        const float lim = ob.w + R;
        in = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < lim * lim;
      }
      cand |= (unsigned long long)__ballot_sync(FULL, in) << base;
    }
    cand_lo = (uint32_t)cand;
    cand_hi = (uint32_t)(cand >> 32);
    sparse = 3 * __popcll(cand) < sc.n_obs;
  };
  if (cullable) {
    const int steps0 = WINDOWED ? min(sc.cull_steps, sc.H) : sc.H;
    if (coop) cull_warp(steps0);
    else cull(steps0);
  }
  float cost = 0.f;
  float4 eps = make_float4(0.f, 0.f, 0.f, 0.f);
  const bool ar1 = a.rho != 0.f;
  noise::PhiloxSteps ph(id_lo, id_hi, keys);
  // WINDOWED: the horizon spans several windows (a kernel of its own, so that a
  // horizon of one window keeps a loop without culling code)
  int next_cull = cullable ? sc.cull_steps : sc.H;
  for (int k = 0; k < sc.H; ++k) {
    if constexpr (WINDOWED) {
      if (k == next_cull) {
        if (coop) cull_warp(min(sc.cull_steps, sc.H - k));
        else cull(min(sc.cull_steps, sc.H - k));
        next_cull += sc.cull_steps;
      }
    }
    uint32_t c[4];
    ph.next(c, keys);  // the block of counter (id_lo, id_hi, k, 0)
    const float2 z01 = box_muller(c[0], c[1]);
    const float2 z23 = box_muller(c[2], c[3]);
    // AR(1) temporal correlation: eps_0 = xi_0, eps_k = rho eps_{k-1} + rho_c xi_k;
    // white noise (rho = 0) takes eps = xi without the arithmetic (a uniform branch)
    if (ar1) {
      const float cx = k == 0 ? 1.f : a.rho_c;
      eps.x = fmaf(a.rho, eps.x, cx * z01.x);
      eps.y = fmaf(a.rho, eps.y, cx * z01.y);
      eps.z = fmaf(a.rho, eps.z, cx * z23.x);
      eps.w = fmaf(a.rho, eps.w, cx * z23.y);
    } else {
      eps = make_float4(z01.x, z01.y, z23.x, z23.y);
    }
    // sigma eps + nominal as one fused multiply-add, as the MPPI update forms it
    // (no nominal: + 0, the product itself)
    const float4 m = nom ? nom[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 act = make_float4(fmaf(sc.sigma, eps.x, m.x), fmaf(sc.sigma, eps.y, m.y),
                                   fmaf(sc.sigma, eps.z, m.z), fmaf(sc.sigma, eps.w, m.w));
    CtrlHold h;
    decode_command<SIM_FIRST_PRINCIPLES, SIM_CTRL_ATTITUDE>(act, P, h);
    one_step<SIM_FIRST_PRINCIPLES, INTEG, SIM_CTRL_ATTITUDE, MOTOR, SYM>(s, h, P, drag, sc.dt);
    const float ex = s[0] - gx, ey = s[1] - gy, ez = s[2] - gz;
    float pen = 0.f;
    auto test = [&](int o) {
      const float4 ob = sc.obs[o];
      const float dx = s[0] - ob.x, dy = s[1] - ob.y, dz = s[2] - ob.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < sc.r2[o]) pen += ob.w - sqrt_approx(d2);
    };
    if (sparse) {
      for (uint32_t m = cand_lo; m; m &= m - 1u) test(__ffs(m) - 1);
      for (uint32_t m = cand_hi; m; m &= m - 1u) test(32 + __ffs(m) - 1);
    } else {
      // dense: obstacles outside the reach bound add exactly zero, so testing them is harmless
      for (int o = 0; o < sc.n_obs; ++o) test(o);
    }
    cost += sqrt_approx(fmaf(ex, ex, fmaf(ey, ey, ez * ez))) + sc.w_obs * pen;
  }
  return cost;
}

template <int INTEG, int MOTOR, bool PERSET, bool WINDOWED, bool SYM>
__global__ void __launch_bounds__(256) sample_kernel(Args a, Scene sc, DevParams P0) {
  const unsigned long long seed = *a.seed;
  __shared__ uint2 keys[10];
  for (int r = threadIdx.x; r < 10; r += blockDim.x)
    keys[r] = philox_round_key((uint32_t)seed, (uint32_t)(seed >> 32), r);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < a.total; r += stride) {
    const int d = (int)(r / sc.S);
    const int smp = (int)(r - (long long)d * sc.S);
    int w;
    if (a.offsets) {  // largest w with offsets[w] <= d
      int lo = 0, hi = a.M - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.offsets[mid] <= d) lo = mid;
        else hi = mid - 1;
      }
      w = lo;
    } else {
      w = d / a.N;
    }
    float cost;
    if constexpr (PERSET) {
      const DevParams P = a.params[a.set_of_world[w]];
      cost = rollout<INTEG, MOTOR, WINDOWED, SYM>(a, sc, P, r, d, smp, w, keys);
    } else {
      cost = rollout<INTEG, MOTOR, WINDOWED, SYM>(a, sc, P0, r, d, smp, w, keys);
    }
    a.cost[r] = cost;
  }
}

template <int INTEG, int MOTOR, bool PERSET, bool WINDOWED, bool SYM = false>
static cudaError_t launch_t(const Args& a, const Scene& sc, const DevParams& P, int tpb,
                            cudaStream_t st) {
  static int cached[16][9] = {};  // per instantiation
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slot = tpb / 32;
  int per_sm = (dev < 16 && slot <= 8) ? cached[dev][slot] : 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_kernel<INTEG, MOTOR, PERSET, WINDOWED, SYM>,
                                                  tpb, 0);
    if (per_sm < 1) per_sm = 1;
    if (dev < 16 && slot <= 8) cached[dev][slot] = per_sm;
  }
  long long grid = (long long)sms * per_sm;
  const long long need = (a.total + tpb - 1) / tpb;
  if (grid > need) grid = need;
  sample_kernel<INTEG, MOTOR, PERSET, WINDOWED, SYM><<<(unsigned)grid, tpb, 0, st>>>(a, sc, P);
  return cudaGetLastError();
}

__global__ void philox_kernel(const unsigned long long* seed, unsigned long long first_id, long long n,
                              int step, uint32_t* words, float* normals) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long s = *seed, id = first_id + (unsigned long long)i;
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step, 0u};
  philox4x32_10(c, (uint32_t)s, (uint32_t)(s >> 32));
  if (words) {
    words[4 * i] = c[0];
    words[4 * i + 1] = c[1];
    words[4 * i + 2] = c[2];
    words[4 * i + 3] = c[3];
  }
  if (normals) {
    const float2 a = box_muller(c[0], c[1]), b = box_muller(c[2], c[3]);
    normals[4 * i] = a.x;
    normals[4 * i + 1] = a.y;
    normals[4 * i + 2] = b.x;
    normals[4 * i + 3] = b.y;
  }
}

}  // namespace sp

cudaError_t launch_philox(const unsigned long long* seed, unsigned long long first_id, long long n,
                          int step, uint32_t* words, float* normals, cudaStream_t st) {
  const int tpb = 256;
  sp::philox_kernel<<<(unsigned)((n + tpb - 1) / tpb), tpb, 0, st>>>(seed, first_id, n, step, words,
                                                                     normals);
  return cudaGetLastError();
}

cudaError_t launch_sample(const float4* planes, int n, const int* offsets, int M, int N,
                          const float* goals, const float* nominal, const unsigned long long* seed,
                          const DevParams* params, const int32_t* set_of_world, const DevParams& P0,
                          bool per_set, bool general_motor, int integrator, const float* obstacles,
                          int n_obs, float w_obs, float sigma, float dt, int S, int H, float* cost,
                          int tpb, cudaStream_t st, int n_ctrl, float rho) {
  sp::Args a;
  a.planes = planes;
  a.offsets = offsets;
  a.goals = goals;
  a.nominal = nominal;
  a.seed = seed;
  a.params = params;
  a.set_of_world = set_of_world;
  a.cost = cost;
  a.total = (long long)n * S;
  a.n = n;
  a.M = M;
  a.N = N;
  a.n_ctrl = n_ctrl;
  a.S_c = n_ctrl > 0 ? S / n_ctrl : S;
  a.rho = rho;
  a.rho_c = sqrtf(1.f - rho * rho);
  sp::Scene sc;
  for (int o = 0; o < SIM_MAX_OBSTACLES; ++o) {
    sc.obs[o] = o < n_obs ? make_float4(obstacles[4 * o], obstacles[4 * o + 1], obstacles[4 * o + 2],
                                        obstacles[4 * o + 3])
                          : make_float4(0.f, 0.f, 0.f, 0.f);
    sc.r2[o] = o < n_obs ? obstacles[4 * o + 3] * obstacles[4 * o + 3] : 0.f;
  }
  sc.n_obs = n_obs;
  sc.w_obs = w_obs;
  sc.sigma = sigma;
  sc.dt = dt;
  sc.S = S;
  sc.H = H;
  // culling windows of about 0.1 s: a Crazyflie-class drone (thrust-to-weight
  // about 2) moves at most ~0.3 m + 0.1 |v| in that time
  sc.cull_steps = (int)std::min<double>(H, std::max(1.0, std::floor(0.1 / dt + 0.5)));
  // culling runs only for lag rotors; with those, a horizon of several windows
  // takes the windowed kernel
  const bool windowed = sc.cull_steps < H;
  // the lag-rotor variants come in two forms: Jx = Jy in every set (the union of the
  // sets' flags lacks PF_ASYM_XY) or not
  const bool sym = (P0.flags & PF_ASYM_XY) == 0;
#define CF_S(I, MO, WI)                                                      \
  return per_set ? sp::launch_t<I, MO, true, WI>(a, sc, P0, tpb, st)          \
                 : sp::launch_t<I, MO, false, WI>(a, sc, P0, tpb, st)
#define CF_L(I, WI)                                                                        \
  return per_set ? (sym ? sp::launch_t<I, MOTOR_LAG, true, WI, true>(a, sc, P0, tpb, st)    \
                        : sp::launch_t<I, MOTOR_LAG, true, WI, false>(a, sc, P0, tpb, st))  \
                 : (sym ? sp::launch_t<I, MOTOR_LAG, false, WI, true>(a, sc, P0, tpb, st)   \
                        : sp::launch_t<I, MOTOR_LAG, false, WI, false>(a, sc, P0, tpb, st))
  if (integrator == SIM_RK4) {
    if (general_motor) CF_S(SIM_RK4, MOTOR_GENERAL, false);
    if (windowed) CF_L(SIM_RK4, true);
    CF_L(SIM_RK4, false);
  }
  if (general_motor) CF_S(SIM_EULER, MOTOR_GENERAL, false);
  if (windowed) CF_L(SIM_EULER, true);
  CF_L(SIM_EULER, false);
#undef CF_S
#undef CF_L
}

}  // namespace cf
