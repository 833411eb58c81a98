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

// Round r of Philox4x32-10 xors the key (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85)
// into the high product halves.  The round keys depend on the seed alone: the
// sampling kernel builds the ten once per block in shared memory and every draw
// reads them from there.
__device__ __forceinline__ uint2 philox_round_key(uint32_t k0, uint32_t k1, uint32_t r) {
  return make_uint2(k0 + r * 0x9E3779B9u, k1 + r * 0xBB67AE85u);
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], const uint2* keys) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint2 k = keys[r];
    // one widening multiply gives both halves of each 32 x 32 -> 64-bit product
    unsigned long long p0, p1;
    asm("mul.wide.u32 %0, %1, 0xD2511F53;" : "=l"(p0) : "r"(c[0]));
    asm("mul.wide.u32 %0, %1, 0xCD9E8D57;" : "=l"(p1) : "r"(c[2]));
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k.x, n2 = hi0 ^ c[3] ^ k.y;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint2 keys[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) keys[r] = philox_round_key(k0, k1, r);
  philox4x32_10(c, keys);
}

// Two standard normals from two words: u = ((w >> 9) + 0.5) 2^-23 (exact),
// r = sqrt(-2 ln u1), angle 2 pi u2 (evaluated as 2 pi u2 - pi, in [-pi, pi)).
__device__ __forceinline__ float2 box_muller(uint32_t w1, uint32_t w2) {
  // the float with a zero exponent and mantissa w >> 9 is 1 + (w >> 9) 2^-23;
  // subtracting 1 - 2^-24 is exact and leaves ((w >> 9) + 0.5) 2^-23
  const float u1 = __uint_as_float((w1 >> 9) + 0x3F800000u) - 0.99999994039535522f;
  const float u2 = __uint_as_float((w2 >> 9) + 0x3F800000u) - 0.99999994039535522f;
  const float r = sqrt_approx(-2.f * logf(u1));  // within 1 ulp of the rounded root
  float s, c;
  __sincosf(fmaf(6.28318530717958648f, u2, -3.14159265358979324f), &s, &c);
  return make_float2(-r * c, -r * s);
}

template <int INTEG, int MOTOR, bool WINDOWED>
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
  if (cullable) cull(WINDOWED ? min(sc.cull_steps, sc.H) : sc.H);
  float cost = 0.f;
  float4 eps = make_float4(0.f, 0.f, 0.f, 0.f);
  // WINDOWED: the horizon spans several windows (a kernel of its own, so that a
  // horizon of one window keeps a loop without culling code)
  int next_cull = cullable ? sc.cull_steps : sc.H;
  for (int k = 0; k < sc.H; ++k) {
    if constexpr (WINDOWED) {
      if (k == next_cull) {
        cull(min(sc.cull_steps, sc.H - k));
        next_cull += sc.cull_steps;
      }
    }
    uint32_t c[4] = {id_lo, id_hi, (uint32_t)k, 0u};
    philox4x32_10(c, keys);
    const float2 z01 = box_muller(c[0], c[1]);
    const float2 z23 = box_muller(c[2], c[3]);
    // AR(1) temporal correlation: eps_0 = xi_0, eps_k = rho eps_{k-1} + rho_c xi_k
    // (rho = 0, rho_c = 1: white noise, eps = xi exactly)
    const float cx = k == 0 ? 1.f : a.rho_c;
    eps.x = fmaf(a.rho, eps.x, cx * z01.x);
    eps.y = fmaf(a.rho, eps.y, cx * z01.y);
    eps.z = fmaf(a.rho, eps.z, cx * z23.x);
    eps.w = fmaf(a.rho, eps.w, cx * z23.y);
    // sigma eps + nominal as one fused multiply-add, as the MPPI update forms it
    // (no nominal: + 0, the product itself)
    const float4 m = nom ? nom[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 act = make_float4(fmaf(sc.sigma, eps.x, m.x), fmaf(sc.sigma, eps.y, m.y),
                                   fmaf(sc.sigma, eps.z, m.z), fmaf(sc.sigma, eps.w, m.w));
    CtrlHold h;
    decode_command<SIM_FIRST_PRINCIPLES, SIM_CTRL_ATTITUDE>(act, P, h);
    one_step<SIM_FIRST_PRINCIPLES, INTEG, SIM_CTRL_ATTITUDE, MOTOR>(s, h, P, drag, sc.dt);
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

template <int INTEG, int MOTOR, bool PERSET, bool WINDOWED>
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
      cost = rollout<INTEG, MOTOR, WINDOWED>(a, sc, P, r, d, smp, w, keys);
    } else {
      cost = rollout<INTEG, MOTOR, WINDOWED>(a, sc, P0, r, d, smp, w, keys);
    }
    a.cost[r] = cost;
  }
}

template <int INTEG, int MOTOR, bool PERSET, bool WINDOWED>
static cudaError_t launch_t(const Args& a, const Scene& sc, const DevParams& P, int tpb,
                            cudaStream_t st) {
  static int cached[16][9] = {};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int slot = tpb / 32;
  int per_sm = (dev < 16 && slot <= 8) ? cached[dev][slot] : 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_kernel<INTEG, MOTOR, PERSET, WINDOWED>,
                                                  tpb, 0);
    if (per_sm < 1) per_sm = 1;
    if (dev < 16 && slot <= 8) cached[dev][slot] = per_sm;
  }
  long long grid = (long long)sms * per_sm;
  const long long need = (a.total + tpb - 1) / tpb;
  if (grid > need) grid = need;
  sample_kernel<INTEG, MOTOR, PERSET, WINDOWED><<<(unsigned)grid, tpb, 0, st>>>(a, sc, P);
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

// MPPI / iCEM update: one block per drone, warp c = controller c.
struct MppiArgs {
  const float* cost;  // [n][S]
  float* mean;        // [n][C][H][4]: in = current means, out = updated means shifted one step
  float* plan;        // [n][H][4]: updated mean of the best controller
  float* best_cost;   // [n]
  const unsigned long long* seed;
  int n, S, H, C, S_c, n_e;
  float sigma, rho, rho_c, inv_lam;
};

__device__ __forceinline__ bool lex_less(float a, int ia, float b, int ib) {
  return a < b || (a == b && ia < ib);
}

// Order-preserving map of float costs to unsigned keys (-0 and +0 share a key;
// NaN maps to ~0u, above every other key, and is never selected).
__device__ __forceinline__ uint32_t cost_key(float v) {
  if (v != v) return 0xFFFFFFFFu;
  const uint32_t b = __float_as_uint(v + 0.f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_cost(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// The elites of one controller, for one warp: the n_e smallest (cost, index)
// pairs of cc[0..S_c), ties to the lower index, NaN never selected.  On return
// lanes 0 .. n-1 hold one elite each (el_c, el_i; the others INFINITY and
// 0x7fffffff), n = min(n_e, number of non-NaN costs), and jmin is the smallest
// cost (INFINITY if there is none).  Up to 2048 costs (64 per lane, kept in
// registers as keys): a bisection over the key range finds the threshold T
// with count(key <= T) >= n, counting with warp reductions and stopping as soon
// as exactly n keys lie at or below the midpoint; the elites are the keys < T
// and the lowest-index keys equal to T up to n, compacted into lanes in index
// order through stage[32] (cost) and stage_i[32] (index) in shared memory.
// More costs: n rounds of a warp arg-min, reading them from memory each round.
constexpr int ELITE_REG = 64;
__device__ __forceinline__ void select_elites(const float* cc, int S_c, int n_e, int lane,
                                              float* stage, int* stage_i, float& el_c, int& el_i,
                                              float& jmin) {
  const unsigned FULL = 0xffffffffu;
  el_c = INFINITY;
  el_i = 0x7fffffff;
  if (S_c <= 32 * ELITE_REG) {
    uint32_t kr[ELITE_REG];
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
    int nv = 0;
    // every lane loads all its slots (clamped index) before using any: guarded
    // loads were issued one at a time
    float cv[ELITE_REG];
#pragma unroll
    for (int j = 0; j < ELITE_REG; ++j) cv[j] = cc[min(lane + 32 * j, S_c - 1)];
#pragma unroll
    for (int j = 0; j < ELITE_REG; ++j) {
      const int s = lane + 32 * j;
      kr[j] = s < S_c ? cost_key(cv[j]) : 0xFFFFFFFFu;
      if (kr[j] != 0xFFFFFFFFu) {
        kmin = min(kmin, kr[j]);
        kmax = max(kmax, kr[j]);
        ++nv;
      }
    }
    nv = __reduce_add_sync(FULL, nv);
    kmin = __reduce_min_sync(FULL, kmin);
    kmax = __reduce_max_sync(FULL, kmax);
    const int n = min(n_e, nv);
    jmin = n > 0 ? key_cost(kmin) : INFINITY;
    if (n == 0) return;
    auto count_le = [&](uint32_t t) {
      int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
      for (int j = 0; j < ELITE_REG; j += 4) {
        c0 += kr[j] <= t;
        c1 += kr[j + 1] <= t;
        c2 += kr[j + 2] <= t;
        c3 += kr[j + 3] <= t;
      }
      return __reduce_add_sync(FULL, (c0 + c1) + (c2 + c3));
    };
    uint32_t lo = kmin, hi = kmax;  // invariant: count(<= hi) = c_hi >= n
    int c_hi = nv;
    while (lo < hi && c_hi != n) {
      const uint32_t mid = lo + ((hi - lo) >> 1);
      const int c = count_le(mid);
      if (c >= n) {
        hi = mid;
        c_hi = c;
      } else {
        lo = mid + 1;
      }
    }
    const uint32_t T = hi;
    const unsigned below = (1u << lane) - 1u;
    int base = 0;
    auto put = [&](bool take, int j) {
      const unsigned m = __ballot_sync(FULL, take);
      if (take) {
        const int slot = base + __popc(m & below);
        stage[slot] = key_cost(kr[j]);
        stage_i[slot] = lane + 32 * j;
      }
      base += __popc(m);
    };
    if (c_hi == n) {  // the elites are the keys <= T
#pragma unroll
      for (int j = 0; j < ELITE_REG; ++j) put(kr[j] <= T, j);
    } else {  // ties at T: the keys < T, then the lowest-index keys equal to T
      int quota = n - (T > 0u ? count_le(T - 1u) : 0);
#pragma unroll
      for (int j = 0; j < ELITE_REG; ++j) {
        const unsigned eq = __ballot_sync(FULL, kr[j] == T);
        put(kr[j] < T || (kr[j] == T && __popc(eq & below) < quota), j);
        quota -= min(__popc(eq), quota);
      }
    }
    __syncwarp();
    if (lane < n) {
      el_c = stage[lane];
      el_i = stage_i[lane];
    }
    __syncwarp();
    return;
  }
  float prev_c = -INFINITY;
  int prev_i = -1;
  for (int e = 0; e < n_e; ++e) {
    float bc = INFINITY;
    int bi = 0x7fffffff;
    for (int s = lane; s < S_c; s += 32) {
      const float v = cc[s];
      if (v == v && lex_less(prev_c, prev_i, v, s) && lex_less(v, s, bc, bi)) {
        bc = v;
        bi = s;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oc = __shfl_xor_sync(FULL, bc, o);
      const int oi = __shfl_xor_sync(FULL, bi, o);
      if (lex_less(oc, oi, bc, bi)) {
        bc = oc;
        bi = oi;
      }
    }
    if (lane == e && bi != 0x7fffffff) {
      el_c = bc;
      el_i = bi;
    }
    prev_c = bc;
    prev_i = bi;
  }
  jmin = __shfl_sync(FULL, el_c, 0);
}

__global__ void mppi_update_kernel(MppiArgs a) {
  __shared__ float jmin_s[32];
  __shared__ float stage[32][32];
  __shared__ int stage_i[32][32];
  const int d = blockIdx.x;
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* cc = a.cost + (size_t)d * a.S + (size_t)c * a.S_c;
  float el_c, jmin;
  int el_i;
  select_elites(cc, a.S_c, a.n_e, lane, stage[c], stage_i[c], el_c, el_i, jmin);
  if (lane == 0) jmin_s[c] = jmin;
  __syncthreads();
  int cbest = 0;
  for (int q = 1; q < a.C; ++q)
    if (jmin_s[q] < jmin_s[cbest]) cbest = q;
  if (threadIdx.x == 0) a.best_cost[d] = jmin_s[cbest];
  const bool mine = lane < a.n_e && el_i != 0x7fffffff;
  const float wgt = mine ? expf(-(el_c - jmin) * a.inv_lam) : 0.f;
  float wsum = wgt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
  const float inv_w = 1.f / wsum;
  const unsigned long long id =
      (unsigned long long)d * a.S + (unsigned long long)c * a.S_c + (mine ? (unsigned)el_i : 0u);
  const unsigned long long sd = *a.seed;
  uint2 keys[10];
#pragma unroll
  for (int r = 0; r < 10; ++r) keys[r] = philox_round_key((uint32_t)sd, (uint32_t)(sd >> 32), r);
  float4* mrow = reinterpret_cast<float4*>(a.mean) + ((size_t)d * a.C + c) * a.H;
  float4* prow = reinterpret_cast<float4*>(a.plan) + (size_t)d * a.H;
  float4 eps = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 last = make_float4(0.f, 0.f, 0.f, 0.f);
  // Steps in groups of G: the group's Philox + Box-Muller chains are independent
  // of each other, and its 4 G sums share one shuffle tree.  The mean rows come
  // 32 steps at a time, one per lane, each row read before the warm-start shift
  // overwrites it (row k - 1 is written at step k).
  constexpr int G = 4;
  float4 mk = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k0 = 0; k0 < a.H; k0 += G) {
    if ((k0 & 31) == 0) mk = k0 + lane < a.H ? mrow[k0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
    float2 z[G][2];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      z[u][0] = z[u][1] = make_float2(0.f, 0.f);
      if (mine && k0 + u < a.H) {
        uint32_t ct[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(k0 + u), 0u};
        philox4x32_10(ct, keys);
        z[u][0] = box_muller(ct[0], ct[1]);
        z[u][1] = box_muller(ct[2], ct[3]);
      }
    }
    float4 v[G];
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int k = k0 + u;
      const float4 m = make_float4(__shfl_sync(0xffffffffu, mk.x, k & 31),
                                   __shfl_sync(0xffffffffu, mk.y, k & 31),
                                   __shfl_sync(0xffffffffu, mk.z, k & 31),
                                   __shfl_sync(0xffffffffu, mk.w, k & 31));
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mine && k < a.H) {
        const float cx = k == 0 ? 1.f : a.rho_c;
        eps.x = fmaf(a.rho, eps.x, cx * z[u][0].x);
        eps.y = fmaf(a.rho, eps.y, cx * z[u][0].y);
        eps.z = fmaf(a.rho, eps.z, cx * z[u][1].x);
        eps.w = fmaf(a.rho, eps.w, cx * z[u][1].y);
        v[u].x = wgt * clampf(fmaf(a.sigma, eps.x, m.x), -1.f, 1.f);
        v[u].y = wgt * clampf(fmaf(a.sigma, eps.y, m.y), -1.f, 1.f);
        v[u].z = wgt * clampf(fmaf(a.sigma, eps.z, m.z), -1.f, 1.f);
        v[u].w = wgt * clampf(fmaf(a.sigma, eps.w, m.w), -1.f, 1.f);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        v[u].x += __shfl_xor_sync(0xffffffffu, v[u].x, o);
        v[u].y += __shfl_xor_sync(0xffffffffu, v[u].y, o);
        v[u].z += __shfl_xor_sync(0xffffffffu, v[u].z, o);
        v[u].w += __shfl_xor_sync(0xffffffffu, v[u].w, o);
      }
    }
#pragma unroll
    for (int u = 0; u < G; ++u) {
      const int k = k0 + u;
      if (k < a.H) {
        last = make_float4(v[u].x * inv_w, v[u].y * inv_w, v[u].z * inv_w, v[u].w * inv_w);
        if (lane == 0) {
          if (k > 0) mrow[k - 1] = last;  // warm start: shift by one step
          if (c == cbest) prow[k] = last;
        }
      }
    }
  }
  if (lane == 0) mrow[a.H - 1] = last;
}

// One warp per row of S_c costs: the row's elites (sim_mppi_select_elites).
__global__ void __launch_bounds__(256) elite_select_kernel(const float* cost, long long rows, int S_c,
                                                           int n_e, int* idx, float* jmin) {
  __shared__ float stage[8][32];
  __shared__ int stage_i[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * 8 + w;
  if (row >= rows) return;  // the whole warp leaves together
  float el_c, jm;
  int el_i;
  select_elites(cost + row * S_c, S_c, n_e, lane, stage[w], stage_i[w], el_c, el_i, jm);
  if (lane < n_e) idx[row * n_e + lane] = el_i == 0x7fffffff ? -1 : el_i;
  if (lane == 0 && jmin) jmin[row] = jm;
}

}  // namespace sp

cudaError_t launch_mppi_update(const float* cost, float* mean, float* plan, float* best_cost,
                               const unsigned long long* seed, int n, int S, int H, int C, int n_e,
                               float sigma, float rho, float lambda, cudaStream_t st) {
  sp::MppiArgs a;
  a.cost = cost;
  a.mean = mean;
  a.plan = plan;
  a.best_cost = best_cost;
  a.seed = seed;
  a.n = n;
  a.S = S;
  a.H = H;
  a.C = C;
  a.S_c = S / C;
  a.n_e = n_e;
  a.sigma = sigma;
  a.rho = rho;
  a.rho_c = sqrtf(1.f - rho * rho);
  a.inv_lam = 1.f / lambda;
  sp::mppi_update_kernel<<<n, 32 * C, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_elite_select(const float* cost, long long rows, int S_c, int n_e, int* idx,
                                float* jmin, cudaStream_t st) {
  sp::elite_select_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(cost, rows, S_c, n_e, idx, jmin);
  return cudaGetLastError();
}

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
#define CF_S(I, MO, WI)                                                      \
  return per_set ? sp::launch_t<I, MO, true, WI>(a, sc, P0, tpb, st)          \
                 : sp::launch_t<I, MO, false, WI>(a, sc, P0, tpb, st)
  if (integrator == SIM_RK4) {
    if (general_motor) CF_S(SIM_RK4, MOTOR_GENERAL, false);
    if (windowed) CF_S(SIM_RK4, MOTOR_LAG, true);
    CF_S(SIM_RK4, MOTOR_LAG, false);
  }
  if (general_motor) CF_S(SIM_EULER, MOTOR_GENERAL, false);
  if (windowed) CF_S(SIM_EULER, MOTOR_LAG, true);
  CF_S(SIM_EULER, MOTOR_LAG, false);
#undef CF_S
}

}  // namespace cf
