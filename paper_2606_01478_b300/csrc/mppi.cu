// MPPI / iCEM update on top of the sampled rollouts (Materials and Methods,
// Model Predictive Path Integral): per controller, the elites -- the n_e
// lowest costs, ties to the lower sample index, NaN never selected -- are
// averaged with exponential weights w_e = exp(-(J_e - J_min) / lambda); the
// controller with the lowest best cost gives the plan; every controller's new
// mean is warm-started (shifted one step).  The elites' actions are not stored
// by the sampling kernel: their noise is regenerated from the same Philox
// counters.
//
// Two kernels cover the sizes:
//  * warp path (S_c <= 2048 costs and n_e <= 32 elites per controller): one
//    block per drone, one warp per controller, the costs in registers as
//    order-preserving keys and a bisection over the key range;
//  * cluster path (larger): one 512-thread CTA per (drone, controller), the
//    controllers of a drone in one thread-block cluster.  The CTA finds the
//    n_e-th smallest key with at most three 2048-bucket histogram passes over
//    the costs (the first over [min, max] of the keys, each next one inside the
//    bucket that holds it), compacts the elites into shared memory in index
//    order with one counting and one writing pass, and averages them with every
//    thread regenerating the noise of its elites.  The best controller is found
//    through distributed shared memory: each CTA publishes its J_min, and after
//    a cluster barrier every CTA reads its peers'.
#include <cooperative_groups.h>

#include <cmath>

#include "internal.h"
#include "noise.cuh"

namespace cg = cooperative_groups;

namespace cf {
namespace mp {

using noise::box_muller;
using noise::philox4x32_10;
using noise::philox_round_key;

struct MppiArgs {
  const float* cost;  // [n][S]
  float* mean;        // [n][C][H][4]: in = current means, out = updated means shifted one step
  float* plan;        // [n][H][4]: updated mean of the best controller
  float* best_cost;   // [n]
  const unsigned long long* seed;
  int n, S, H, C, S_c, n_e;
  float sigma, rho, rho_c, inv_lam;
};

// Order-preserving map of float costs to unsigned keys (-0 and +0 share a key;
// NaN maps to ~0u, above every other key, and is never selected).
constexpr uint32_t NAN_KEY = 0xFFFFFFFFu;
__device__ __forceinline__ uint32_t cost_key(float v) {
  if (v != v) return NAN_KEY;
  const uint32_t b = __float_as_uint(v + 0.f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_cost(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// ------------------------------------------------------------------ warp path

// The elites of one controller, for one warp: the n_e smallest (cost, index)
// pairs of cc[0..S_c), S_c <= 2048, ties to the lower index, NaN never
// selected.  On return lanes 0 .. n-1 hold one elite each (el_c, el_i; the
// others INFINITY and 0x7fffffff), in index order, n = min(n_e, number of
// non-NaN costs), and jmin is the smallest cost (INFINITY if there is none).
// The costs sit in registers as keys (64 per lane); a bisection over the key
// range finds the threshold T with count(key <= T) >= n, counting with warp
// reductions and stopping as soon as exactly n keys lie at or below the
// midpoint; the elites are the keys < T and the lowest-index keys equal to T up
// to n, compacted into lanes through stage[32] (cost) and stage_i[32] (index)
// in shared memory.
constexpr int ELITE_REG = 64;
constexpr int WARP_MAX_COSTS = 32 * ELITE_REG;
constexpr int WARP_MAX_ELITES = 32;
__device__ __forceinline__ void select_elites_warp(const float* cc, int S_c, int n_e, int lane,
                                                   float* stage, int* stage_i, float& el_c,
                                                   int& el_i, float& jmin) {
  const unsigned FULL = 0xffffffffu;
  el_c = INFINITY;
  el_i = 0x7fffffff;
  uint32_t kr[ELITE_REG];
  uint32_t kmin = NAN_KEY, kmax = 0u;
  int nv = 0;
  // every lane loads all its slots (clamped index) before using any: guarded
  // loads were issued one at a time
  float cv[ELITE_REG];
#pragma unroll
  for (int j = 0; j < ELITE_REG; ++j) cv[j] = cc[min(lane + 32 * j, S_c - 1)];
#pragma unroll
  for (int j = 0; j < ELITE_REG; ++j) {
    const int s = lane + 32 * j;
    kr[j] = s < S_c ? cost_key(cv[j]) : NAN_KEY;
    if (kr[j] != NAN_KEY) {
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
}

__global__ void mppi_update_warp_kernel(MppiArgs a) {
  __shared__ float jmin_s[32];
  __shared__ float stage[32][32];
  __shared__ int stage_i[32][32];
  const int d = blockIdx.x;
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* cc = a.cost + (size_t)d * a.S + (size_t)c * a.S_c;
  float el_c, jmin;
  int el_i;
  select_elites_warp(cc, a.S_c, a.n_e, lane, stage[c], stage_i[c], el_c, el_i, jmin);
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

// One warp per row of S_c <= 2048 costs: the row's elites (sim_mppi_select_elites).
__global__ void __launch_bounds__(256) elite_select_warp_kernel(const float* cost, long long rows,
                                                                int S_c, int n_e, int* idx,
                                                                float* jmin) {
  __shared__ float stage[8][32];
  __shared__ int stage_i[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * 8 + w;
  if (row >= rows) return;  // the whole warp leaves together
  float el_c, jm;
  int el_i;
  select_elites_warp(cost + row * S_c, S_c, n_e, lane, stage[w], stage_i[w], el_c, el_i, jm);
  if (lane < n_e) idx[row * n_e + lane] = el_i == 0x7fffffff ? -1 : el_i;
  if (lane == 0 && jmin) jmin[row] = jm;
}

// ------------------------------------------------------------------ block path

constexpr int BT = 512;        // threads of a block-path CTA
constexpr int BW = BT / 32;    // its warps
constexpr int BINS = 2048;     // buckets of one narrowing pass
constexpr int MAXE = SIM_MAX_ELITES;
static_assert(BINS == 4 * BT, "each thread scans four buckets");

struct alignas(16) BlockSel {
  uint32_t hist[BINS];
  float el_c[MAXE];  // the elites' costs and sample indices, in index order
  int el_i[MAXE];
  uint32_t wmin[BW], wmax[BW], wpre[BW];
  int wcnt[2][BW];
  uint32_t kmin;
  int nv, n, bsel, before;
};
// the input mean rows (float4) follow BlockSel in dynamic shared memory
static_assert(sizeof(BlockSel) % 16 == 0, "float4 rows after BlockSel must be 16-byte aligned");

// The n = min(n_e, number of non-NaN costs) elites of cc[0..S_c) into
// sm.el_c / sm.el_i (index order), with sm.n and sm.kmin (the smallest key).
// Every thread of the block calls it; it ends with a __syncthreads.
__device__ __forceinline__ void select_elites_block(const float* __restrict__ cc, int S_c, int n_e,
                                                    BlockSel& sm) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // range and count of the non-NaN keys
  uint32_t kmin = NAN_KEY, kmax = 0u;
  int nv = 0;
  for (int s = tid; s < S_c; s += BT) {
    const uint32_t k = cost_key(cc[s]);
    if (k != NAN_KEY) {
      kmin = min(kmin, k);
      kmax = max(kmax, k);
      ++nv;
    }
  }
  kmin = __reduce_min_sync(FULL, kmin);
  kmax = __reduce_max_sync(FULL, kmax);
  nv = __reduce_add_sync(FULL, nv);
  if (lane == 0) {
    sm.wmin[w] = kmin;
    sm.wmax[w] = kmax;
    sm.wcnt[0][w] = nv;
  }
  __syncthreads();
  {
    uint32_t a = NAN_KEY, b = 0u;
    int c = 0;
    for (int q = 0; q < BW; ++q) {
      a = min(a, sm.wmin[q]);
      b = max(b, sm.wmax[q]);
      c += sm.wcnt[0][q];
    }
    kmin = a;
    kmax = b;
    nv = c;
  }
  __syncthreads();  // the partials are rewritten below
  const int n = min(n_e, nv);
  if (tid == 0) {
    sm.kmin = kmin;
    sm.nv = nv;
    sm.n = n;
  }
  if (n == 0) {
    __syncthreads();
    return;
  }
  // Narrow [lo, hi] down to the n-th smallest key.  below = keys < lo.  Every
  // thread holds the same lo, hi, below and exact (read from shared memory).
  uint32_t lo = kmin, hi = kmax, T = kmax;
  int below = 0;
  bool exact = nv == n;  // every non-NaN key is an elite
  while (!exact && lo < hi) {
    const int sh = max(0, 21 - __clz(hi - lo));  // (hi - lo) >> sh < 2048
    for (int b = tid; b < BINS; b += BT) sm.hist[b] = 0u;
    if (tid == 0) {
      sm.bsel = 0;
      sm.before = 0;
    }
    __syncthreads();
    for (int s = tid; s < S_c; s += BT) {
      const uint32_t k = cost_key(cc[s]);
      if (k >= lo && k <= hi) atomicAdd(&sm.hist[(k - lo) >> sh], 1u);
    }
    __syncthreads();
    // the bucket holding the (n - below)-th smallest key of [lo, hi]: each
    // thread owns four consecutive buckets; exclusive prefix over the block
    const uint32_t need = (uint32_t)(n - below);
    uint32_t h[4], loc = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      h[j] = sm.hist[4 * tid + j];
      loc += h[j];
    }
    uint32_t incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sm.wpre[w] = incl;
    __syncthreads();
    uint32_t run = incl - loc;
    for (int q = 0; q < w; ++q) run += sm.wpre[q];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (run < need && run + h[j] >= need) {
        sm.bsel = 4 * tid + j;
        sm.before = (int)run;
      }
      run += h[j];
    }
    __syncthreads();
    const int b = min(max(sm.bsel, 0), BINS - 1);
    const uint32_t cnt = sm.hist[b];
    below += sm.before;
    lo += (uint32_t)b << sh;
    hi = (uint32_t)min((unsigned long long)hi, (unsigned long long)lo + ((1ull << sh) - 1ull));
    if (below + (int)cnt == n) {  // exactly n keys at or below this bucket's top
      exact = true;
      T = hi;
    }
    __syncthreads();  // hist, wpre, bsel are rewritten by the next pass
  }
  if (!exact) T = lo;  // lo == hi: the keys < T, then the quota lowest-index keys equal to T
  const int quota = n - below;
  // Compaction in index order: warp w owns the contiguous range [s0, s1).
  const int chunk = ((S_c + BW - 1) / BW + 31) & ~31;
  const int s0 = min(S_c, w * chunk), s1 = min(S_c, s0 + chunk);
  int c_lt = 0, c_eq = 0;
  for (int s = s0 + lane; s < s1; s += 32) {
    const uint32_t k = cost_key(cc[s]);
    c_lt += exact ? (k <= T) : (k < T);
    c_eq += (!exact && k == T);
  }
  c_lt = __reduce_add_sync(FULL, c_lt);
  c_eq = __reduce_add_sync(FULL, c_eq);
  if (lane == 0) {
    sm.wcnt[0][w] = c_lt;
    sm.wcnt[1][w] = c_eq;
  }
  __syncthreads();
  int lt_base = 0, eq_base = 0;
  for (int q = 0; q < w; ++q) {
    lt_base += sm.wcnt[0][q];
    eq_base += sm.wcnt[1][q];
  }
  const unsigned bel = (1u << lane) - 1u;
  for (int s = s0; s < s1; s += 32) {
    const int i = s + lane;
    const uint32_t k = i < s1 ? cost_key(cc[i]) : NAN_KEY;  // NaN key: neither below nor at T
    const bool lt = exact ? k <= T : k < T;
    const bool eq = !exact && k == T;
    const unsigned mlt = __ballot_sync(FULL, lt), meq = __ballot_sync(FULL, eq);
    const int eq_before = eq_base + __popc(meq & bel);
    if (lt || (eq && eq_before < quota)) {
      const int slot = lt_base + __popc(mlt & bel) + min(eq_before, quota);
      if (slot < MAXE) {  // slot < n <= MAXE by construction
        sm.el_c[slot] = key_cost(k);
        sm.el_i[slot] = i;
      }
    }
    lt_base += __popc(mlt);
    eq_base += __popc(meq);
  }
  __syncthreads();
}

// Weighted mean of the elites of one controller, every thread regenerating the
// noise of elites e = tid + j BT (j < EPT).  Sums per group of G steps: a warp
// shuffle tree, then the warps' partials added in warp order (fixed order, so
// repeated runs give identical results).
template <int EPT>
__device__ __forceinline__ void weighted_mean_block(const MppiArgs& a, const BlockSel& sm,
                                                    const float4* mrow_in, float* mrow_out,
                                                    float* prow, bool best, int d, int c,
                                                    float jmin, const uint2* keys,
                                                    float (*red)[16]) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int n = sm.n;
  float wgt[EPT];
  unsigned long long id[EPT];
  float4 eps[EPT];
  float ws = 0.f;
  const unsigned long long base = (unsigned long long)d * a.S + (unsigned long long)c * a.S_c;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = tid + j * BT;
    const bool mine = e < n;
    wgt[j] = mine ? expf(-(sm.el_c[e] - jmin) * a.inv_lam) : 0.f;
    id[j] = base + (mine ? (unsigned)sm.el_i[e] : 0u);
    eps[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    ws += wgt[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(FULL, ws, o);
  if (lane == 0) red[w][0] = ws;
  __syncthreads();
  float wsum = 0.f;
  for (int q = 0; q < BW; ++q) wsum += red[q][0];
  const float inv_w = 1.f / wsum;
  __syncthreads();  // red is rewritten below
  constexpr int G = 4;
  for (int k0 = 0; k0 < a.H; k0 += G) {
    float4 v[G];
#pragma unroll
    for (int u = 0; u < G; ++u) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (tid + j * BT >= n) continue;
      float2 z[G][2];
#pragma unroll
      for (int u = 0; u < G; ++u) {
        z[u][0] = z[u][1] = make_float2(0.f, 0.f);
        if (k0 + u < a.H) {
          uint32_t ct[4] = {(uint32_t)id[j], (uint32_t)(id[j] >> 32), (uint32_t)(k0 + u), 0u};
          philox4x32_10(ct, keys);
          z[u][0] = box_muller(ct[0], ct[1]);
          z[u][1] = box_muller(ct[2], ct[3]);
        }
      }
#pragma unroll
      for (int u = 0; u < G; ++u) {
        const int k = k0 + u;
        if (k < a.H) {
          const float cx = k == 0 ? 1.f : a.rho_c;
          float4& e = eps[j];
          e.x = fmaf(a.rho, e.x, cx * z[u][0].x);
          e.y = fmaf(a.rho, e.y, cx * z[u][0].y);
          e.z = fmaf(a.rho, e.z, cx * z[u][1].x);
          e.w = fmaf(a.rho, e.w, cx * z[u][1].y);
          const float4 m = mrow_in[k];
          v[u].x += wgt[j] * clampf(fmaf(a.sigma, e.x, m.x), -1.f, 1.f);
          v[u].y += wgt[j] * clampf(fmaf(a.sigma, e.y, m.y), -1.f, 1.f);
          v[u].z += wgt[j] * clampf(fmaf(a.sigma, e.z, m.z), -1.f, 1.f);
          v[u].w += wgt[j] * clampf(fmaf(a.sigma, e.w, m.w), -1.f, 1.f);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        v[u].x += __shfl_xor_sync(FULL, v[u].x, o);
        v[u].y += __shfl_xor_sync(FULL, v[u].y, o);
        v[u].z += __shfl_xor_sync(FULL, v[u].z, o);
        v[u].w += __shfl_xor_sync(FULL, v[u].w, o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < G; ++u) {
        red[w][4 * u] = v[u].x;
        red[w][4 * u + 1] = v[u].y;
        red[w][4 * u + 2] = v[u].z;
        red[w][4 * u + 3] = v[u].w;
      }
    }
    __syncthreads();
    if (tid < 4 * G) {
      const int k = k0 + (tid >> 2), ch = tid & 3;
      if (k < a.H) {
        float t = 0.f;
        for (int q = 0; q < BW; ++q) t += red[q][tid];
        const float val = t * inv_w;
        if (k > 0) mrow_out[4 * (k - 1) + ch] = val;  // warm start: shift by one step
        if (k == a.H - 1) mrow_out[4 * k + ch] = val;  // the last step repeated
        if (best) prow[4 * k + ch] = val;
      }
    }
    __syncthreads();
  }
}

// One CTA per (drone, controller); the C controllers of a drone form one
// cluster (cluster rank = controller).  Dynamic shared memory: BlockSel, then
// the controller's H input mean rows.
__global__ void __launch_bounds__(BT, 1) mppi_update_cluster_kernel(MppiArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  BlockSel& sm = *reinterpret_cast<BlockSel*>(smem);
  float4* mrow_in = reinterpret_cast<float4*>(smem + sizeof(BlockSel));
  __shared__ float red[BW][16];
  __shared__ uint2 keys[10];
  __shared__ float jmin_s;
  __shared__ int cbest_s;
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int d = blockIdx.x / a.C;
  const int tid = threadIdx.x;
  float4* mrow = reinterpret_cast<float4*>(a.mean) + ((size_t)d * a.C + c) * a.H;
  for (int k = tid; k < a.H; k += BT) mrow_in[k] = mrow[k];
  if (tid < 10) {
    const unsigned long long sd = *a.seed;
    keys[tid] = philox_round_key((uint32_t)sd, (uint32_t)(sd >> 32), tid);
  }
  select_elites_block(a.cost + (size_t)d * a.S + (size_t)c * a.S_c, a.S_c, a.n_e, sm);
  if (tid == 0) jmin_s = sm.n > 0 ? key_cost(sm.kmin) : INFINITY;
  cluster.sync();  // every controller's J_min is published
  if (tid == 0) {
    int cb = 0;
    float jb = *cluster.map_shared_rank(&jmin_s, 0);
    for (int q = 1; q < a.C; ++q) {
      const float jq = *cluster.map_shared_rank(&jmin_s, q);
      if (jq < jb) {
        jb = jq;
        cb = q;
      }
    }
    cbest_s = cb;
    if (c == 0) a.best_cost[d] = jb;
  }
  cluster.sync();  // the peers' reads are done before any CTA moves on (or exits)
  const int n = sm.n;
  const float jmin = jmin_s;
  const bool best = cbest_s == c;
  float* mout = reinterpret_cast<float*>(mrow);
  float* prow = a.plan + (size_t)d * a.H * 4;
  if (n <= BT)
    weighted_mean_block<1>(a, sm, mrow_in, mout, prow, best, d, c, jmin, keys, red);
  else if (n <= 2 * BT)
    weighted_mean_block<2>(a, sm, mrow_in, mout, prow, best, d, c, jmin, keys, red);
  else if (n <= 4 * BT)
    weighted_mean_block<4>(a, sm, mrow_in, mout, prow, best, d, c, jmin, keys, red);
  else
    weighted_mean_block<8>(a, sm, mrow_in, mout, prow, best, d, c, jmin, keys, red);
}

// One CTA per row (sim_mppi_select_elites beyond the warp path's sizes).
__global__ void __launch_bounds__(BT, 1) elite_select_block_kernel(const float* cost, int S_c,
                                                                   int n_e, int* idx, float* jmin) {
  extern __shared__ __align__(16) unsigned char smem[];
  BlockSel& sm = *reinterpret_cast<BlockSel*>(smem);
  const long long row = blockIdx.x;
  select_elites_block(cost + row * S_c, S_c, n_e, sm);
  const int n = sm.n;
  for (int e = threadIdx.x; e < n_e; e += BT) idx[row * n_e + e] = e < n ? sm.el_i[e] : -1;
  if (threadIdx.x == 0 && jmin) jmin[row] = n > 0 ? key_cost(sm.kmin) : INFINITY;
}

}  // namespace mp

bool mppi_uses_warp_path(int S_c, int n_e) {
  return S_c <= mp::WARP_MAX_COSTS && n_e <= mp::WARP_MAX_ELITES;
}

cudaError_t launch_mppi_update(const float* cost, float* mean, float* plan, float* best_cost,
                               const unsigned long long* seed, int n, int S, int H, int C, int n_e,
                               float sigma, float rho, float lambda, cudaStream_t st) {
  mp::MppiArgs a;
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
  if (mppi_uses_warp_path(a.S_c, n_e)) {
    mp::mppi_update_warp_kernel<<<n, 32 * C, 0, st>>>(a);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(mp::BlockSel) + (size_t)H * sizeof(float4);
  cudaError_t e = cudaFuncSetAttribute(mp::mppi_update_cluster_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)((long long)n * C), 1, 1);
  cfg.blockDim = dim3(mp::BT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mp::mppi_update_cluster_kernel, a);
}

cudaError_t launch_elite_select(const float* cost, long long rows, int S_c, int n_e, int* idx,
                                float* jmin, cudaStream_t st) {
  if (mppi_uses_warp_path(S_c, n_e)) {
    mp::elite_select_warp_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(cost, rows, S_c, n_e,
                                                                              idx, jmin);
    return cudaGetLastError();
  }
  const size_t smem = sizeof(mp::BlockSel);
  cudaError_t e = cudaFuncSetAttribute(mp::elite_select_block_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mp::elite_select_block_kernel<<<(unsigned)rows, mp::BT, smem, st>>>(cost, S_c, n_e, idx, jmin);
  return cudaGetLastError();
}

}  // namespace cf
