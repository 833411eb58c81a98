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
//  * cluster path (larger): one thread-block cluster of up to 16 CTAs per
//    (drone, controller), each CTA holding a slice of the controller's cost
//    keys in shared memory; histogram narrowing, compaction and the weighted
//    mean are split over the cluster's CTAs, which agree through distributed
//    shared memory (see the section's comment).  sim_mppi_select_elites runs
//    the same kernels without the mean.
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

// ------------------------------------------------------------------ cluster path
//
// One thread-block cluster of P CTAs (P = 1, 2, 4, 8 or 16) per (drone, controller)
// -- or per row of sim_mppi_select_elites.  CTA p owns the contiguous slice
// [p L, (p + 1) L) of the controller's S_c samples (L = ceil(S_c / P)) and keeps
// its cost keys in shared memory when the slice fits.  The CTAs of a cluster
// agree on every decision by reading each other's shared memory (distributed
// shared memory) between cluster barriers:
//  1. range and count of the controller's keys; for the update also every
//     controller's smallest cost (each CTA reads its share of all the drone's
//     costs), so each cluster knows the best controller on its own;
//  2. up to three narrowing passes: every CTA builds a 2048-bucket histogram of
//     its keys inside [lo, hi]; CTA p adds bucket range p of all the cluster's
//     histograms (reduce-scatter); every CTA then finds the bucket holding the
//     n-th smallest key from the P segment totals and that segment's buckets;
//  3. compaction in index order: CTA offsets from the cluster's counts (the
//     update needs them only when ties at the threshold are rationed), warp
//     offsets within the CTA, lanes by ballot; ties at the threshold go to the
//     lowest indices across the whole controller;
//  4. (update) each CTA averages its own elites -- every thread regenerating the
//     noise of its elites -- into per-step partial sums; after a barrier, CTA p
//     adds the P partials of its share of the steps in rank order (a fixed
//     order: repeated runs give identical results) and writes the warm-started
//     means and, in the best controller's cluster, the plan.

constexpr int CT = 512;        // threads of a cluster-path CTA
constexpr int CW = CT / 32;    // its warps
constexpr int BINS = 2048;     // buckets of one narrowing pass
constexpr int MAXE = SIM_MAX_ELITES;
constexpr int KCAP = 24576;    // cost keys of a CTA's slice kept in shared memory
constexpr int MAXC = SIM_MPPI_CLUSTER_MAX_CTRL;
constexpr int U4 = 8;          // float4 loads in flight per thread when streaming costs
constexpr int XI_F4 = 2048;    // (elite, step) noise buffer of the few-elite mean: 32 KB
constexpr int MAXP = 16;       // CTAs per cluster at most (the peer-read loops are unrolled to it)

struct ClusterArgs {
  const float* cost;  // update: [n][S]; selection: [rows][S_c]
  int S, S_c, C, n_e, P, L;
  bool cached;        // the slice's keys are kept in shared memory
  // update
  float* mean;
  float* plan;
  float* best_cost;
  const unsigned long long* seed;
  int H;
  float sigma, rho, rho_c, inv_lam;
  // selection
  int* idx;
  float* jmin;
};

struct alignas(16) ClusterSmem {
  uint32_t hist[BINS];
  uint32_t segb[BINS];       // this CTA's bucket range of the cluster-wide histogram
  float el_c[MAXE];          // this CTA's elites (costs, sample indices), index order
  int el_i[MAXE];
  // published to the cluster
  uint32_t kmin, kmax, seg_total;
  int nv, cnt_lt, cnt_eq;
  uint32_t cmin[MAXC];       // smallest key of each controller within this CTA's share
  float wsum;
  // block-local
  uint32_t wred[3][CW];
  int wcnt[2][CW];
  uint32_t g_kmin, g_kmax;
  int g_nv, bsel, before, seg_sel, cta_lt, cta_eq, cbest;
  float jmin_c, jmin_best;
};
// float4 arrays follow ClusterSmem in dynamic shared memory
static_assert(sizeof(ClusterSmem) % 16 == 0, "float4 arrays after ClusterSmem must be aligned");

template <typename T>
__device__ __forceinline__ T* peer(cg::cluster_group& cl, T* p, int rank) {
  return cl.map_shared_rank(p, rank);
}

// Key of cost i of the CTA's slice (shared memory when cached).
__device__ __forceinline__ uint32_t slice_key(const ClusterArgs& a, const uint32_t* keys,
                                              const float* cc, int s0, int i) {
  return a.cached ? keys[i - s0] : cost_key(cc[i]);
}

// f(i, x) for every i in [s0, s1) with x = base[i]: 16-byte vector loads over the
// aligned interior (U4 of them in flight per thread), scalar loads for the
// unaligned head and tail.
template <typename F>
__device__ __forceinline__ void stream_costs(const float* base, int s0, int s1, F&& f) {
  const int tid = threadIdx.x;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(base + s0);
  const int head = min(s1 - s0, (int)(((16u - (unsigned)(addr & 15u)) & 15u) >> 2));
  if (tid < head) f(s0 + tid, base[s0 + tid]);
  const int a0 = s0 + head;
  const int n4 = (s1 - a0) >> 2;
  const float4* b4 = reinterpret_cast<const float4*>(base + a0);
  for (int j = tid; j < n4; j += U4 * CT) {
    float4 v[U4];
#pragma unroll
    for (int u = 0; u < U4; ++u) {
      const int jj = j + u * CT;
      v[u] = jj < n4 ? b4[jj] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < U4; ++u) {
      const int jj = j + u * CT;
      if (jj < n4) {
        const int i = a0 + 4 * jj;
        f(i, v[u].x);
        f(i + 1, v[u].y);
        f(i + 2, v[u].z);
        f(i + 3, v[u].w);
      }
    }
  }
  const int t0 = a0 + 4 * n4;
  if (tid < s1 - t0) f(t0 + tid, base[t0 + tid]);
}

// The weighted mean of a CTA that holds few elites (n_local < CT / 2): every
// thread draws the noise of (elite, step) pairs of a chunk of steps into
// shared memory (xi[step][elite]); thread e then runs elite e's AR(1) noise,
// action and weight in step order; warp w adds the elites' values of steps
// w, w + CW, ... in a fixed order into part[k].
__device__ __forceinline__ void cta_partial_mean_few(const ClusterArgs& a, ClusterSmem& sm,
                                                     int n_local, unsigned long long base,
                                                     float jmin, const float4* mean_in,
                                                     float4* part, float4* xi, const uint2* keys,
                                                     float (*red)[16]) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const bool mine = tid < n_local;
  const float wgt = mine ? expf(-(sm.el_c[tid] - jmin) * a.inv_lam) : 0.f;
  float ws = wgt;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(FULL, ws, o);
  if (lane == 0) red[w][0] = ws;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int q = 0; q < CW; ++q) t += red[q][0];
    sm.wsum = t;
  }
  float4 eps = make_float4(0.f, 0.f, 0.f, 0.f);
  const int KS = max(1, min(a.H, XI_F4 / max(n_local, 1)));
  for (int k0 = 0; k0 < a.H; k0 += KS) {
    const int kc = min(KS, a.H - k0);
    for (int q = tid; q < n_local * kc; q += CT) {
      const int kk = q / n_local, e = q - kk * n_local;
      const unsigned long long id = base + (unsigned)sm.el_i[e];
      uint32_t ct[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(k0 + kk), 0u};
      philox4x32_10(ct, keys);
      const float2 z01 = box_muller(ct[0], ct[1]), z23 = box_muller(ct[2], ct[3]);
      xi[q] = make_float4(z01.x, z01.y, z23.x, z23.y);
    }
    __syncthreads();
    if (mine) {
      for (int kk = 0; kk < kc; ++kk) {
        const int k = k0 + kk;
        const float4 z = xi[kk * n_local + tid];
        const float cx = k == 0 ? 1.f : a.rho_c;
        eps.x = fmaf(a.rho, eps.x, cx * z.x);
        eps.y = fmaf(a.rho, eps.y, cx * z.y);
        eps.z = fmaf(a.rho, eps.z, cx * z.z);
        eps.w = fmaf(a.rho, eps.w, cx * z.w);
        const float4 m = mean_in[k];
        xi[kk * n_local + tid] = make_float4(wgt * clampf(fmaf(a.sigma, eps.x, m.x), -1.f, 1.f),
                                             wgt * clampf(fmaf(a.sigma, eps.y, m.y), -1.f, 1.f),
                                             wgt * clampf(fmaf(a.sigma, eps.z, m.z), -1.f, 1.f),
                                             wgt * clampf(fmaf(a.sigma, eps.w, m.w), -1.f, 1.f));
      }
    }
    __syncthreads();
    for (int kk = w; kk < kc; kk += CW) {
      float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int e = lane; e < n_local; e += 32) {
        const float4 v = xi[kk * n_local + e];
        t.x += v.x;
        t.y += v.y;
        t.z += v.z;
        t.w += v.w;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(FULL, t.x, o);
        t.y += __shfl_xor_sync(FULL, t.y, o);
        t.z += __shfl_xor_sync(FULL, t.z, o);
        t.w += __shfl_xor_sync(FULL, t.w, o);
      }
      if (lane == 0) part[k0 + kk] = t;
    }
    __syncthreads();  // xi is rewritten by the next chunk
  }
}

// The MPPI average of this CTA's n_local elites into part[k] (unscaled per-step
// sums over its elites) and sm.wsum; EPT elites per thread.
template <int EPT>
__device__ __forceinline__ void cta_partial_mean(const ClusterArgs& a, ClusterSmem& sm, int n_local,
                                                 unsigned long long base, float jmin,
                                                 const float4* mean_in, float4* part,
                                                 const uint2* keys, float (*red)[16]) {
  const unsigned FULL = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float wgt[EPT];
  unsigned long long id[EPT];
  float4 eps[EPT];
  float ws = 0.f;
#pragma unroll
  for (int j = 0; j < EPT; ++j) {
    const int e = tid + j * CT;
    const bool mine = e < n_local;
    wgt[j] = mine ? expf(-(sm.el_c[e] - jmin) * a.inv_lam) : 0.f;
    id[j] = base + (mine ? (unsigned)sm.el_i[e] : 0u);
    eps[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    ws += wgt[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(FULL, ws, o);
  if (lane == 0) red[w][0] = ws;
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int q = 0; q < CW; ++q) t += red[q][0];
    sm.wsum = t;
  }
  __syncthreads();  // red is rewritten below
  constexpr int G = 4;
  for (int k0 = 0; k0 < a.H; k0 += G) {
    float4 v[G];
#pragma unroll
    for (int u = 0; u < G; ++u) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < EPT; ++j) {
      if (tid + j * CT >= n_local) continue;
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
          const float4 m = mean_in[k];
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
      const int k = k0 + (tid >> 2);
      if (k < a.H) {
        float t = 0.f;
        for (int q = 0; q < CW; ++q) t += red[q][tid];
        reinterpret_cast<float*>(part)[4 * k + (tid & 3)] = t;
      }
    }
    __syncthreads();
  }
}

template <bool UPDATE>
__global__ void __launch_bounds__(CT, 1) elite_cluster_kernel(ClusterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  ClusterSmem& sm = *reinterpret_cast<ClusterSmem*>(smem);
  float4* part = reinterpret_cast<float4*>(smem + sizeof(ClusterSmem));
  float4* mean_in = part + (UPDATE ? a.H : 0);
  float4* xi = mean_in + (UPDATE ? a.H : 0);  // update: XI_F4 float4, then the keys
  uint32_t* keys = reinterpret_cast<uint32_t*>(xi + (UPDATE ? XI_F4 : 0));
  __shared__ float red[CW][16];
  __shared__ uint2 rkeys[10];
  const unsigned FULL = 0xffffffffu;
  cg::cluster_group cluster = cg::this_cluster();
  const int p = (int)cluster.block_rank();
  const int P = a.P;
  const long long grp = blockIdx.x / P;  // (drone, controller) or row
  const int c = UPDATE ? (int)(grp % a.C) : 0;
  const long long d = UPDATE ? grp / a.C : grp;
  const float* rowp = a.cost + d * (long long)a.S;
  const float* cc = rowp + (size_t)c * a.S_c;
  const int s0 = min(a.S_c, p * a.L), s1 = min(a.S_c, s0 + a.L);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float4* mrow = UPDATE ? reinterpret_cast<float4*>(a.mean) + ((size_t)d * a.C + c) * a.H : nullptr;
  if (UPDATE) {
    for (int k = tid; k < a.H; k += CT) mean_in[k] = mrow[k];
    if (tid < 10) {
      const unsigned long long sd = *a.seed;
      rkeys[tid] = philox_round_key((uint32_t)sd, (uint32_t)(sd >> 32), tid);
    }
  }
  // 1. the slice's keys, their range and count; every controller's smallest key
  uint32_t kmin = NAN_KEY, kmax = 0u;
  int nv = 0;
  stream_costs(cc, s0, s1, [&](int i, float x) {
    const uint32_t k = cost_key(x);
    if (a.cached) keys[i - s0] = k;
    if (k != NAN_KEY) {
      kmin = min(kmin, k);
      kmax = max(kmax, k);
      ++nv;
    }
  });
  uint32_t cm[MAXC];
#pragma unroll
  for (int q = 0; q < MAXC; ++q) cm[q] = NAN_KEY;
  if (UPDATE) {
    // the other controllers' minima over the same slice positions: every
    // controller's loads of a batch are issued before any is used (one round
    // trip per batch instead of one per controller)
    constexpr int UM = 4;
    for (int b = s0 + tid; b < s1; b += UM * CT) {
      float v[MAXC][UM];
#pragma unroll
      for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int u = 0; u < UM; ++u) {
          const int i = b + u * CT;
          v[q][u] = (q < a.C && q != c && i < s1) ? rowp[(size_t)q * a.S_c + i] : __int_as_float(0x7fffffff);
        }
#pragma unroll
      for (int q = 0; q < MAXC; ++q)
#pragma unroll
        for (int u = 0; u < UM; ++u) cm[q] = min(cm[q], cost_key(v[q][u]));
    }
#pragma unroll
    for (int q = 0; q < MAXC; ++q)
      if (q == c) cm[q] = kmin;
  }
  kmin = __reduce_min_sync(FULL, kmin);
  kmax = __reduce_max_sync(FULL, kmax);
  nv = __reduce_add_sync(FULL, nv);
#pragma unroll
  for (int q = 0; q < MAXC; ++q) cm[q] = __reduce_min_sync(FULL, cm[q]);
  __shared__ uint32_t wcm[CW][MAXC];
  if (lane == 0) {
    sm.wred[0][w] = kmin;
    sm.wred[1][w] = kmax;
    sm.wcnt[0][w] = nv;
#pragma unroll
    for (int q = 0; q < MAXC; ++q) wcm[w][q] = cm[q];
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t x = NAN_KEY, y = 0u;
    int z = 0;
    for (int q = 0; q < CW; ++q) {
      x = min(x, sm.wred[0][q]);
      y = max(y, sm.wred[1][q]);
      z += sm.wcnt[0][q];
    }
    sm.kmin = x;
    sm.kmax = y;
    sm.nv = z;
    for (int q = 0; q < MAXC; ++q) {
      uint32_t m = NAN_KEY;
      for (int r = 0; r < CW; ++r) m = min(m, wcm[r][q]);
      sm.cmin[q] = m;
    }
  }
  cluster.sync();  // every CTA's slice statistics are published
  if (w == 0) {  // lane r reads CTA r's statistics
    uint32_t x = NAN_KEY, y = 0u;
    int z = 0;
    uint32_t cmq[MAXC];
#pragma unroll
    for (int q = 0; q < MAXC; ++q) cmq[q] = NAN_KEY;
    if (lane < P) {
      const ClusterSmem* o = peer(cluster, &sm, lane);
      x = o->kmin;
      y = o->kmax;
      z = o->nv;
#pragma unroll
      for (int q = 0; q < MAXC; ++q) cmq[q] = o->cmin[q];
    }
    x = __reduce_min_sync(FULL, x);
    y = __reduce_max_sync(FULL, y);
    z = __reduce_add_sync(FULL, z);
#pragma unroll
    for (int q = 0; q < MAXC; ++q) cmq[q] = __reduce_min_sync(FULL, cmq[q]);
    if (lane == 0) {
      sm.g_kmin = x;
      sm.g_kmax = y;
      sm.g_nv = z;
      sm.jmin_c = z > 0 ? key_cost(x) : INFINITY;
      if (UPDATE) {  // the best controller: lowest smallest cost, ties to the lower index
        int cb = 0;
        float jb = cmq[0] != NAN_KEY ? key_cost(cmq[0]) : INFINITY;
        for (int q = 1; q < a.C; ++q) {
          const float jq = cmq[q] != NAN_KEY ? key_cost(cmq[q]) : INFINITY;
          if (jq < jb) {
            jb = jq;
            cb = q;
          }
        }
        sm.cbest = cb;
        sm.jmin_best = jb;
      }
    }
  }
  __syncthreads();
  const int gnv = sm.g_nv;
  const int n = min(a.n_e, gnv);
  // 2. narrow [lo, hi] down to the n-th smallest key (every CTA holds the same values)
  uint32_t lo = sm.g_kmin, hi = sm.g_kmax, T = hi;
  int below = 0;
  bool exact = gnv == n;  // every non-NaN key is an elite (also n == 0)
  const int SEG = BINS / P;
  while (!exact && lo < hi) {
    const int sh = max(0, 21 - __clz(hi - lo));  // (hi - lo) >> sh < 2048
    for (int b = tid; b < BINS; b += CT) sm.hist[b] = 0u;
    __syncthreads();
    for (int i = s0 + tid; i < s1; i += CT) {
      const uint32_t k = slice_key(a, keys, cc, s0, i);
      if (k >= lo && k <= hi) atomicAdd(&sm.hist[(k - lo) >> sh], 1u);
    }
    __syncthreads();
    cluster.sync();  // every CTA's histogram is complete
    // reduce-scatter: CTA p adds bucket range p of the P histograms
    uint32_t ssum = 0u;
    for (int b = tid; b < SEG; b += CT) {
      uint32_t hv[MAXP];  // all peers' loads in flight, then added in rank order
#pragma unroll
      for (int r = 0; r < MAXP; ++r) hv[r] = r < P ? peer(cluster, &sm.hist[0], r)[p * SEG + b] : 0u;
      uint32_t t = 0u;
#pragma unroll
      for (int r = 0; r < MAXP; ++r) t += hv[r];
      sm.segb[b] = t;
      ssum += t;
    }
    ssum = __reduce_add_sync(FULL, ssum);
    if (lane == 0) sm.wred[2][w] = ssum;
    __syncthreads();
    if (tid == 0) {
      uint32_t t = 0u;
      for (int q = 0; q < CW; ++q) t += sm.wred[2][q];
      sm.seg_total = t;
    }
    cluster.sync();  // the cluster-wide bucket segments are published
    const uint32_t need = (uint32_t)(n - below);
    if (w == 0) {  // lane r reads segment r's total; the first segment reaching need
      const uint32_t t = lane < P ? *peer(cluster, &sm.seg_total, lane) : 0u;
      uint32_t incl = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += x;
      }
      const unsigned hit = __ballot_sync(FULL, lane < P && incl >= need);
      const int s = hit ? __ffs(hit) - 1 : P - 1;
      const uint32_t run = __shfl_sync(FULL, incl - t, s);
      if (lane == 0) {
        sm.seg_sel = s;
        sm.before = (int)run;
        sm.bsel = s * SEG;
      }
    }
    __syncthreads();
    {
      const int s = sm.seg_sel;
      const uint32_t* sb = peer(cluster, &sm.segb[0], s);
      const uint32_t need_in = need - (uint32_t)sm.before;
      // each thread owns four consecutive buckets of the segment
      uint32_t h[4], loc = 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int b = 4 * tid + j;
        h[j] = b < SEG ? sb[b] : 0u;
        loc += h[j];
      }
      uint32_t incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += x;
      }
      if (lane == 31) sm.wred[2][w] = incl;
      __syncthreads();
      uint32_t run = incl - loc;
      for (int q = 0; q < w; ++q) run += sm.wred[2][q];
      const int before0 = sm.before;
      __syncthreads();  // every thread has read sm.before
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (run < need_in && run + h[j] >= need_in) {
          sm.bsel = s * SEG + 4 * tid + j;
          sm.before = before0 + (int)run;
        }
        run += h[j];
      }
    }
    __syncthreads();
    const int b = min(max(sm.bsel, 0), BINS - 1);
    const uint32_t cnt = peer(cluster, &sm.segb[0], b / SEG)[b % SEG];
    below += sm.before;
    lo += (uint32_t)b << sh;
    hi = (uint32_t)min((unsigned long long)hi, (unsigned long long)lo + ((1ull << sh) - 1ull));
    if (below + (int)cnt == n) {
      exact = true;
      T = hi;
    }
    cluster.sync();  // before the next pass rewrites hist, segb and the totals
  }
  if (!exact) T = lo;
  const int quota = n - below;
  // 3. compaction in index order
  const int len = s1 - s0;
  const int chunk = ((len + CW - 1) / CW + 31) & ~31;
  const int w0 = s0 + min(len, w * chunk), w1 = s0 + min(len, w * chunk + chunk);
  int c_lt = 0, c_eq = 0;
  if (n > 0) {
    for (int i = w0 + lane; i < w1; i += 32) {
      const uint32_t k = slice_key(a, keys, cc, s0, i);
      c_lt += exact ? (k <= T) : (k < T);
      c_eq += (!exact && k == T);
    }
  }
  c_lt = __reduce_add_sync(FULL, c_lt);
  c_eq = __reduce_add_sync(FULL, c_eq);
  if (lane == 0) {
    sm.wcnt[0][w] = c_lt;
    sm.wcnt[1][w] = c_eq;
  }
  __syncthreads();
  if (tid == 0) {
    int x = 0, y = 0;
    for (int q = 0; q < CW; ++q) {
      x += sm.wcnt[0][q];
      y += sm.wcnt[1][q];
    }
    sm.cnt_lt = x;
    sm.cnt_eq = y;
  }
  // Slots need the counts of the CTAs before this one: the selection's global
  // slots always, the update's local slots only when ties at the threshold are
  // rationed (every CTA takes the same branch).
  const bool need_counts = !UPDATE || !exact;
  if (need_counts) cluster.sync();  // every CTA's counts are published
  if (need_counts && w == 0) {  // lane r < p reads CTA r's counts
    int x = 0, y = 0;
    if (lane < p) {
      const ClusterSmem* o = peer(cluster, &sm, lane);
      x = o->cnt_lt;
      y = o->cnt_eq;
    }
    x = __reduce_add_sync(FULL, x);
    y = __reduce_add_sync(FULL, y);
    if (lane == 0) {
      sm.cta_lt = x;
      sm.cta_eq = y;
    }
  } else if (!need_counts && tid == 0) {
    sm.cta_lt = 0;  // unused by the update's exact case
    sm.cta_eq = 0;
  }
  __syncthreads();
  const int cta_lt = sm.cta_lt, cta_eq = sm.cta_eq;
  int lt_w = 0, eq_w = 0;
  for (int q = 0; q < w; ++q) {
    lt_w += sm.wcnt[0][q];
    eq_w += sm.wcnt[1][q];
  }
  const unsigned bel = (1u << lane) - 1u;
  if (n > 0) {
    int lt_base = lt_w, eq_base = cta_eq + eq_w;  // lt: within the CTA; eq: controller-wide
    for (int i0 = w0; i0 < w1; i0 += 32) {
      const int i = i0 + lane;
      const uint32_t k = i < w1 ? slice_key(a, keys, cc, s0, i) : NAN_KEY;
      const bool lt = exact ? k <= T : k < T;
      const bool eq = !exact && k == T;
      const unsigned mlt = __ballot_sync(FULL, lt), meq = __ballot_sync(FULL, eq);
      const int eq_before = eq_base + __popc(meq & bel);
      if (lt || (eq && eq_before < quota)) {
        const int taken_eq = min(eq_before, quota);
        if (UPDATE) {  // local slot: this CTA's elites before this one
          const int slot = lt_base + __popc(mlt & bel) + taken_eq - min(cta_eq, quota);
          if (slot < MAXE) {
            sm.el_c[slot] = key_cost(k);
            sm.el_i[slot] = i;
          }
        } else {  // controller-wide slot
          const int slot = cta_lt + lt_base + __popc(mlt & bel) + taken_eq;
          if (slot < a.n_e) a.idx[d * a.n_e + slot] = i;
        }
      }
      lt_base += __popc(mlt);
      eq_base += __popc(meq);
    }
  }
  if (!UPDATE) {
    if (p == 0) {
      for (int e = n + tid; e < a.n_e; e += CT) a.idx[d * a.n_e + e] = -1;
      if (tid == 0 && a.jmin) a.jmin[d] = sm.jmin_c;
    }
    cluster.sync();  // peers' reads of this CTA's shared memory are done
    return;
  }
  __syncthreads();
  // 4. this CTA's weighted partial sums, then the cluster's reduction in rank order
  const int n_local = n > 0 ? sm.cnt_lt + (min(cta_eq + sm.cnt_eq, quota) - min(cta_eq, quota)) : 0;
  const float jmin = sm.jmin_c;
  const unsigned long long base = (unsigned long long)d * a.S + (unsigned long long)c * a.S_c;
  if (2 * n_local < CT)
    cta_partial_mean_few(a, sm, n_local, base, jmin, mean_in, part, xi, rkeys, red);
  else if (n_local <= CT)
    cta_partial_mean<1>(a, sm, n_local, base, jmin, mean_in, part, rkeys, red);
  else if (n_local <= 2 * CT)
    cta_partial_mean<2>(a, sm, n_local, base, jmin, mean_in, part, rkeys, red);
  else if (n_local <= 4 * CT)
    cta_partial_mean<4>(a, sm, n_local, base, jmin, mean_in, part, rkeys, red);
  else
    cta_partial_mean<8>(a, sm, n_local, base, jmin, mean_in, part, rkeys, red);
  cluster.sync();  // every CTA's partial sums are published
  if (w == 0) {  // lane r reads CTA r's weight sum; added in rank order
    const float v = lane < P ? *peer(cluster, &sm.wsum, lane) : 0.f;
    float wt = 0.f;
    for (int r = 0; r < P; ++r) wt += __shfl_sync(FULL, v, r);
    if (lane == 0) red[0][0] = 1.f / wt;
  }
  __syncthreads();
  {
    const float inv_w = red[0][0];
    const int HS = (a.H + P - 1) / P;
    const int k0 = min(a.H, p * HS), k1 = min(a.H, k0 + HS);
    const bool best = sm.cbest == c;
    float* mout = reinterpret_cast<float*>(mrow);
    float* prow = a.plan + (size_t)d * a.H * 4;
    for (int x = 4 * k0 + tid; x < 4 * k1; x += CT) {
      const int k = x >> 2;
      float pv[MAXP];  // all peers' loads in flight, then added in rank order
#pragma unroll
      for (int r = 0; r < MAXP; ++r)
        pv[r] = r < P ? reinterpret_cast<const float*>(peer(cluster, part, r))[x] : 0.f;
      float t = 0.f;
#pragma unroll
      for (int r = 0; r < MAXP; ++r)
        if (r < P) t += pv[r];
      const float val = t * inv_w;
      if (k > 0) mout[x - 4] = val;        // warm start: shift by one step
      if (k == a.H - 1) mout[x] = val;     // the last step repeated
      if (best) prow[x] = val;
    }
    if (c == 0 && p == 0 && tid == 0) a.best_cost[d] = sm.jmin_best;
  }
  cluster.sync();  // peers' reads of this CTA's partial sums are done
}

}  // namespace mp

bool mppi_uses_warp_path(int S_c, int n_e) {
  return S_c <= mp::WARP_MAX_COSTS && n_e <= mp::WARP_MAX_ELITES;
}

// Whether clusters of 16 CTAs (a non-portable size, opted into per kernel) of
// this kernel can be placed on the current device with this much shared memory;
// queried once per device.
static bool cluster16_ok(void (*kern)(mp::ClusterArgs), size_t smem) {
  static int known[64][2] = {};  // per device and kernel: 0 unknown, 1 yes, -1 no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return false;
  }
  const int which = kern == mp::elite_cluster_kernel<true> ? 1 : 0;
  if (known[dev][which]) return known[dev][which] > 0;
  bool ok = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(mp::CT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
  }
  cudaGetLastError();
  known[dev][which] = ok ? 1 : -1;
  return ok;
}

// CTAs per controller on the cluster path: a power of two, up to 16 where the
// device places clusters of 16 (else 8), giving slices of at most about 6k
// costs (12k at 8 CTAs).
static int cluster_ctas(int S_c, int max_P) {
  int P = 1;
  while (P < max_P && (S_c + P - 1) / P > (max_P > 8 ? 6144 : 12288)) P *= 2;
  return P;
}

// Shared memory of a cluster-path CTA (the key cache sized for `L` keys).
static size_t cluster_smem(bool update, int H, bool cached, int L) {
  return sizeof(mp::ClusterSmem) + (update ? (2 * (size_t)H + mp::XI_F4) * sizeof(float4) : 0) +
         (cached ? (size_t)L * sizeof(uint32_t) : 0);
}

// Fills a.P, a.L and a.cached for a controller of S_c costs and launches.
static cudaError_t launch_cluster(mp::ClusterArgs& a, bool update, long long groups,
                                  cudaStream_t st) {
  auto kern = update ? mp::elite_cluster_kernel<true> : mp::elite_cluster_kernel<false>;
  // the largest shared-memory size at 16 CTAs per controller decides the probe
  const bool big = cluster16_ok(kern, cluster_smem(update, update ? SIM_MPPI_CLUSTER_MAX_H : 0, true,
                                                   mp::KCAP));
  a.P = cluster_ctas(a.S_c, big ? 16 : 8);
  a.L = (a.S_c + a.P - 1) / a.P;
  a.cached = a.L <= mp::KCAP;
  const size_t smem = cluster_smem(update, a.H, a.cached, a.L);
  if (groups * a.P >= (1ll << 31)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (a.P > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(groups * a.P), 1, 1);
  cfg.blockDim = dim3(mp::CT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

cudaError_t launch_mppi_update(const float* cost, float* mean, float* plan, float* best_cost,
                               const unsigned long long* seed, int n, int S, int H, int C, int n_e,
                               float sigma, float rho, float lambda, cudaStream_t st) {
  const int S_c = S / C;
  if (mppi_uses_warp_path(S_c, n_e)) {
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
    a.S_c = S_c;
    a.n_e = n_e;
    a.sigma = sigma;
    a.rho = rho;
    a.rho_c = sqrtf(1.f - rho * rho);
    a.inv_lam = 1.f / lambda;
    mp::mppi_update_warp_kernel<<<n, 32 * C, 0, st>>>(a);
    return cudaGetLastError();
  }
  mp::ClusterArgs a = {};
  a.cost = cost;
  a.S = S;
  a.S_c = S_c;
  a.C = C;
  a.n_e = n_e;
  a.mean = mean;
  a.plan = plan;
  a.best_cost = best_cost;
  a.seed = seed;
  a.H = H;
  a.sigma = sigma;
  a.rho = rho;
  a.rho_c = sqrtf(1.f - rho * rho);
  a.inv_lam = 1.f / lambda;
  return launch_cluster(a, true, (long long)n * C, st);
}

cudaError_t launch_elite_select(const float* cost, long long rows, int S_c, int n_e, int* idx,
                                float* jmin, cudaStream_t st) {
  if (mppi_uses_warp_path(S_c, n_e)) {
    mp::elite_select_warp_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(cost, rows, S_c, n_e,
                                                                              idx, jmin);
    return cudaGetLastError();
  }
  mp::ClusterArgs a = {};
  a.cost = cost;
  a.S = S_c;
  a.S_c = S_c;
  a.C = 1;
  a.n_e = n_e;
  a.idx = idx;
  a.jmin = jmin;
  return launch_cluster(a, false, rows, st);
}

}  // namespace cf
