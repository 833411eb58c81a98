// Differentiable policy rollout (backpropagation through time).
//
// The paper trains policies with exact analytic gradients through the unrolled
// dynamics and the onboard controller stack (Materials and Methods,
// Backpropagation Through Time).  Here, per drone:
//   obs_k = [p_k - r_k, q_k, v_k, w_k];  a_k = MLP(obs_k)  (13 -> 64 -> 64 -> 4, tanh)
//   x_{k+1} = R Euler steps of the first-principles model under the attitude
//             interface with action a_k held (controller, mixer, motor lag,
//             Eqs. 1-6); R = 1, or 10 for a 50 Hz policy on 500 Hz physics
//   L = (1/M) sum_w sum_k |p_{k+1} - r_{k+1}|^2 + w_act |a_k|^2          (squared objective)
// or the paper's tracking reward (BPTT section, reward equation), as a loss:
//   L = (1/M) sum_w sum_k -exp(-2 |p_{k+1} - r_{k+1}|) + w_theta theta_{k+1}
//         + sum_i w_act,i a_k,i^2 + w_dact,i (a_k,i - a_{k-1},i)^2,   a_{-1} = 0,
//   theta = 2 atan2(|(qx, qy)|, |(qz, qw)|) the tilt from upright.
// Forward kernel: rollout + loss, checkpoints of x (and, for the reward, of the
// previous action) every C steps.
// Backward kernel: per segment, recompute the C R sub-step states from the
// checkpoint, then sweep them in reverse with the hand-written adjoint of the step and of
// the MLP; accumulate dL/dW per CTA; dL/dx0 per drone.
//
// Layout: one CTA = 4 warps = 64 drones; warp v owns drones 16v..16v+15 of the
// CTA (one m16 MMA tile; lane l handles drone l & 15 of the tile for the
// per-drone dynamics, lanes 16..31 duplicate lanes 0..15).  The MLP runs on
// tensor cores with mma.sync m16n8k16 (bf16 inputs, fp32 accumulate).  Weights
// are bf16 values; by default (LO) activations and adjoints enter the MMAs as
// hi + lo bf16 pairs (2 MMAs, ~2^-16 relative), dW products as hi*hi + hi*lo +
// lo*hi; without LO only the hi parts are multiplied (plain bf16 operands,
// ~2^-8 relative), the precision-for-speed variant.
// The accumulator fragment of one layer is the A fragment of the next, so
// activations stay in registers between layers.
#include <cuda_bf16.h>

#include "internal.h"
#include "physics.cuh"

namespace cf {
namespace ro {

constexpr int OFF_W1 = 0, OFF_B1 = 832, OFF_W2 = 896, OFF_B2 = 4992, OFF_W3 = 5056,
              OFF_B3 = 5312, NPOL = 5316, NPOL_PAD = 5376;
constexpr int TPB = 128, DPC = 64;  // threads and drones per CTA
constexpr int S16 = 24, S64 = 72;   // padded smem row strides (bf16 elements)

struct __align__(16) Smem {
  __nv_bfloat16 W1[64 * S16];  // [i][c]  (c < 13 used)
  __nv_bfloat16 W2[64 * S64];  // [j][i]
  __nv_bfloat16 W3[16 * S64];  // [o][j]  (o < 4 used)
  __nv_bfloat16 obs[2][DPC * S16];  // hi, lo; column 13 = 1 (bias column); the adjoint's recompute
  // activation tiles [buffer][hi, lo] (column 64 = 1): the adjoint's reverse sweep
  // reads step k from buffer k & 1 while step k - 1 is prepared in the other
  __nv_bfloat16 h1[2][2][DPC * S64];
  __nv_bfloat16 h2[2][2][DPC * S64];
  // adjoint tiles [step parity][hi, lo]: written by the compute warps at step k,
  // read by the weight-gradient warps while the compute warps run step k - 1
  __nv_bfloat16 dz1[2][2][DPC * S64];
  __nv_bfloat16 dz2[2][2][DPC * S64];
  __nv_bfloat16 dz3[2][2][DPC * S16];
  __nv_bfloat16 obsr[2][2][DPC * S16];  // the reverse sweep's observation tiles (dW1 operand)
  float b1[64], b2[64], b3[8];
  float act[DPC][4];  // the actions of the forward rollout and of the adjoint's recompute
  // the adjoint's recompute: one h2 tile per warp, hi then lo, staged for the bulk
  // stores into the activation cache (column 64 = 1, the bias column of the tiles)
  __nv_bfloat16 stage[4][16 * S64];
  float dobs[DPC][16];
  // adjoint kernel: double-buffered prefetch of the next step's state row, its
  // step record (StepRecord: five float4) and previous action (cp.async)
  float pre_x[2][DPC][20];
  float pre_q[2][DPC][20];
  float4 pre_a[2][DPC];
  float actb[2][DPC][4];  // actions of the reverse sweep [buffer]
  // reverse-sweep hand-off per step parity: full (4 compute-warp arrivals: the
  // step's tiles are written), empty (4 weight-gradient-warp arrivals: read);
  // ready[v][b]: buffer b holds step k's activations, actions and observation rows
  // for warp v's rows (32 arrivals of the warp that prepared it); per segment
  // parity: seg_done (4 recompute-warp arrivals: the segment is written), seg_free
  // (4 weight-gradient-warp arrivals: the segment has been swept)
  unsigned long long full[2], empty[2];
  unsigned long long ready[4][2];
  unsigned long long seg_done[2], seg_free[2];
};
static_assert(sizeof(Smem) <= 227 * 1024, "one CTA per SM within the opt-in shared-memory limit");

struct RolloutArgs {
  const float* x0;        // [n][20]
  const uint16_t* w;      // [NPOL] bf16 bits, packed W1 b1 W2 b2 W3 b3
  const float* p_ref;     // [H + 1][n][3]
  float* ckpt;            // [n_ckpt][n][20]
  float* seg;             // [2][C R + 1][n][20] recomputed segment states by segment parity
  float* seg_q;           // [2][C R][n][FQ_FLOATS] their step records (StepRecord)
  float* loss_w;          // [n] per-drone loss
  float* part;            // [n_cta][NPOL_PAD] dW partials
  float* dx0;             // [n][20]
  uint4* hcache;          // [2][C][n_warps][CACHE_CHUNKS] h2 and actions per step, by segment parity
  const float* dL;        // device scalar: upstream gradient of the loss
  uint32_t* status;       // device status word or null (SIM_FLAG_TIMEOUT when a bounded wait gave up)
  float4* ckpt_a;         // [n_ckpt][n] previous action at each checkpoint (reward objective)
  float4* seg_a;          // [2][C][n] previous action of each segment step (reward objective)
  int n, H, C, R;
  int fused;              // adjoint kernel: run the forward pass first (sim_rollout_grad)
  float dt, w_act, inv_n;
  float w_theta, w_a[4], w_da[4];  // tracking-reward weights
  int store_ckpt;
};

// ------------------------------------------------------------------ MMA helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Asynchronous global -> shared copies (sm_80+ cp.async), completed by the
// issuing thread's cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t r[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t r[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}

// D += A (16x16, row) * B (16x8, col); bf16 inputs, fp32 accumulators.
__device__ __forceinline__ void mma(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// x ~= hi + lo with hi = bf16(x), lo = bf16(x - hi); two values per 32-bit word.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 f = __bfloat1622float2(h);
  __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
  hi = *reinterpret_cast<uint32_t*>(&h);
  lo = *reinterpret_cast<uint32_t*>(&l);
}

__device__ __forceinline__ float2 unpack2(uint32_t hi, uint32_t lo) {
  const float2 h = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&hi));
  const float2 l = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&lo));
  return make_float2(h.x + l.x, h.y + l.y);
}

// A fragments (hi, lo) of k-tile kk from accumulator fragments c[8][4]
// (n-tiles 2kk, 2kk+1 form the 16 columns of k-tile kk).
__device__ __forceinline__ void c_to_a(const float c[8][4], int kk, uint32_t ah[4], uint32_t al[4]) {
  split2(c[2 * kk][0], c[2 * kk][1], ah[0], al[0]);
  split2(c[2 * kk][2], c[2 * kk][3], ah[1], al[1]);
  split2(c[2 * kk + 1][0], c[2 * kk + 1][1], ah[2], al[2]);
  split2(c[2 * kk + 1][2], c[2 * kk + 1][3], ah[3], al[3]);
}

// Fragment rows and columns of an x4 matrix move (ldmatrix / stmatrix): lanes 8j..8j+7
// address the rows of 8x8 matrix j = (rows 0-7 | 8-15) x (columns +0 | +8) of a
// 16 x 16 block, the order of an A fragment (c_to_a) of one k-tile.
__device__ __forceinline__ int frag_row(int lane) { return (lane & 7) + ((lane >> 3) & 1) * 8; }
__device__ __forceinline__ int frag_col(int lane) { return (lane >> 4) * 8; }

__device__ __forceinline__ void stsm_x4(void* p, const uint32_t r[4]) {
  asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(smem_addr(p)),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
               : "memory");
}

// Store accumulator fragments c[8][4] (rows r0 + g, r0 + g + 8; 64 columns) as
// hi/lo bf16 into a [*][S64] tile pair: per k-tile, the A fragments' hi and lo
// words go out by one matrix store each (rows of 144 bytes keep the eight rows of
// each 8x8 matrix on distinct banks).
__device__ __forceinline__ void store_c64(__nv_bfloat16 (*t)[DPC * S64], int r0, int lane,
                                          const float c[8][4]) {
  const int at = (r0 + frag_row(lane)) * S64 + frag_col(lane);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t h[4], l[4];
    c_to_a(c, kk, h, l);
    stsm_x4(&t[0][at + 16 * kk], h);
    stsm_x4(&t[1][at + 16 * kk], l);
  }
}

// Reload accumulator-fragment values (hi + lo) from a [*][S64] tile pair.
__device__ __forceinline__ void load_c64(__nv_bfloat16 (*t)[DPC * S64], int r0, int lane,
                                         float c[8][4]) {
  const int at = (r0 + frag_row(lane)) * S64 + frag_col(lane);
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t h[4], l[4];
    ldsm_x4(h, &t[0][at + 16 * kk]);
    ldsm_x4(l, &t[1][at + 16 * kk]);
    const float2 a0 = unpack2(h[0], l[0]), a1 = unpack2(h[1], l[1]);
    const float2 a2 = unpack2(h[2], l[2]), a3 = unpack2(h[3], l[3]);
    c[2 * kk][0] = a0.x;
    c[2 * kk][1] = a0.y;
    c[2 * kk][2] = a1.x;
    c[2 * kk][3] = a1.y;
    c[2 * kk + 1][0] = a2.x;
    c[2 * kk + 1][1] = a2.y;
    c[2 * kk + 1][2] = a3.x;
    c[2 * kk + 1][3] = a3.y;
  }
}

// ------------------------------------------------------------------ MLP

__device__ void load_weights(Smem& s, const uint16_t* __restrict__ w) {
  const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(w);
  const __nv_bfloat16 z = __float2bfloat16(0.f);
  for (int e = threadIdx.x; e < 64 * S16; e += blockDim.x) {
    const int i = e / S16, c = e % S16;
    s.W1[e] = c < 13 ? wb[OFF_W1 + i * 13 + c] : z;
  }
  for (int e = threadIdx.x; e < 64 * S64; e += blockDim.x) {
    const int j = e / S64, i = e % S64;
    s.W2[e] = i < 64 ? wb[OFF_W2 + j * 64 + i] : z;
  }
  for (int e = threadIdx.x; e < 16 * S64; e += blockDim.x) {
    const int o = e / S64, j = e % S64;
    s.W3[e] = (o < 4 && j < 64) ? wb[OFF_W3 + o * 64 + j] : z;
  }
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    s.b1[e] = __bfloat162float(wb[OFF_B1 + e]);
    s.b2[e] = __bfloat162float(wb[OFF_B2 + e]);
  }
  if (threadIdx.x < 8) s.b3[threadIdx.x] = threadIdx.x < 4 ? __bfloat162float(wb[OFF_B3 + threadIdx.x]) : 0.f;
  // constant columns of the activation tiles: 1 in the bias column, 0 padding
  const __nv_bfloat16 one = __float2bfloat16(1.f);
  for (int r = threadIdx.x; r < DPC; r += blockDim.x) {
    for (int c = 64; c < S64; ++c) {
      for (int b = 0; b < 2; ++b) {
        s.h1[b][0][r * S64 + c] = c == 64 ? one : z;
        s.h1[b][1][r * S64 + c] = z;
        s.h2[b][0][r * S64 + c] = c == 64 ? one : z;
        s.h2[b][1][r * S64 + c] = z;
      }
      for (int b = 0; b < 2; ++b) {
        s.dz1[b][0][r * S64 + c] = z;
        s.dz1[b][1][r * S64 + c] = z;
        s.dz2[b][0][r * S64 + c] = z;
        s.dz2[b][1][r * S64 + c] = z;
      }
    }
    for (int c = 64; c < S64; ++c) s.stage[r >> 4][(r & 15) * S64 + c] = c == 64 ? one : z;
    for (int c = 0; c < S16; ++c) {
      s.obs[0][r * S16 + c] = z;
      s.obs[1][r * S16 + c] = z;
      for (int b = 0; b < 2; ++b) {
        s.dz3[b][0][r * S16 + c] = z;
        s.dz3[b][1][r * S16 + c] = z;
        s.obsr[b][0][r * S16 + c] = z;
        s.obsr[b][1][r * S16 + c] = z;
      }
    }
  }
}

// Write one drone's observation row (hi, lo; bias column 13 = 1).
__device__ __forceinline__ void put_obs(__nv_bfloat16 (*t)[DPC * S16], int row, const float* x, const float r[3]) {
  float o[16];
  o[0] = x[0] - r[0];
  o[1] = x[1] - r[1];
  o[2] = x[2] - r[2];
#pragma unroll
  for (int j = 3; j < 13; ++j) o[j] = x[j];
  o[13] = 1.f;
  o[14] = 0.f;
  o[15] = 0.f;
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    uint32_t h, l;
    split2(o[j], o[j + 1], h, l);
    *reinterpret_cast<uint32_t*>(&t[0][row * S16 + j]) = h;
    *reinterpret_cast<uint32_t*>(&t[1][row * S16 + j]) = l;
  }
}

// The same row written by both half-warps (which hold the same drones): columns
// 8 half .. 8 half + 7.  Used by the adjoint's warp roles (half the work per lane
// there: forward + adjoint 1.552 -> 1.514 ms); the forward kernel, whose step is one
// warp's chain, measured 0.36 -> 0.48 ms with it and keeps the whole-row form.
__device__ __forceinline__ void put_obs_half(__nv_bfloat16 (*t)[DPC * S16], int row, const float* x,
                                             const float r[3], int half) {
  float o[8];
  if (half == 0) {
    o[0] = x[0] - r[0];
    o[1] = x[1] - r[1];
    o[2] = x[2] - r[2];
#pragma unroll
    for (int j = 3; j < 8; ++j) o[j] = x[j];
  } else {
#pragma unroll
    for (int j = 0; j < 5; ++j) o[j] = x[8 + j];
    o[5] = 1.f;
    o[6] = 0.f;
    o[7] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < 8; j += 2) {
    uint32_t h, l;
    split2(o[j], o[j + 1], h, l);
    *reinterpret_cast<uint32_t*>(&t[0][row * S16 + 8 * half + j]) = h;
    *reinterpret_cast<uint32_t*>(&t[1][row * S16 + 8 * half + j]) = l;
  }
}

// tanh from its definition, tanh x = 1 - 2 / (exp(2 x) + 1), on the hardware
// base-2 exponential and reciprocal approximations: absolute error about 2e-7 for
// either sign (the activations then enter the tensor cores as hi + lo bf16 pairs,
// ~2^-16 relative); saturates to +1 (the exponential overflows to infinity, the
// reciprocal to 0) and to -1 (the exponential underflows to 0).
__device__ __forceinline__ float tanh_fast(float x) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x * 2.88539008177792681f));  // 2 / ln 2
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(e + 1.f));
  return fmaf(-2.f, r, 1.f);
}

// Two tanh values for one reciprocal: with p = exp(2 |a|) + 1 and q = exp(2 |b|) + 1,
// 1/p = q / (p q) and 1/q = p / (p q) (about 2 ulp apart from the separate
// reciprocals).  |x| is clamped to 15 first, where tanh already rounds to +-1 in
// float, so that p q stays finite.
__device__ __forceinline__ void tanh_pair(float& a, float& b) {
  float ea, eb, r;
  const float ya = fminf(fabsf(a), 15.f) * 2.88539008177792681f;
  const float yb = fminf(fabsf(b), 15.f) * 2.88539008177792681f;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ea) : "f"(ya));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(eb) : "f"(yb));
  const float p = ea + 1.f, q = eb + 1.f;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p * q));
  a = copysignf(fmaf(-2.f, r * q, 1.f), a);
  b = copysignf(fmaf(-2.f, r * p, 1.f), b);
}

// The MLP's activations: separate reciprocals with hi + lo operands (their
// latency-bound chain measured slower with the pairing: forward 0.375 ->
// 0.403 ms), paired with plain bf16 operands (fewer XU operations: forward
// 0.326 -> 0.311 ms, forward + adjoint 1.421 -> 1.382 ms).
template <bool LO>
__device__ __forceinline__ void tanh2(float& a, float& b) {
  if constexpr (LO) {
    a = tanh_fast(a);
    b = tanh_fast(b);
  } else {
    tanh_pair(a, b);
  }
}

// Layer 1 of the MLP for the warp's 16 drones (rows r0..r0+15) from an obs tile
// pair (hi, lo): h1 (fp32 accumulator fragments, after tanh).
template <bool LO>
__device__ __forceinline__ void mlp_layer1(Smem& s, const __nv_bfloat16 (*obs)[DPC * S16], int r0,
                                           int lane, float h1[8][4]) {
  const int tq = lane & 3;
  const int arow = r0 + (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  uint32_t oh[4], ol[4];
  ldsm_x4(oh, &obs[0][arow * S16 + acol]);
  ldsm_x4(ol, &obs[1][arow * S16 + acol]);
  // z1[d][i] = sum_c obs[d][c] W1[i][c] + b1[i]
  const int brow = (lane & 7) + (lane >> 4) * 8, bcol = ((lane >> 3) & 1) * 8;
  // the hi products of all eight n-tiles, then the lo ones: consecutive MMAs
  // accumulate into different tiles (each tile's order is hi, lo either way)
  uint32_t b[4][4];
#pragma unroll
  for (int n = 0; n < 8; n += 2) ldsm_x4(b[n >> 1], &s.W1[(8 * n + brow) * S16 + bcol]);
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float b0 = s.b1[8 * n + 2 * tq], b1v = s.b1[8 * n + 2 * tq + 1];
    float* c = h1[n];
    c[0] = b0;
    c[1] = b1v;
    c[2] = b0;
    c[3] = b1v;
    mma(c, oh, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
  }
  if constexpr (LO) {
#pragma unroll
    for (int n = 0; n < 8; ++n) mma(h1[n], ol, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
  }
#pragma unroll
  for (int n = 0; n < 8; ++n)
#pragma unroll
    for (int e = 0; e < 4; e += 2) tanh2<LO>(h1[n][e], h1[n][e + 1]);
}

// MLP forward for the warp's 16 drones (rows r0..r0+15).  Returns h1, h2
// (fp32 accumulator fragments, after tanh) and writes the actions to act.
template <bool LO>
__device__ void mlp_forward(Smem& s, int r0, int lane, float h1[8][4], float h2[8][4],
                            float (*act)[4]) {
  const int g = lane >> 2, tq = lane & 3;
  const int bcol = ((lane >> 3) & 1) * 8, brow = (lane & 7) + (lane >> 4) * 8;
  mlp_layer1<LO>(s, s.obs, r0, lane, h1);
  // layer 2: z2[d][j] = sum_i h1[d][i] W2[j][i] + b2[j]
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    const float b0 = s.b2[8 * n + 2 * tq], b1v = s.b2[8 * n + 2 * tq + 1];
    h2[n][0] = b0;
    h2[n][1] = b1v;
    h2[n][2] = b0;
    h2[n][3] = b1v;
  }
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t ah[4], al[4];
    c_to_a(h1, kk, ah, al);
    uint32_t b[4][4];
#pragma unroll
    for (int n = 0; n < 8; n += 2) ldsm_x4(b[n >> 1], &s.W2[(8 * n + brow) * S64 + 16 * kk + bcol]);
#pragma unroll
    for (int n = 0; n < 8; ++n) mma(h2[n], ah, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    if constexpr (LO) {
#pragma unroll
      for (int n = 0; n < 8; ++n) mma(h2[n], al, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    }
  }
#pragma unroll
  for (int n = 0; n < 8; ++n)
#pragma unroll
    for (int e = 0; e < 4; e += 2) tanh2<LO>(h2[n][e], h2[n][e + 1]);
  // layer 3: z3[d][o] = sum_j h2[d][j] W3[o][j] + b3[o]
  float z3[4];
  z3[0] = s.b3[2 * tq];
  z3[1] = s.b3[2 * tq + 1];
  z3[2] = z3[0];
  z3[3] = z3[1];
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t ah[4], al[4];
    c_to_a(h2, kk, ah, al);
    uint32_t b[2];
    ldsm_x2(b, &s.W3[(lane & 7) * S64 + 16 * kk + bcol]);
    mma(z3, ah, b[0], b[1]);
    if constexpr (LO) mma(z3, al, b[0], b[1]);
  }
  if (tq < 2) {
    act[r0 + g][2 * tq] = tanh_fast(z3[0]);
    act[r0 + g][2 * tq + 1] = tanh_fast(z3[1]);
    act[r0 + g + 8][2 * tq] = tanh_fast(z3[2]);
    act[r0 + g + 8][2 * tq + 1] = tanh_fast(z3[3]);
  }
}

// MLP backward for the warp's 16 drones, given dz3 rows in s.dz3 and the
// forward activations in buffer b of s.h1 / s.h2 (hi + lo).  Writes dz1, dz2 tiles and the
// observation adjoint into s.dobs.
template <bool LO>
__device__ void mlp_backward(Smem& s, int r0, int lane, int b, float sb2[8][2]) {
  const int g = lane >> 2, tq = lane & 3;
  const int arow = r0 + (lane & 7) + ((lane >> 3) & 1) * 8, acol = (lane >> 4) * 8;
  // transposed B fragments: storage [k][n]
  const int trow = (lane & 7) + ((lane >> 3) & 1) * 8, tcol = (lane >> 4) * 8;
  float d[8][4];
  // dh2[d][j] = sum_o dz3[d][o] W3[o][j]
  {
    uint32_t ah[4], al[4];
    ldsm_x4(ah, &s.dz3[b][0][arow * S16 + acol]);
    ldsm_x4(al, &s.dz3[b][1][arow * S16 + acol]);
    uint32_t b[4][4];
#pragma unroll
    for (int n = 0; n < 8; n += 2) ldsm_x4_t(b[n >> 1], &s.W3[trow * S64 + 8 * n + tcol]);
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      d[n][0] = d[n][1] = d[n][2] = d[n][3] = 0.f;
      mma(d[n], ah, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    }
    if constexpr (LO) {
#pragma unroll
      for (int n = 0; n < 8; ++n) mma(d[n], al, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    }
  }
  // dz2 = dh2 (1 - h2^2)
  {
    float h[8][4];
    load_c64(s.h2[b], r0, lane, h);
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) d[n][e] *= fmaf(-h[n][e], h[n][e], 1.f);
  }
  // db2: this lane's two drones (rows g, g + 8) of columns 8 n + 2 tq, + 1
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    sb2[n][0] += d[n][0] + d[n][2];
    sb2[n][1] += d[n][1] + d[n][3];
  }
  store_c64(s.dz2[b], r0, lane, d);
  // dh1[d][i] = sum_j dz2[d][j] W2[j][i]
  float e1[8][4];
#pragma unroll
  for (int n = 0; n < 8; ++n) e1[n][0] = e1[n][1] = e1[n][2] = e1[n][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t ah[4], al[4];
    c_to_a(d, kk, ah, al);
    uint32_t b[4][4];
#pragma unroll
    for (int n = 0; n < 8; n += 2) ldsm_x4_t(b[n >> 1], &s.W2[(16 * kk + trow) * S64 + 8 * n + tcol]);
#pragma unroll
    for (int n = 0; n < 8; ++n) mma(e1[n], ah, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    if constexpr (LO) {
#pragma unroll
      for (int n = 0; n < 8; ++n) mma(e1[n], al, b[n >> 1][2 * (n & 1)], b[n >> 1][2 * (n & 1) + 1]);
    }
  }
  // dz1 = dh1 (1 - h1^2)
  {
    float h[8][4];
    load_c64(s.h1[b], r0, lane, h);
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int e = 0; e < 4; ++e) e1[n][e] *= fmaf(-h[n][e], h[n][e], 1.f);
  }
  store_c64(s.dz1[b], r0, lane, e1);
  // dobs[d][c] = sum_i dz1[d][i] W1[i][c]
  float o[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    uint32_t ah[4], al[4];
    c_to_a(e1, kk, ah, al);
    uint32_t b[4];
    ldsm_x4_t(b, &s.W1[(16 * kk + trow) * S16 + tcol]);
    mma(o[0], ah, b[0], b[1]);
    mma(o[1], ah, b[2], b[3]);
    if constexpr (LO) mma(o[0], al, b[0], b[1]);
    if constexpr (LO) mma(o[1], al, b[2], b[3]);
  }
#pragma unroll
  for (int n = 0; n < 2; ++n) {
    s.dobs[r0 + g][8 * n + 2 * tq] = o[n][0];
    s.dobs[r0 + g][8 * n + 2 * tq + 1] = o[n][1];
    s.dobs[r0 + g + 8][8 * n + 2 * tq] = o[n][2];
    s.dobs[r0 + g + 8][8 * n + 2 * tq + 1] = o[n][3];
  }
}

// dW accumulation over the CTA's 64 drones for this step (warp v's slice):
//   dW2 rows j in [16v, 16v+16) x columns 0..63
//   dW1 rows i in [16v, 16v+16) x columns 0..15 (13 = bias b1)
//   dW3 transposed: rows j in [16v, 16v+16) x columns o in [0, 8) (o < 4 used)
// (db2 and db3, the sums of dz2 and dz3 over drones and steps, are summed by the
// compute warps, which hold dz2 and dz3 in registers.)
struct DwAcc {
  float w2[8][4];
  float w1[2][4];
  float w3[4];
};

template <bool LO>
__device__ void accumulate_dw(Smem& s, int v, int lane, DwAcc& acc, int hb) {
  // A = dz^T: A(row m, col d) = dz[d][m], storage [d][m] -> transposed load
  const int arow = (lane & 7) + (lane >> 4) * 8, acol = ((lane >> 3) & 1) * 8;
  // B(k = d, n) = act[d][n], storage [d][n] -> transposed load
  const int brow = (lane & 7) + ((lane >> 3) & 1) * 8, bcol = (lane >> 4) * 8;
#pragma unroll
  for (int kd = 0; kd < 4; ++kd) {
    const int d0 = 16 * kd;
    uint32_t ah[4], al[4];
    // dW2
    ldsm_x4_t(ah, &s.dz2[hb][0][(d0 + arow) * S64 + 16 * v + acol]);
    ldsm_x4_t(al, &s.dz2[hb][1][(d0 + arow) * S64 + 16 * v + acol]);
    // four n-tiles at a time, product by product (hi hi, hi lo, lo hi), so that
    // consecutive MMAs accumulate into different tiles (each tile's order is kept)
#pragma unroll
    for (int n0 = 0; n0 < 8; n0 += 4) {
      uint32_t bh[2][4], bl[2][4];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        ldsm_x4_t(bh[p], &s.h1[hb][0][(d0 + brow) * S64 + 8 * (n0 + 2 * p) + bcol]);
        if constexpr (LO) ldsm_x4_t(bl[p], &s.h1[hb][1][(d0 + brow) * S64 + 8 * (n0 + 2 * p) + bcol]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) mma(acc.w2[n0 + q], ah, bh[q >> 1][2 * (q & 1)], bh[q >> 1][2 * (q & 1) + 1]);
      if constexpr (LO) {
#pragma unroll
        for (int q = 0; q < 4; ++q) mma(acc.w2[n0 + q], ah, bl[q >> 1][2 * (q & 1)], bl[q >> 1][2 * (q & 1) + 1]);
#pragma unroll
        for (int q = 0; q < 4; ++q) mma(acc.w2[n0 + q], al, bh[q >> 1][2 * (q & 1)], bh[q >> 1][2 * (q & 1) + 1]);
      }
    }
    // dW1
    ldsm_x4_t(ah, &s.dz1[hb][0][(d0 + arow) * S64 + 16 * v + acol]);
    ldsm_x4_t(al, &s.dz1[hb][1][(d0 + arow) * S64 + 16 * v + acol]);
    {
      uint32_t bh[4], bl[4];
      ldsm_x4_t(bh, &s.obsr[hb][0][(d0 + brow) * S16 + bcol]);
      ldsm_x4_t(bl, &s.obsr[hb][1][(d0 + brow) * S16 + bcol]);
#pragma unroll
      for (int u = 0; u < 2; ++u) mma(acc.w1[u], ah, bh[2 * u], bh[2 * u + 1]);
      if constexpr (LO) {
#pragma unroll
        for (int u = 0; u < 2; ++u) mma(acc.w1[u], ah, bl[2 * u], bl[2 * u + 1]);
#pragma unroll
        for (int u = 0; u < 2; ++u) mma(acc.w1[u], al, bh[2 * u], bh[2 * u + 1]);
      }
    }
    // dW3^T = h2^T dz3: A = h2^T (rows j of this warp's slice), B = dz3 (k = d,
    // n = o; 4 of its 8 columns used) -- one n-tile where dW3 = dz3^T h2 would
    // spend two m-tiles on the 4 used output rows
    ldsm_x4_t(ah, &s.h2[hb][0][(d0 + arow) * S64 + 16 * v + acol]);
    if constexpr (LO) ldsm_x4_t(al, &s.h2[hb][1][(d0 + arow) * S64 + 16 * v + acol]);
    {
      uint32_t bh[2], bl[2];
      ldsm_x2_t(bh, &s.dz3[hb][0][(d0 + brow) * S16]);
      if constexpr (LO) ldsm_x2_t(bl, &s.dz3[hb][1][(d0 + brow) * S16]);
      mma(acc.w3, ah, bh[0], bh[1]);
      if constexpr (LO) {
        mma(acc.w3, ah, bl[0], bl[1]);
        mma(acc.w3, al, bh[0], bh[1]);
      }
    }
  }
}

__device__ void store_dw(const DwAcc& acc, int v, int lane, float* __restrict__ part) {
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int rr = g + (e >= 2 ? 8 : 0), cc = 2 * tq + (e & 1);
    // dW2
#pragma unroll
    for (int n = 0; n < 8; ++n) part[OFF_W2 + (16 * v + rr) * 64 + 8 * n + cc] = acc.w2[n][e];
    // dW1 / db1
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const int i = 16 * v + rr, c = 8 * n + cc;
      if (c < 13) part[OFF_W1 + i * 13 + c] = acc.w1[n][e];
      else if (c == 13) part[OFF_B1 + i] = acc.w1[n][e];
    }
    // dW3 (transposed slice: row j, column o)
    if (cc < 4) part[OFF_W3 + cc * 64 + 16 * v + rr] = acc.w3[e];
  }
}

// ------------------------------------------------------------------ dynamics

// Euler step of the first-principles model under the attitude interface
// (first-order-lag rotors, no drag), a = the policy action.
// The attitude error is taken from quaternions (attitude_command_q, attitude_error2_q:
// the same e_R as the matrix form) and the thrust direction from q.
__device__ __forceinline__ void policy_step(float* x, const float a[4], const DevParams& P, float dt) {
  float qd[4], Td, ex, ey, ez, tx, ty, tz, Wc[4], d[17];
  attitude_command_q(make_float4(a[0], a[1], a[2], a[3]), P, qd, Td);
  attitude_error2_q(x, qd, ex, ey, ez);
  attitude_torque_e(ex, ey, ez, x[10], x[11], x[12], P, tx, ty, tz);
  mixer(Td, tx, ty, tz, P, Wc);
  deriv_fp<MOTOR_LAG>(x, Wc, P, false, d);
  // element pairs on the packed FP32 instructions (same rounding as fmaf per lane)
  const float2 dt2 = make_float2(dt, dt);
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const float2 r = __ffma2_rn(dt2, make_float2(d[j], d[j + 1]), make_float2(x[j], x[j + 1]));
    x[j] = r.x;
    x[j + 1] = r.y;
  }
  x[16] = fmaf(dt, d[16], x[16]);
  const float in = rsqrt_approx(fmaf(x[3], x[3], fmaf(x[4], x[4], fmaf(x[5], x[5], x[6] * x[6]))));
  x[3] *= in;
  x[4] *= in;
  x[5] *= in;
  x[6] *= in;
}

// Forward quantities of one policy_step that its adjoint needs besides the
// pre- and post-step states: 1 / |q~| of the normalisation, the mixer's factors
// d W_cmd / d f per rotor (0 where the thrust clip or a zero command stops the
// gradient), the attitude error's parts (v, w) = qd2* (x) q, twice the desired
// quaternion qd2 and the half-angle products it is built from.
constexpr int FQ_FLOATS = 20;  // 19 used; rows of five float4
struct StepRecord {
  float in, gWf[4], vx, vy, vz, we, dx, dy, dz, dw, sr, cr, ka, kb, kc, kd;
};

// policy_step that also records the step's forward quantities (the same
// arithmetic as policy_step: the state comes out bit for bit the same).
__device__ __forceinline__ void policy_step_rec(float* x, const float a[4], const DevParams& P, float dt,
                                                StepRecord& q) {
  const float ac0 = clampf(a[0], -1.f, 1.f), ac1 = clampf(a[1], -1.f, 1.f);
  const float ac2 = clampf(a[2], -1.f, 1.f), ac3 = clampf(a[3], -1.f, 1.f);
  float sr, cr, sp, cp, sy, cy;  // of the half angles
  __sincosf(ac0 * P.half_max_angle, &sr, &cr);
  __sincosf(ac1 * P.half_max_angle, &sp, &cp);
  __sincosf(ac2 * P.half_max_angle, &sy, &cy);
  const float cp2 = cp + cp, sp2 = sp + sp;
  const float ka = cp2 * cy, kb = sp2 * sy, kc = sp2 * cy, kd = cp2 * sy;
  // twice the desired quaternion (attitude_command_q)
  const float dx = fmaf(sr, ka, -cr * kb), dy = fmaf(cr, kc, sr * kd);
  const float dz = fmaf(cr, kd, -sr * kc), dw = fmaf(cr, ka, sr * kb);
  const float Td = fmaf(P.ts_mg, ac3, P.mg);
  const float qx = x[3], qy = x[4], qz = x[5], qw = x[6];
  // (v, w) = qd2* (x) q, 2 e_R = w v (attitude_error2_q)
  const float vx = fmaf(dw, qx, fmaf(-qw, dx, fmaf(-dy, qz, dz * qy)));
  const float vy = fmaf(dw, qy, fmaf(-qw, dy, fmaf(-dz, qx, dx * qz)));
  const float vz = fmaf(dw, qz, fmaf(-qw, dz, fmaf(-dx, qy, dy * qx)));
  const float we = fmaf(dw, qw, fmaf(dx, qx, fmaf(dy, qy, dz * qz)));
  float tx, ty, tz;
  attitude_torque_e(we * vx, we * vy, we * vz, x[10], x[11], x[12], P, tx, ty, tz);
  const float A = 0.25f * Td, X = tx * P.mix_a, Y = ty * P.mix_a, Z = tz * P.mix_k;
  float f[4], Wc[4];
  f[0] = (A - X) - (Y + Z);
  f[1] = (A - X) + (Y + Z);
  f[2] = (A + X) + (Y - Z);
  f[3] = (A + X) - (Y - Z);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    Wc[r] = sqrt_approx(clampf(f[r], 0.f, P.fmax) * P.inv_kf);
    // W = sqrt(f / kf): dW/df = 1 / (2 kf W) inside the clip
    const bool pass = f[r] >= 0.f && f[r] <= P.fmax && Wc[r] > 0.f;
    q.gWf[r] = pass ? __fdividef(0.5f * P.inv_kf, Wc[r]) : 0.f;
  }
  float d[17];
  deriv_fp<MOTOR_LAG>(x, Wc, P, false, d);
  // element pairs on the packed FP32 instructions (same rounding as fmaf per lane)
  const float2 dt2 = make_float2(dt, dt);
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const float2 r = __ffma2_rn(dt2, make_float2(d[j], d[j + 1]), make_float2(x[j], x[j + 1]));
    x[j] = r.x;
    x[j + 1] = r.y;
  }
  x[16] = fmaf(dt, d[16], x[16]);
  const float in = rsqrt_approx(fmaf(x[3], x[3], fmaf(x[4], x[4], fmaf(x[5], x[5], x[6] * x[6]))));
  x[3] *= in;
  x[4] *= in;
  x[5] *= in;
  x[6] *= in;
  q.in = in;
  q.vx = vx;
  q.vy = vy;
  q.vz = vz;
  q.we = we;
  q.dx = dx;
  q.dy = dy;
  q.dz = dz;
  q.dw = dw;
  q.sr = sr;
  q.cr = cr;
  q.ka = ka;
  q.kb = kb;
  q.kc = kc;
  q.kd = kd;
}

__device__ __forceinline__ void store_record(float* __restrict__ base, int i, const StepRecord& q) {
  float4* p = reinterpret_cast<float4*>(base + (size_t)i * FQ_FLOATS);
  p[0] = make_float4(q.in, q.gWf[0], q.gWf[1], q.gWf[2]);
  p[1] = make_float4(q.gWf[3], q.vx, q.vy, q.vz);
  p[2] = make_float4(q.we, q.dx, q.dy, q.dz);
  p[3] = make_float4(q.dw, q.sr, q.cr, q.ka);
  p[4] = make_float4(q.kb, q.kc, q.kd, 0.f);
}
__device__ __forceinline__ void record_from(const float* f, StepRecord& q) {
  q.in = f[0];
  q.gWf[0] = f[1];
  q.gWf[1] = f[2];
  q.gWf[2] = f[3];
  q.gWf[3] = f[4];
  q.vx = f[5];
  q.vy = f[6];
  q.vz = f[7];
  q.we = f[8];
  q.dx = f[9];
  q.dy = f[10];
  q.dz = f[11];
  q.dw = f[12];
  q.sr = f[13];
  q.cr = f[14];
  q.ka = f[15];
  q.kb = f[16];
  q.kc = f[17];
  q.kd = f[18];
}

// Adjoint of policy_step.  In: x (pre-step state), xn (post-step state), the
// step's record q, a, lam = dL/dx_{k+1}.  Out: lam = dL/dx_k through the step (the
// observation path is added by the caller), ga = dL/da through the controller.
__device__ void policy_step_adjoint(const float* x, const float* xn, const StepRecord& q, const float a[4],
                                    float* lam, float ga[4], const DevParams& P, float dt) {
  const float in = q.in;
  const float vx = q.vx, vy = q.vy, vz = q.vz, we = q.we;
  const float dx = q.dx, dy = q.dy, dz = q.dz, dw = q.dw;
  const float sr = q.sr, cr = q.cr, ka = q.ka, kb = q.kb, kc = q.kc, kd = q.kd;
  const float qx = x[3], qy = x[4], qz = x[5], qw = x[6];
  const float wx = x[10], wy = x[11], wz = x[12];
  // ---------------- reverse: normalisation q' = qt / |qt|
  {
    // the normalised quaternion is the post-step state's (policy_step's q~ in)
    const float q0 = xn[3], q1 = xn[4], q2 = xn[5], q3 = xn[6];
    const float dot = fmaf(q0, lam[3], fmaf(q1, lam[4], fmaf(q2, lam[5], q3 * lam[6])));
    lam[3] = (lam[3] - q0 * dot) * in;
    lam[4] = (lam[4] - q1 * dot) * in;
    lam[5] = (lam[5] - q2 * dot) * in;
    lam[6] = (lam[6] - q3 * dot) * in;
  }
  // x_tilde = x + dt * xdot: mu = dt * lam (adjoint of xdot); lam stays (identity)
  float mu[17];
#pragma unroll
  for (int j = 0; j < 17; ++j) mu[j] = dt * lam[j];
  // p' = v
  lam[7] += mu[0];
  lam[8] += mu[1];
  lam[9] += mu[2];
  // q' = 1/2 q (x) [w, 0]
  lam[3] += 0.5f * (-wz * mu[4] + wy * mu[5] - wx * mu[6]);
  lam[4] += 0.5f * (wz * mu[3] - wx * mu[5] - wy * mu[6]);
  lam[5] += 0.5f * (-wy * mu[3] + wx * mu[4] - wz * mu[6]);
  lam[6] += 0.5f * (wx * mu[3] + wy * mu[4] + wz * mu[5]);
  float gwx = 0.5f * (qw * mu[3] + qz * mu[4] - qy * mu[5] - qx * mu[6]);
  float gwy = 0.5f * (-qz * mu[3] + qw * mu[4] + qx * mu[5] - qy * mu[6]);
  float gwz = 0.5f * (qy * mu[3] - qx * mu[4] + qw * mu[5] - qz * mu[6]);
  // v' = (T/m) R e_z - g e_z
  const float s0 = x[13] * x[13], s1 = x[14] * x[14], s2 = x[15] * x[15], s3 = x[16] * x[16];
  const float T = P.kf * ((s0 + s1) + (s2 + s3));
  const float Tm = T * P.inv_m;
  const float r02 = 2.f * fmaf(qx, qz, qw * qy);
  const float r12 = 2.f * fmaf(qy, qz, -qw * qx);
  const float r22 = (qw * qw + qz * qz) - (qx * qx + qy * qy);
  const float gT = P.inv_m * fmaf(mu[7], r02, fmaf(mu[8], r12, mu[9] * r22));
  {
    const float g02 = Tm * mu[7], g12 = Tm * mu[8], g22 = Tm * mu[9];
    lam[3] += 2.f * (qz * g02 - qw * g12 - qx * g22);
    lam[4] += 2.f * (qw * g02 + qz * g12 - qy * g22);
    lam[5] += 2.f * (qx * g02 + qy * g12 + qz * g22);
    lam[6] += 2.f * (qy * g02 - qx * g12 + qw * g22);
  }
  // w' = tau_rotor / J + (cJx wy wz, cJy wz wx, cJz wx wy)
  const float gtx = mu[10] * P.inv_Jx, gty = mu[11] * P.inv_Jy, gtz = mu[12] * P.inv_Jz;
  gwx += P.cJy * wz * mu[11] + P.cJz * wy * mu[12];
  gwy += P.cJx * wz * mu[10] + P.cJz * wx * mu[12];
  gwz += P.cJx * wy * mu[10] + P.cJy * wx * mu[11];
  // rotor wrench of s_i = W_i^2
  const float gs0 = P.kf * gT - P.kfa * gtx - P.kfa * gty - P.km * gtz;
  const float gs1 = P.kf * gT - P.kfa * gtx + P.kfa * gty + P.km * gtz;
  const float gs2 = P.kf * gT + P.kfa * gtx + P.kfa * gty - P.km * gtz;
  const float gs3 = P.kf * gT + P.kfa * gtx - P.kfa * gty + P.km * gtz;
  lam[13] += 2.f * x[13] * gs0 - P.cv_up * mu[13];
  lam[14] += 2.f * x[14] * gs1 - P.cv_up * mu[14];
  lam[15] += 2.f * x[15] * gs2 - P.cv_up * mu[15];
  lam[16] += 2.f * x[16] * gs3 - P.cv_up * mu[16];
  // ---------------- controller: W_cmd -> mixer -> torque -> attitude error
  float gf[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) gf[r] = P.cv_up * mu[13 + r] * q.gWf[r];
  const float gA = (gf[0] + gf[1]) + (gf[2] + gf[3]);
  const float gX = (gf[2] + gf[3]) - (gf[0] + gf[1]);
  const float gY = (gf[1] + gf[2]) - (gf[0] + gf[3]);
  const float gZ = (gf[1] + gf[3]) - (gf[0] + gf[2]);
  const float gTd = 0.25f * gA;
  const float gtcx = P.mix_a * gX, gtcy = P.mix_a * gY, gtcz = P.mix_k * gZ;
  // tau = -KRJh e - KwJ w  (e = 2 e_R)
  const float gex = -P.KRJh_x * gtcx, gey = -P.KRJh_y * gtcy, gez = -P.KRJh_z * gtcz;
  gwx -= P.KwJ_x * gtcx;
  gwy -= P.KwJ_y * gtcy;
  gwz -= P.KwJ_z * gtcz;
  lam[10] += gwx;
  lam[11] += gwy;
  lam[12] += gwz;
  // 2 e_R = w v with (v, w) = qd2* (x) q: gw = ge . v, gv = w ge
  const float gw_ = fmaf(gex, vx, fmaf(gey, vy, gez * vz));
  const float gvx = gex * we, gvy = gey * we, gvz = gez * we;
  // through q (v and w are bilinear in qd2 and q)
  lam[3] += fmaf(gvx, dw, fmaf(-gvy, dz, fmaf(gvz, dy, gw_ * dx)));
  lam[4] += fmaf(gvx, dz, fmaf(gvy, dw, fmaf(-gvz, dx, gw_ * dy)));
  lam[5] += fmaf(-gvx, dy, fmaf(gvy, dx, fmaf(gvz, dw, gw_ * dz)));
  lam[6] += fmaf(-gvx, dx, fmaf(-gvy, dy, fmaf(-gvz, dz, gw_ * dw)));
  // through qd2
  const float gdx = fmaf(-gvx, qw, fmaf(gvy, qz, fmaf(-gvz, qy, gw_ * qx)));
  const float gdy = fmaf(-gvx, qz, fmaf(-gvy, qw, fmaf(gvz, qx, gw_ * qy)));
  const float gdz = fmaf(gvx, qy, fmaf(-gvy, qx, fmaf(-gvz, qw, gw_ * qz)));
  const float gdw = fmaf(gvx, qx, fmaf(gvy, qy, fmaf(gvz, qz, gw_ * qw)));
  // qd2 = 2 qz(yaw) (x) qy(pitch) (x) qx(roll) of the half angles hr, hp, hy:
  // d qd2 / d hr = (dw, dz, -dy, -dx); with ka = 2 cp cy, kb = 2 sp sy, kc = 2 sp cy,
  // kd = 2 cp sy, d/d hp maps (ka, kb, kc, kd) to (-kc, kd, ka, -kb) and d/d hy to
  // (-kd, kc, -kb, ka)
  const float gphi = fmaf(gdx, dw, fmaf(gdy, dz, fmaf(-gdz, dy, -gdw * dx)));
  const float gth = fmaf(-gdx, fmaf(sr, kc, cr * kd), fmaf(gdy, fmaf(cr, ka, -sr * kb),
                    fmaf(-gdz, fmaf(cr, kb, sr * ka), gdw * fmaf(sr, kd, -cr * kc))));
  const float gpsi = fmaf(-gdx, fmaf(sr, kd, cr * kc), fmaf(gdy, fmaf(sr, ka, -cr * kb),
                     fmaf(gdz, fmaf(cr, ka, sr * kb), gdw * fmaf(sr, kc, -cr * kd))));
  // clip(a, -1, 1) passes the gradient inside [-1, 1] (inclusive)
  ga[0] = (a[0] >= -1.f && a[0] <= 1.f) ? gphi * P.half_max_angle : 0.f;
  ga[1] = (a[1] >= -1.f && a[1] <= 1.f) ? gth * P.half_max_angle : 0.f;
  ga[2] = (a[2] >= -1.f && a[2] <= 1.f) ? gpsi * P.half_max_angle : 0.f;
  ga[3] = (a[3] >= -1.f && a[3] <= 1.f) ? gTd * P.ts_mg : 0.f;
}

__device__ __forceinline__ void load_row(const float* __restrict__ base, int i, float* x) {
  const float4* p = reinterpret_cast<const float4*>(base + (size_t)i * 20);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 v = p[j];
    x[4 * j] = v.x;
    x[4 * j + 1] = v.y;
    x[4 * j + 2] = v.z;
    x[4 * j + 3] = v.w;
  }
  x[16] = base[(size_t)i * 20 + 16];
}

__device__ __forceinline__ void store_row(float* __restrict__ base, int i, const float* x) {
  float4* p = reinterpret_cast<float4*>(base + (size_t)i * 20);
#pragma unroll
  for (int j = 0; j < 4; ++j) p[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
  p[4] = make_float4(x[16], 0.f, 0.f, 0.f);
}

// Prefetch helper (one lane per drone): a 20-float row (a state row or a step record).
static_assert(FQ_FLOATS == 20, "step records prefetch like state rows");
__device__ __forceinline__ void prefetch_row(float* dst, const float* __restrict__ base, int i) {
  const float* q = base + (size_t)i * 20;
#pragma unroll
  for (int j = 0; j < 5; ++j) cp_async16(dst + 4 * j, q + 4 * j);
}

__device__ __forceinline__ void ref_at(const float* __restrict__ p_ref, int k, int n, int i,
                                      float r[3]) {
  const float* q = p_ref + ((size_t)k * n + i) * 3;
  r[0] = q[0];
  r[1] = q[1];
  r[2] = q[2];
}

__device__ __forceinline__ void ref_at_pinned(const float* __restrict__ p_ref, int k, int n, int i,
                                             float r[3]) {
  const float* q = p_ref + ((size_t)k * n + i) * 3;
  asm volatile("ld.global.nc.f32 %0, [%3];\n\tld.global.nc.f32 %1, [%3+4];\n\tld.global.nc.f32 %2, [%3+8];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]) : "l"(q));
}

// ------------------------------------------------------------------ activation cache

// One warp's cached step (rows 16 v..16 v + 15 at one step of a segment) is three
// contiguous runs, laid out as they sit in shared memory: its 16 rows of h2 hi and
// of h2 lo (TILE_CHUNKS 16-byte chunks each, padded rows as in the tiles) and its
// 16 action rows.  The recompute warp writes it from its staging tile, the
// weight-gradient warp that prepares the step copies it into the tile buffers,
// both as bulk copies (cp.async.bulk: one thread, the copy engine of the SM).
constexpr int TILE_CHUNKS = 16 * S64 * 2 / 16, CACHE_CHUNKS = 2 * TILE_CHUNKS + 16;
constexpr uint32_t TILE_BYTES = TILE_CHUNKS * 16, ACT_BYTES = 16 * 16;
constexpr uint32_t CACHE_BYTES = 2 * TILE_BYTES + ACT_BYTES;
static_assert(CACHE_BYTES == CACHE_CHUNKS * 16, "cache entry = two tiles + action rows");
static_assert(offsetof(Smem, h2) % 16 == 0 && offsetof(Smem, actb) % 16 == 0 && offsetof(Smem, act) % 16 == 0 &&
                  offsetof(Smem, stage) % 16 == 0 && (DPC * S64 * 2) % 16 == 0 && (16 * S64 * 2) % 16 == 0,
              "bulk copies start on 16-byte boundaries");

// L2 priorities of the cache traffic: an entry is written once per segment and
// read back once in the reverse sweep, so its writes ask L2 to keep it
// (evict_last) and its read marks it as done (evict_first); once consumed it is
// dropped from L2 without a write-back (cache_discard).
__device__ __forceinline__ unsigned long long l2_keep() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_done() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_s2g(void* g, const void* sm, uint32_t bytes,
                                         unsigned long long pol) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;\n" ::"l"(g),
               "r"(smem_addr(sm)), "r"(bytes), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* sm, const void* g, uint32_t bytes,
                                         unsigned long long* mbar, unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
          smem_addr(sm)),
      "l"(g), "r"(bytes), "r"(smem_addr(mbar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// wait until none of this thread's bulk groups still reads its source
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
// wait until all of this thread's bulk groups have completed (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// order this thread's shared-memory writes before bulk copies that read them
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// order global-memory accesses of bulk copies with this thread's synchronisation
// (after the writer's completed bulk stores, before the reader's bulk loads)
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
}
// raise the transaction count of the barrier's current phase (no arrival)
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(m)), "r"(bytes)
               : "memory");
}

// The recompute warp's copy-out of one step: h2 (after tanh) through its staging
// tile, hi then lo (one tile of shared memory: each copy has read the tile before
// the next part is staged), and its action rows from act.
__device__ __forceinline__ void cache_put(Smem& s, int v, int r0, int lane, const float h2[8][4], uint4* g) {
  __nv_bfloat16* t = s.stage[v];
  const int at = frag_row(lane) * S64 + frag_col(lane);
  const unsigned long long pol = l2_keep();
  if (lane == 0) bulk_wait_read();  // the previous step's lo copy
  __syncwarp();
#pragma unroll
  for (int half = 0; half < 2; ++half) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      uint32_t h[4], l[4];
      c_to_a(h2, kk, h, l);
      stsm_x4(&t[at + 16 * kk], half ? l : h);
    }
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) {
      bulk_s2g(g + half * TILE_CHUNKS, t, TILE_BYTES, pol);
      if (!half) bulk_s2g(g + 2 * TILE_CHUNKS, s.act[r0], ACT_BYTES, pol);
      bulk_commit();
      if (!half) bulk_wait_read();
    }
    __syncwarp();
  }
}

// Bring cache entry g back into rows r0..r0+15 of buffer b; the barrier's phase
// waits for all CACHE_BYTES (besides its arrivals).
__device__ __forceinline__ void cache_load(Smem& s, int b, int r0, const uint4* g,
                                           unsigned long long* mbar) {
  const unsigned long long pol = l2_done();
  mbar_expect_tx(mbar, CACHE_BYTES);
  bulk_g2s(s.h2[b][0] + r0 * S64, g, TILE_BYTES, mbar, pol);
  bulk_g2s(s.h2[b][1] + r0 * S64, g + TILE_CHUNKS, TILE_BYTES, mbar, pol);
  bulk_g2s(s.actb[b][r0], g + 2 * TILE_CHUNKS, ACT_BYTES, mbar, pol);
}

// Drop a consumed cache entry from L2 without writing it back: the lanes of the
// warp invalidate its 128-byte lines (entries start on 128-byte boundaries: the
// workspace is 256-byte aligned and CACHE_BYTES is a multiple of 128).
static_assert(CACHE_BYTES % 128 == 0, "cache entries are whole 128-byte lines");
__device__ __forceinline__ void cache_discard(const uint4* g, int lane) {
  const char* e = reinterpret_cast<const char*>(g);
  for (int l = lane; l < (int)(CACHE_BYTES / 128); l += 32)
    asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(e + 128 * l) : "memory");
}

// ------------------------------------------------------------------ objectives

// Loss of one step: x = post-step state, r = reference at that step, act the
// step's action, ap the previous one.
template <int OBJ>
__device__ __forceinline__ float step_loss(const float* x, const float r[3], const float act[4],
                                           const float ap[4], const RolloutArgs& a) {
  const float ex = x[0] - r[0], ey = x[1] - r[1], ez = x[2] - r[2];
  if (OBJ == SIM_OBJ_SQUARED)
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez)) +
           a.w_act * fmaf(act[0], act[0], fmaf(act[1], act[1], fmaf(act[2], act[2], act[3] * act[3])));
  const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
  const float s = sqrtf(fmaf(x[3], x[3], x[4] * x[4])), c = sqrtf(fmaf(x[5], x[5], x[6] * x[6]));
  float L = fmaf(a.w_theta, 2.f * atan2f(s, c), -expf(-2.f * d));
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float da = act[o] - ap[o];
    L = fmaf(a.w_a[o] * act[o], act[o], fmaf(a.w_da[o] * da, da, L));
  }
  return L;
}

// Adds sd * dL_step/dx (position and attitude terms) to lam; xn = post-step state.
template <int OBJ>
__device__ __forceinline__ void step_loss_state_adjoint(const float* xn, const float r[3], float sd,
                                                        const RolloutArgs& a, float* lam) {
  const float ex = xn[0] - r[0], ey = xn[1] - r[1], ez = xn[2] - r[2];
  if (OBJ == SIM_OBJ_SQUARED) {
    lam[0] = fmaf(2.f * sd, ex, lam[0]);
    lam[1] = fmaf(2.f * sd, ey, lam[1]);
    lam[2] = fmaf(2.f * sd, ez, lam[2]);
    return;
  }
  // d/dp of -exp(-2 |e|) = 2 exp(-2 |e|) e / |e|  (0 at e = 0)
  const float d = sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez)));
  if (d > 0.f) {
    const float g = 2.f * sd * expf(-2.f * d) / d;
    lam[0] = fmaf(g, ex, lam[0]);
    lam[1] = fmaf(g, ey, lam[1]);
    lam[2] = fmaf(g, ez, lam[2]);
  }
  // theta = 2 atan2(s, c): d theta = 2 (c ds - s dc) / (s^2 + c^2),
  // ds = (qx dqx + qy dqy) / s, dc = (qz dqz + qw dqw) / c  (0 at the kinks)
  const float s2 = fmaf(xn[3], xn[3], xn[4] * xn[4]), c2 = fmaf(xn[5], xn[5], xn[6] * xn[6]);
  const float s = sqrtf(s2), c = sqrtf(c2), n2 = s2 + c2;
  const float gw = 2.f * sd * a.w_theta / n2;
  if (s > 0.f) {
    const float g = gw * c / s;
    lam[3] = fmaf(g, xn[3], lam[3]);
    lam[4] = fmaf(g, xn[4], lam[4]);
  }
  if (c > 0.f) {
    const float g = -gw * s / c;
    lam[5] = fmaf(g, xn[5], lam[5]);
    lam[6] = fmaf(g, xn[6], lam[6]);
  }
}

// ------------------------------------------------------------------ kernels

template <int OBJ, bool LO>
__global__ void __launch_bounds__(TPB) rollout_fwd_kernel(RolloutArgs a, DevParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  load_weights(s, a.w);
  __syncthreads();
  const int lane = threadIdx.x & 31, v = threadIdx.x >> 5;
  const int r0 = 16 * v, row = r0 + (lane & 15);
  const int i = blockIdx.x * DPC + row;
  const bool valid = i < a.n;
  const int ii = valid ? i : a.n - 1;  // out-of-range rows shadow the last drone
  float x[17];
  load_row(a.x0, ii, x);
  float loss = 0.f;
  float ap[4] = {0.f, 0.f, 0.f, 0.f};  // previous action (a_{-1} = hover = 0)
  // reference positions at steps k, k + 1 and k + 2: each is loaded two steps
  // before its first use, so that a cold load's latency overlaps two steps' work
  float r[3], rn[3];
  ref_at(a.p_ref, 0, a.n, ii, r);
  ref_at(a.p_ref, 1, a.n, ii, rn);
  for (int k = 0; k < a.H; ++k) {
    float rnn[3] = {0.f, 0.f, 0.f};
    if (k + 2 <= a.H) ref_at_pinned(a.p_ref, k + 2, a.n, ii, rnn);
    if (a.store_ckpt && (k % a.C) == 0 && valid && lane < 16) {
      store_row(a.ckpt + (size_t)(k / a.C) * a.n * 20, i, x);
      if (OBJ == SIM_OBJ_TRACKING_REWARD)
        a.ckpt_a[(size_t)(k / a.C) * a.n + i] = make_float4(ap[0], ap[1], ap[2], ap[3]);
    }
    if (lane < 16) put_obs(s.obs, row, x, r);
    __syncwarp();
    float h1[8][4], h2[8][4];
    mlp_forward<LO>(s, r0, lane, h1, h2, s.act);
    __syncwarp();
    float act[4] = {s.act[row][0], s.act[row][1], s.act[row][2], s.act[row][3]};
    __syncwarp();
    for (int j = 0; j < a.R; ++j) policy_step(x, act, P, a.dt);
    loss += step_loss<OBJ>(x, rn, act, ap, a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r[c] = rn[c];
      rn[c] = rnn[c];
    }
#pragma unroll
    for (int o = 0; o < 4; ++o) ap[o] = act[o];
  }
  if (valid && lane < 16) a.loss_w[i] = loss;
}

// mbarrier helpers for the adjoint's warp hand-off (all threads of a role arrive).
// Waits are bounded: 2^18 polls of try_wait, which suspends the thread for up to a
// hardware time limit while the phase is incomplete -- measured on B300 at ~3.8 us,
// so a wait gives up after about a second (at least ~6 ms if it never suspends),
// far above the longest wait of the hand-off (~0.1 ms); the caller flags a timeout.
__device__ __forceinline__ void mbar_init(unsigned long long* m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* m) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(m)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* m, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < (1 << 18) && !done; ++it)
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(m)), "r"(parity)
        : "memory");
  return done != 0;
}

// Failure-detection self-test of the bounded waits: one warp arrives once on a
// barrier that expects two arrivals, so the phase never completes; every thread's
// wait (the same bounded wait as the adjoint's hand-off) gives up, and the kernel
// sets SIM_FLAG_TIMEOUT and returns.  Nothing faults, traps or hangs.
__global__ void wait_selftest_kernel(uint32_t* status) {
  __shared__ unsigned long long m;
  if (threadIdx.x == 0) mbar_init(&m, 2);
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive(&m);
  const bool done = mbar_wait(&m, 0);
  if (!done && threadIdx.x == 0) atomicOr(status, SIM_FLAG_TIMEOUT);
}

// The adjoint runs three warp roles per CTA, each role one warp per 16-drone block.
// Warps 8-11 (recompute) run one segment ahead of the reverse sweep: from the
// segment's checkpoint they step its states forward with the policy in the loop and
// write the states (segment rows, and the state after the segment), each step's
// record of forward quantities (StepRecord) and each step's h2 and actions (the
// activation cache) into the segment buffer of the segment's parity; launched for
// sim_rollout_grad (a.fused) they first run the forward pass itself.  Warps 0-3
// (compute) sweep a recomputed segment in reverse: per step the loss and step
// adjoints and the MLP backward, which leave the step's dz tiles in shared memory.  Warps 4-7 (weight gradient) accumulate dW over the CTA's 64 drones from
// those tiles while the compute warps already run the next (earlier) step, and then
// prepare step k - 2 for compute warp v's drones in the freed buffer: h2 and the
// actions come back from the cache, h1 is recomputed from the segment state (one
// layer).  Hand-offs, all on shared-memory barriers with bounded waits:
//   full[b] / empty[b]   per step parity b = k & 1: the compute threads arrive when
//                        the step's tiles are written, the weight-gradient threads when
//                        they have read them;
//   ready[v][b]          the 32 lanes of the warp that prepared buffer b for warp v's
//                        rows arrive;
//   seg_done[p]          the recompute threads arrive when the segment of parity p
//                        is written;
//   seg_free[p]          the weight-gradient threads arrive when the compute warps
//                        have finished the segment of parity p, so that the recompute
//                        may write the segment after next into its buffer.
template <int OBJ, bool LO>
__global__ void __launch_bounds__(3 * TPB, 1) rollout_bwd_kernel(RolloutArgs a, DevParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  load_weights(s, a.w);
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&s.full[b], TPB);
      mbar_init(&s.empty[b], TPB);
      for (int v = 0; v < 4; ++v) mbar_init(&s.ready[v][b], 32);
      mbar_init(&s.seg_done[b], TPB);
      mbar_init(&s.seg_free[b], TPB);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nseg = (a.H + a.C - 1) / a.C;
  bool timed_out = false;
  // protocol waits: after this thread's first timeout the rest are skipped (the
  // results are then void and flagged), so a broken hand-off costs one wait limit
  auto wait_on = [&](unsigned long long* m, uint32_t par) {
    if (!timed_out && !mbar_wait(m, par)) timed_out = true;
  };
  // segment buffers of parity p: rows [C R + 1][n][20], step records [C R][n][20],
  // previous actions [C][n] (tracking reward), activation cache [C][n / 16][CACHE_CHUNKS]
  const size_t seg_stride = (size_t)(a.C * a.R + 1) * a.n * 20;
  auto seg_rows = [&](int sg) { return a.seg + (size_t)(sg & 1) * seg_stride; };
  auto seg_prev = [&](int sg) { return a.seg_a + (size_t)(sg & 1) * a.C * a.n; };
  auto seg_recs = [&](int sg) { return a.seg_q + (size_t)(sg & 1) * a.C * a.R * a.n * FQ_FLOATS; };
  // cache entry of warp rows 16 v at step j of a segment of parity p
  auto cache_at = [&](int p, int v, int j) {
    return a.hcache + (((size_t)p * a.C + j) * gridDim.x * 4 + (size_t)blockIdx.x * 4 + v) * CACHE_CHUNKS;
  };
  // barrier phase of segment sg's use of its parity's barriers: segments are taken
  // in reverse, so the u-th one (u = nseg - 1 - sg) is its parity's (u >> 1)-th
  auto seg_phase = [&](int sg) { return (uint32_t)(((nseg - 1 - sg) >> 1) & 1); };
  // drones of warp v (any role): rows 16 v + (lane & 15) of the CTA's 64;
  // out-of-range rows shadow the last drone (finite data; their seed and dz are zero)
  const int v = warp & 3;
  const int r0 = 16 * v, row = r0 + (lane & 15);
  const int i = blockIdx.x * DPC + row;
  const bool valid = i < a.n;
  const int ii = valid ? i : a.n - 1;
  if (warp >= 8) {
    // ---------------- recompute warps
    // Jobs in order: with a.fused, first the forward pass over all segments
    // (checkpoints, per-drone loss; its last segment is recorded for the reverse
    // sweep as a recompute would record it), then the recomputes of the segments
    // before it from their checkpoints, last first.  One loop body serves both.
    const int nrec = a.fused ? nseg - 1 : nseg;  // segments recomputed from checkpoints
    const int njobs = a.fused ? nseg + nrec : nrec;
    float x[17];
    float4 ap4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float loss = 0.f;
    for (int job = 0; job < njobs; ++job) {
      const bool fwd = a.fused && job < nseg;
      const int sg = fwd ? job : nrec - 1 - (a.fused ? job - nseg : job);
      const bool record = !fwd || sg == nseg - 1;
      const int k0 = sg * a.C, k1 = min(a.H, k0 + a.C);
      // the buffer's previous segment (sg + 2) has been swept
      if (record && sg + 2 < nseg) wait_on(&s.seg_free[sg & 1], seg_phase(sg + 2));
      float* rows = seg_rows(sg);
      if (!fwd) {
        load_row(a.ckpt + (size_t)sg * a.n * 20, ii, x);
        if (OBJ == SIM_OBJ_TRACKING_REWARD) ap4 = a.ckpt_a[(size_t)sg * a.n + ii];
      } else if (sg == 0) {
        load_row(a.x0, ii, x);
      }
      // reference positions of steps k, k + 1 and k + 2 in registers, each loaded
      // two steps before its use
      float rr[3], rr1[3];
      ref_at(a.p_ref, k0, a.n, ii, rr);
      ref_at(a.p_ref, k0 + 1, a.n, ii, rr1);
      for (int k = k0; k < k1; ++k) {
        if (valid && lane < 16) {
          if (fwd && k == k0) {
            store_row(a.ckpt + (size_t)sg * a.n * 20, i, x);
            if (OBJ == SIM_OBJ_TRACKING_REWARD) a.ckpt_a[(size_t)sg * a.n + i] = ap4;
          }
          if (record) {
            store_row(rows + (size_t)(k - k0) * a.R * a.n * 20, i, x);
            if (OBJ == SIM_OBJ_TRACKING_REWARD) seg_prev(sg)[(size_t)(k - k0) * a.n + i] = ap4;
          }
        }
        float rr2[3] = {0.f, 0.f, 0.f};
        if (k + 2 <= a.H) ref_at_pinned(a.p_ref, k + 2, a.n, ii, rr2);
        put_obs_half(s.obs, row, x, rr, lane >> 4);
        __syncwarp();
        float act[4];
        {
          float h1[8][4], h2[8][4];
          mlp_forward<LO>(s, r0, lane, h1, h2, s.act);
          if (record) cache_put(s, v, r0, lane, h2, cache_at(sg & 1, v, k - k0));  // has warp barriers
          else __syncwarp();
#pragma unroll
          for (int o = 0; o < 4; ++o) act[o] = s.act[row][o];
        }
        __syncwarp();  // the observation and action rows are rewritten next step
        for (int j = 0; j < a.R; ++j) {
          if (record && j > 0 && valid && lane < 16)
            store_row(rows + ((size_t)(k - k0) * a.R + j) * a.n * 20, i, x);
          StepRecord q;
          policy_step_rec(x, act, P, a.dt, q);
          if (record && valid && lane < 16)
            store_record(seg_recs(sg) + ((size_t)(k - k0) * a.R + j) * a.n * FQ_FLOATS, i, q);
        }
        if (fwd) {
          const float ap[4] = {ap4.x, ap4.y, ap4.z, ap4.w};
          loss += step_loss<OBJ>(x, rr1, act, ap, a);
        }
        ap4 = make_float4(act[0], act[1], act[2], act[3]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          rr[c] = rr1[c];
          rr1[c] = rr2[c];
        }
      }
      if (fwd && sg == nseg - 1 && valid && lane < 16) a.loss_w[i] = loss;
      if (record) {
        // the state after the segment (the loss term of its last step)
        if (valid && lane < 16) store_row(rows + (size_t)(k1 - k0) * a.R * a.n * 20, i, x);
        // the segment's cache entries are complete before its readers copy them
        // back (they wait for these arrivals first)
        if (lane == 0) {
          bulk_wait_all();
          fence_proxy_async_global();
        }
        mbar_arrive(&s.seg_done[sg & 1]);  // release: this thread's rows
      }
    }
    if (timed_out && a.status) atomicOr(a.status, SIM_FLAG_TIMEOUT);
    return;
  }
  if (warp >= 4) {
    // ---------------- weight-gradient warps: slice v of dW2 / dW1 / dW3
    DwAcc acc;
#pragma unroll
    for (int n = 0; n < 8; ++n) acc.w2[n][0] = acc.w2[n][1] = acc.w2[n][2] = acc.w2[n][3] = 0.f;
#pragma unroll
    for (int n = 0; n < 2; ++n) acc.w1[n][0] = acc.w1[n][1] = acc.w1[n][2] = acc.w1[n][3] = 0.f;
    acc.w3[0] = acc.w3[1] = acc.w3[2] = acc.w3[3] = 0.f;
    // Reverse steps k = H - 1 - t in processing order t.  The step of processing
    // order t + 2 is prepared in two parts: its state and reference are loaded
    // before the dW work of step t (their latency overlaps it); once all four warps
    // of this role have read buffer b = k & 1, its cache entry is copied into the
    // buffer for compute warp v's rows and h1 is recomputed there from the state.
    int seen = nseg;  // lowest segment whose recompute this warp has waited for
    int last[2] = {-1, -1};  // processing order of the last copy issued into buffer 0, 1
    float px[17], pr[3];
    // step k of segment sg (first step k0) is prepared as processing step tp
    auto prep_load = [&](int k, int sg, int k0) {
      if (sg < seen) {
        wait_on(&s.seg_done[sg & 1], seg_phase(sg));
        seen = sg;
      }
      if (valid) load_row(seg_rows(sg) + (size_t)(k - k0) * a.R * a.n * 20, i, px);
      else load_row(a.ckpt + (size_t)sg * a.n * 20, ii, px);
      ref_at(a.p_ref, k, a.n, ii, pr);
    };
    auto prep_store = [&](int k, int sg, int k0, int tp) {
      const int b = k & 1;
      if (lane == 0) {
        fence_proxy_async_global();
        cache_load(s, b, r0, cache_at(sg & 1, v, k - k0), &s.ready[v][b]);
      }
      last[b] = tp;
      put_obs_half(s.obsr[b], row, px, pr, lane >> 4);  // the step's observation rows (dW1 operand)
      __syncwarp();
      float h1[8][4];
      mlp_layer1<LO>(s, s.obsr[b], r0, lane, h1);
      store_c64(s.h1[b], r0, lane, h1);
      mbar_arrive(&s.ready[v][b]);  // with the copied bytes, completes the phase
    };
    // segments (and their first steps) of the step accumulated (k) and of the one
    // prepared (k - 2), followed as k decreases by one per iteration
    int sg = (a.H - 1) / a.C, k0 = sg * a.C;
    int sgp = sg, k0p = k0;
    // t = -2, -1 only prepare the first two steps (one copy of the code for all)
    for (int t = -2; t < a.H; ++t) {
      const int k = a.H - 1 - t, b = k & 1, kp = k - 2;
      const uint32_t par = (uint32_t)((t >> 1) & 1);
      const bool work = t >= 0, ahead = t + 2 < a.H;
      if (ahead && kp < k0p) {
        --sgp;
        k0p -= a.C;
      }
      if (work) {
        wait_on(&s.full[b], par);
        // the compute warp has consumed step k's cache entry: drop its L2 lines
        // without a write-back; the fence orders the discards before the bulk
        // stores that reuse the entry two segments later (issued after seg_free)
        cache_discard(cache_at(sg & 1, v, k - k0), lane);
        fence_proxy_async_global();
        // the compute warps are done with the segment once they finish its first
        // step; so is this warp (its loads of the segment were two steps earlier)
        if (k == k0) mbar_arrive(&s.seg_free[sg & 1]);
      }
      if (ahead) prep_load(kp, sgp, k0p);
      if (work) {
        accumulate_dw<LO>(s, v, lane, acc, b);
        mbar_arrive(&s.empty[b]);
      }
      if (ahead) {
        if (work) wait_on(&s.empty[b], par);
        prep_store(kp, sgp, k0p, t + 2);
      }
      if (work && k == k0) {
        --sg;
        k0 -= a.C;
      }
    }
    // the compute warp consumes every copy issued here; wait (bounded) for the last
    // one into each buffer, so that no copy is in flight when the CTA exits
    for (int b = 0; b < 2; ++b)
      if (last[b] >= 0 && !mbar_wait(&s.ready[v][b], (uint32_t)((last[b] >> 1) & 1))) timed_out = true;
    store_dw(acc, v, lane, a.part + (size_t)blockIdx.x * NPOL_PAD);
    if (timed_out && a.status) atomicOr(a.status, SIM_FLAG_TIMEOUT);
    return;
  }
  // ---------------- compute warps
  const float seed = valid ? (*a.dL) * a.inv_n : 0.f;  // padded rows contribute nothing
  float lam[17];
#pragma unroll
  for (int j = 0; j < 17; ++j) lam[j] = 0.f;
  // smoothness adjoint carried from step k + 1 to a_k: -2 sd w_dact (a_{k+1} - a_k)
  float carry[4] = {0.f, 0.f, 0.f, 0.f};
  // running sums of dz2 (this lane's two drones, its 16 columns of the fragment) and
  // of dz3 (lanes 0-15: their drone), over all steps: db2 and db3 of the warp's drones
  float sb2[8][2], sb3[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int n = 0; n < 8; ++n) sb2[n][0] = sb2[n][1] = 0.f;
  int t = 0;  // reverse steps processed so far (the weight-gradient warps count alike)
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * a.C, k1 = min(a.H, k0 + a.C);
    wait_on(&s.seg_done[sg & 1], seg_phase(sg));
    const float* rows = seg_rows(sg);
    // the state after the segment and the reference at that step (the loss term of
    // the segment's last step); padded rows read the checkpoint instead (finite
    // data; their seed is zero).  Everything read here was published with the
    // segment (seg_done), checkpoints included
    float xn[17], rn[3];
    if (valid) load_row(rows + (size_t)(k1 - k0) * a.R * a.n * 20, i, xn);
    else load_row(a.ckpt + (size_t)sg * a.n * 20, ii, xn);
    ref_at(a.p_ref, k1, a.n, ii, rn);
    // step k's state row, step record and previous action, prefetched during step
    // k + 1 (padded rows take the last drone's record: finite, published with the
    // segment like every row)
    auto prefetch_step = [&](int k) {
      float* bx = s.pre_x[k & 1][row];
      if (valid) prefetch_row(bx, rows + (size_t)(k - k0) * a.R * a.n * 20, i);
      else prefetch_row(bx, a.ckpt + (size_t)sg * a.n * 20, ii);
      prefetch_row(s.pre_q[k & 1][row], seg_recs(sg) + (size_t)(k - k0) * a.R * a.n * FQ_FLOATS, ii);
      if (OBJ == SIM_OBJ_TRACKING_REWARD)
        cp_async16(&s.pre_a[k & 1][row], valid ? &seg_prev(sg)[(size_t)(k - k0) * a.n + i]
                                               : &a.ckpt_a[(size_t)sg * a.n + ii]);
    };
    if (lane < 16) prefetch_step(k1 - 1);
    cp_async_commit();
    // the reference at step k, loaded during step k + 1
    float rnext[3];
    ref_at(a.p_ref, k1 - 1, a.n, ii, rnext);
    for (int k = k1 - 1; k >= k0; --k, ++t) {
      const int b = k & 1;
      cp_async_wait_all();  // this step's state row, step record and previous action
      // this step's tiles and actions, prepared by the weight-gradient warp after
      // all four of them had read the buffer's previous contents
      wait_on(&s.ready[v][b], (uint32_t)((t >> 1) & 1));
      __syncwarp();
      float x[17];
#pragma unroll
      for (int j = 0; j < 17; ++j) x[j] = s.pre_x[b][row][j];
      const float r[3] = {rnext[0], rnext[1], rnext[2]};
      if (k > k0) ref_at(a.p_ref, k - 1, a.n, ii, rnext);
      float ap[4] = {0.f, 0.f, 0.f, 0.f};
      if (OBJ == SIM_OBJ_TRACKING_REWARD) {
        const float4 q = s.pre_a[b][row];
        ap[0] = q.x;
        ap[1] = q.y;
        ap[2] = q.z;
        ap[3] = q.w;
      }
      if (k > k0 && lane < 16) prefetch_step(k - 1);
      cp_async_commit();
      // this step's observation rows (the dW1 operand) are in obsr[b] already, written
      // with its activations by the weight-gradient warp that prepared the step
      const float act[4] = {s.actb[b][row][0], s.actb[b][row][1], s.actb[b][row][2], s.actb[b][row][3]};
      // loss term at policy step k + 1 (state after the last sub-step)
      step_loss_state_adjoint<OBJ>(xn, rn, seed, a, lam);
      // back through the R sub-steps (states before and after each, and its record);
      // the held action collects every sub-step's adjoint
      float ga[4] = {0.f, 0.f, 0.f, 0.f};
      float xq[17];
#pragma unroll
      for (int q = 0; q < 17; ++q) xq[q] = xn[q];
      for (int j = a.R - 1; j >= 0; --j) {
        float xs[17], fq[FQ_FLOATS];
        if (j > 0) {
          if (valid) load_row(rows + ((size_t)(k - k0) * a.R + j) * a.n * 20, i, xs);
          else load_row(a.ckpt + (size_t)sg * a.n * 20, ii, xs);
          const float4* f4 = reinterpret_cast<const float4*>(
              seg_recs(sg) + (((size_t)(k - k0) * a.R + j) * a.n + ii) * FQ_FLOATS);
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            const float4 u = f4[c];
            fq[4 * c] = u.x;
            fq[4 * c + 1] = u.y;
            fq[4 * c + 2] = u.z;
            fq[4 * c + 3] = u.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 17; ++q) xs[q] = x[q];
#pragma unroll
          for (int c = 0; c < FQ_FLOATS; ++c) fq[c] = s.pre_q[b][row][c];
        }
        StepRecord rec;
        record_from(fq, rec);
        float gj[4];
        policy_step_adjoint(xs, xq, rec, act, lam, gj, P, a.dt);
#pragma unroll
        for (int o = 0; o < 4; ++o) ga[o] += gj[o];
#pragma unroll
        for (int q = 0; q < 17; ++q) xq[q] = xs[q];
      }
      if (OBJ == SIM_OBJ_SQUARED) {
#pragma unroll
        for (int o = 0; o < 4; ++o) ga[o] = fmaf(2.f * seed * a.w_act, act[o], ga[o]);
      } else {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          const float sm = 2.f * seed * a.w_da[o] * (act[o] - ap[o]);
          ga[o] = fmaf(2.f * seed * a.w_a[o], act[o], ga[o]) + sm + carry[o];
          carry[o] = -sm;
        }
      }
      // dz3 = ga (1 - a^2); rows of padded drones are zero.  Columns 4-15 of the
      // tiles stay zero from the launch's set-up
      if (lane < 16) {
        float dz[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          dz[o] = valid ? ga[o] * fmaf(-act[o], act[o], 1.f) : 0.f;
          sb3[o] += dz[o];
        }
#pragma unroll
        for (int o = 0; o < 4; o += 2) {
          uint32_t h, l;
          split2(dz[o], dz[o + 1], h, l);
          *reinterpret_cast<uint32_t*>(&s.dz3[b][0][row * S16 + o]) = h;
          *reinterpret_cast<uint32_t*>(&s.dz3[b][1][row * S16 + o]) = l;
        }
      }
      __syncwarp();
      mlp_backward<LO>(s, r0, lane, b, sb2);
      __syncwarp();
      mbar_arrive(&s.full[b]);  // this warp's tiles of step k are written
      // observation adjoint: obs = [p - r, q, v, w]
#pragma unroll
      for (int j = 0; j < 13; ++j) lam[j] += s.dobs[row][j];
#pragma unroll
      for (int j = 0; j < 17; ++j) xn[j] = x[j];
#pragma unroll
      for (int c = 0; c < 3; ++c) rn[c] = r[c];
    }
  }
  // db2, db3 of the CTA: the warp's sums over its lanes (shuffles, fixed order), then
  // over the four compute warps in a fixed order through this warp's rows of dobs
  // (no longer used by the sweep), written by warp 0 into the CTA's partials
  {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int m = 4; m < 32; m <<= 1) sb2[n][c] += __shfl_xor_sync(FULL, sb2[n][c], m);
#pragma unroll
    for (int o = 0; o < 4; ++o)
#pragma unroll
      for (int m = 1; m < 32; m <<= 1) sb3[o] += __shfl_xor_sync(FULL, sb3[o], m);
    float* red = &s.dobs[r0][0];  // 256 floats of this warp
    __syncwarp();
    if (lane < 4) {
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        red[8 * n + 2 * lane] = sb2[n][0];
        red[8 * n + 2 * lane + 1] = sb2[n][1];
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int o = 0; o < 4; ++o) red[64 + o] = sb3[o];
    }
    asm volatile("bar.sync 1, 128;\n" ::: "memory");  // the four compute warps
    if (v == 0) {
      float* part = a.part + (size_t)blockIdx.x * NPOL_PAD;
      for (int u = lane; u < 68; u += 32) {
        const float tot = ((s.dobs[0][u] + s.dobs[16][u]) + s.dobs[32][u]) + s.dobs[48][u];
        if (u < 64) part[OFF_B2 + u] = tot;
        else part[OFF_B3 + u - 64] = tot;
      }
    }
  }
  if (valid && lane < 16) {
    float4* p = reinterpret_cast<float4*>(a.dx0 + (size_t)i * 20);
#pragma unroll
    for (int j = 0; j < 4; ++j) p[j] = make_float4(lam[4 * j], lam[4 * j + 1], lam[4 * j + 2], lam[4 * j + 3]);
    p[4] = make_float4(lam[16], 0.f, 0.f, 0.f);
  }
  if (timed_out && a.status) atomicOr(a.status, SIM_FLAG_TIMEOUT);
}

// Deterministic reductions: dW[p] = sum over CTAs (fixed order, fp64);
// loss = sum over drones / n (one block, fixed-order tree).
__global__ void reduce_dw_kernel(const float* __restrict__ part, int n_cta, float* __restrict__ dW) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPOL) return;
  double acc = 0.0;
  for (int c = 0; c < n_cta; ++c) acc += (double)part[(size_t)c * NPOL_PAD + p];
  dW[p] = (float)acc;
}

__global__ void reduce_loss_kernel(const float* __restrict__ loss_w, int n, float* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) acc += (double)loss_w[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (float)(red[0] / n);
}

// Adam (Kingma & Ba, ICLR 2015) on the fp32 master weights, one block: the
// step count is read once by every thread (t = step + 1) and written back by
// thread 0 at the end, so a captured graph replays successive steps.
__global__ void __launch_bounds__(1024) adam_kernel(const float* __restrict__ g, float* __restrict__ w,
                                                    float* __restrict__ m, float* __restrict__ v,
                                                    __nv_bfloat16* __restrict__ wb, int n, int* step,
                                                    float lr, float b1, float b2, float eps) {
  __shared__ int t_s;
  if (threadIdx.x == 0) t_s = *step + 1;
  __syncthreads();
  const int t = t_s;
  const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
  if (threadIdx.x == 0) *step = t;
}

}  // namespace ro

cudaError_t launch_adam(const float* g, float* w, float* m, float* v, uint16_t* wb, int n, int* step,
                        float lr, float b1, float b2, float eps, cudaStream_t st) {
  ro::adam_kernel<<<1, 1024, 0, st>>>(g, w, m, v, reinterpret_cast<__nv_bfloat16*>(wb), n, step, lr,
                                      b1, b2, eps);
  return cudaGetLastError();
}

size_t rollout_workspace_bytes(int n, int H, int C, int objective, int R) {
  const int n_ck = (H + C - 1) / C;
  const int n_cta = (n + ro::DPC - 1) / ro::DPC;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t b = al((size_t)n_ck * n * 20 * 4) + al((size_t)2 * (C * R + 1) * n * 20 * 4) +
             al((size_t)2 * C * R * n * ro::FQ_FLOATS * 4) + al((size_t)n * 4) +
             al((size_t)n_cta * ro::NPOL_PAD * 4) + al((size_t)2 * C * n_cta * 4 * ro::CACHE_BYTES);
  if (objective == SIM_OBJ_TRACKING_REWARD) b += al((size_t)n_ck * n * 16) + al((size_t)2 * C * n * 16);
  return b;
}

static void carve(void* ws, int n, int H, int C, int R, const RolloutObjective& obj,
                  ro::RolloutArgs& a) {
  const int n_ck = (H + C - 1) / C;
  const int n_cta = (n + ro::DPC - 1) / ro::DPC;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  char* p = (char*)ws;
  a.ckpt = (float*)p;
  p += al((size_t)n_ck * n * 20 * 4);
  a.seg = (float*)p;
  p += al((size_t)2 * (C * R + 1) * n * 20 * 4);
  a.seg_q = (float*)p;
  p += al((size_t)2 * C * R * n * ro::FQ_FLOATS * 4);
  a.loss_w = (float*)p;
  p += al((size_t)n * 4);
  a.part = (float*)p;
  p += al((size_t)n_cta * ro::NPOL_PAD * 4);
  a.hcache = (uint4*)p;
  p += al((size_t)2 * C * n_cta * 4 * ro::CACHE_BYTES);
  if (obj.kind == SIM_OBJ_TRACKING_REWARD) {
    a.ckpt_a = (float4*)p;
    p += al((size_t)n_ck * n * 16);
    a.seg_a = (float4*)p;
  }
  a.R = R;
  a.w_theta = obj.w_theta;
  for (int o = 0; o < 4; ++o) {
    a.w_a[o] = obj.w_act[o];
    a.w_da[o] = obj.w_dact[o];
  }
}

template <typename K>
static cudaError_t launch_rollout_kernel(K kernel, int grid, const ro::RolloutArgs& a,
                                         const DevParams& P, cudaStream_t st, int threads = ro::TPB) {
  const int smem = (int)sizeof(ro::Smem);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  kernel<<<grid, threads, smem, st>>>(a, P);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint32_t* status, cudaStream_t st) {
  ro::wait_selftest_kernel<<<1, 32, 0, st>>>(status);
  return cudaGetLastError();
}

cudaError_t launch_rollout_fwd(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                               int C, int R, float dt, float w_act, const RolloutObjective& obj,
                               const DevParams& P, void* ws, float* loss, bool store_ckpt,
                               cudaStream_t st) {
  ro::RolloutArgs a{};
  carve(ws, n, H, C, R, obj, a);
  a.x0 = x0;
  a.w = w;
  a.p_ref = p_ref;
  a.n = n;
  a.H = H;
  a.C = C;
  a.dt = dt;
  a.w_act = w_act;
  a.store_ckpt = store_ckpt ? 1 : 0;
  const int grid = (n + ro::DPC - 1) / ro::DPC;
  cudaError_t e = obj.kind == SIM_OBJ_TRACKING_REWARD
                      ? (obj.hilo ? launch_rollout_kernel(ro::rollout_fwd_kernel<SIM_OBJ_TRACKING_REWARD, true>, grid, a, P, st)
                                  : launch_rollout_kernel(ro::rollout_fwd_kernel<SIM_OBJ_TRACKING_REWARD, false>, grid, a, P, st))
                      : (obj.hilo ? launch_rollout_kernel(ro::rollout_fwd_kernel<SIM_OBJ_SQUARED, true>, grid, a, P, st)
                                  : launch_rollout_kernel(ro::rollout_fwd_kernel<SIM_OBJ_SQUARED, false>, grid, a, P, st));
  if (e != cudaSuccess) return e;
  ro::reduce_loss_kernel<<<1, 256, 0, st>>>(a.loss_w, n, loss);
  return cudaGetLastError();
}

// The adjoint launch; with loss != null it runs the forward pass first (fused) and
// reduces the loss after it.
static cudaError_t rollout_adjoint(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                                   int C, int R, float dt, float w_act, const RolloutObjective& obj,
                                   const DevParams& P, void* ws, const float* dL, float* dW, float* dx0,
                                   uint32_t* status, float* loss, cudaStream_t st) {
  ro::RolloutArgs a{};
  carve(ws, n, H, C, R, obj, a);
  a.status = status;
  a.x0 = x0;
  a.w = w;
  a.p_ref = p_ref;
  a.dx0 = dx0;
  a.n = n;
  a.H = H;
  a.C = C;
  a.dt = dt;
  a.w_act = w_act;
  a.dL = dL;
  a.inv_n = 1.f / (float)n;
  a.fused = loss != nullptr;
  const int grid = (n + ro::DPC - 1) / ro::DPC;
  cudaError_t e = obj.kind == SIM_OBJ_TRACKING_REWARD
                      ? (obj.hilo ? launch_rollout_kernel(ro::rollout_bwd_kernel<SIM_OBJ_TRACKING_REWARD, true>, grid, a, P, st, 3 * ro::TPB)
                                  : launch_rollout_kernel(ro::rollout_bwd_kernel<SIM_OBJ_TRACKING_REWARD, false>, grid, a, P, st, 3 * ro::TPB))
                      : (obj.hilo ? launch_rollout_kernel(ro::rollout_bwd_kernel<SIM_OBJ_SQUARED, true>, grid, a, P, st, 3 * ro::TPB)
                                  : launch_rollout_kernel(ro::rollout_bwd_kernel<SIM_OBJ_SQUARED, false>, grid, a, P, st, 3 * ro::TPB));
  if (e != cudaSuccess) return e;
  if (loss) ro::reduce_loss_kernel<<<1, 256, 0, st>>>(a.loss_w, n, loss);
  ro::reduce_dw_kernel<<<(ro::NPOL + 255) / 256, 256, 0, st>>>(a.part, grid, dW);
  return cudaGetLastError();
}

cudaError_t launch_rollout_bwd(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                               int C, int R, float dt, float w_act, const RolloutObjective& obj,
                               const DevParams& P, void* ws, const float* dL, float* dW, float* dx0,
                               uint32_t* status, cudaStream_t st) {
  return rollout_adjoint(x0, w, p_ref, n, H, C, R, dt, w_act, obj, P, ws, dL, dW, dx0, status, nullptr, st);
}

cudaError_t launch_rollout_grad(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                                int C, int R, float dt, float w_act, const RolloutObjective& obj,
                                const DevParams& P, void* ws, float* loss, const float* dL, float* dW,
                                float* dx0, uint32_t* status, cudaStream_t st) {
  return rollout_adjoint(x0, w, p_ref, n, H, C, R, dt, w_act, obj, P, ws, dL, dW, dx0, status, loss, st);
}

}  // namespace cf
