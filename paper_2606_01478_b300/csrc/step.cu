// Fused K-step forward kernel: one drone per thread, the 20-float state held in
// registers for all K steps, one coalesced float4-plane read and write per
// launch (the paper's fused step pipeline scanned over steps, Architecture
// section).
#include <utility>

#include <cstdlib>

#include "internal.h"
#include "stepcore.cuh"

namespace cf {

// Programmatic dependent launch of the K-chained step kernels.  A step kernel is
// launched with programmatic stream serialization, so its CTAs may be scheduled
// while the previous kernel of the stream drains; chain_wait (griddepcontrol.wait)
// holds every thread until that kernel has completed and its writes are visible,
// so it precedes every global access of the kernel.  chain_release
// (griddepcontrol.launch_dependents) lets the next kernel be scheduled once every
// CTA of this one has released or exited.  The uniform kernel releases after each
// thread's work, so that the next grid is placed while this one drains, on SMs
// that are emptying: released at the start, a grid of small CTAs was placed beside
// CTAs that still ran, stacked two warps on some sub-partitions and left others
// idle (up to 2x slower launches, varying from run to run).  The persistent
// batched kernels fill every SM at their occupancy, so the next grid can only be
// placed where CTAs exit; they release at the start.  Without the launch attribute
// (or behind a copy or an ordinary kernel) both return at once.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void chain_release() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// CRAZYFLOW_SERIAL_LAUNCH=1 in the environment (read once per process) drops the
// attribute: the same kernels run as plain stream-ordered launches, for
// profilers that do not follow programmatically dependent launches.
static bool serial_launches() {
  static const bool serial = [] {
    const char* e = getenv("CRAZYFLOW_SERIAL_LAUNCH");
    return e && e[0] == '1';
  }();
  return serial;
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_chained(void (*kernel)(KArgs...), int grid, int tpb, cudaStream_t st,
                                  Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = serial_launches() ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// SINGLE: the launch is known to take one step (a.K == 1).  SYM: Jx = Jy in every
// parameter set (first-principles lag-rotor steps drop the zero gyroscopic term).
template <int MODEL, int INTEG, int CTRL, int MOTOR, bool SINGLE = false, bool SYM = false>
__device__ __forceinline__ void run_drone(const StepArgs& a, int i, const DevParams& P) {
  constexpr int NPL = (MODEL == SIM_FIRST_PRINCIPLES) ? 5 : 4;
  const int n = a.n;
  float s[20];
#pragma unroll
  for (int j = 0; j < NPL; ++j) {
    const float4 v = a.planes[(size_t)j * n + i];
    s[4 * j + 0] = v.x;
    s[4 * j + 1] = v.y;
    s[4 * j + 2] = v.z;
    s[4 * j + 3] = v.w;
  }
  const bool drag = (P.flags & PF_DRAG) != 0;
  const int last = a.n_blocks - 1;
  int blk = min(a.t0 / a.hold, last);
  // steps left in the current command block (the last block lasts forever)
  int left = (a.t0 / a.hold >= last) ? 0x7fffffff : a.hold - a.t0 % a.hold;
  CtrlHold h;
  decode_command<MODEL, CTRL>(a.cmd[(size_t)blk * n + i], P, h);
  if (SINGLE || a.K == 1) {
    // a single step never reaches the next command block: no look-ahead load
    one_step<MODEL, INTEG, CTRL, MOTOR, SYM>(s, h, P, drag, a.dt);
  } else {
    // the next block's command, prefetched when this launch reaches it
    float4 next = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.K > left) next = a.cmd[(size_t)min(blk + 1, last) * n + i];
    // outer loop over command-block segments, inner loop over the steps of one
    // segment (no per-step block bookkeeping in the hot loop)
    for (int k = 0; k < a.K;) {
      if (left == 0) {
        ++blk;
        decode_command<MODEL, CTRL>(next, P, h);
        left = (blk >= last) ? 0x7fffffff : a.hold;
        if (a.K - k > left) next = a.cmd[(size_t)min(blk + 1, last) * n + i];
      }
      const int seg = min(left, a.K - k);
      if constexpr (INTEG == SIM_EULER) {
        // the short Euler step unrolled by two (measured faster than the compiler's
        // own choice); RK4 keeps the compiler's (two measured slower there)
#pragma unroll 2
        for (int j = 0; j < seg; ++j) one_step<MODEL, INTEG, CTRL, MOTOR, SYM>(s, h, P, drag, a.dt);
      } else {
        for (int j = 0; j < seg; ++j) one_step<MODEL, INTEG, CTRL, MOTOR, SYM>(s, h, P, drag, a.dt);
      }
      k += seg;
      left -= seg;
    }
  }
  float chk = 0.f;
#pragma unroll
  for (int j = 0; j < 4 * NPL; ++j) chk += s[j];
  if (!isfinite(chk)) atomicOr(a.status, SIM_FLAG_NONFINITE);
#pragma unroll
  for (int j = 0; j < NPL; ++j)
    a.planes[(size_t)j * n + i] = make_float4(s[4 * j], s[4 * j + 1], s[4 * j + 2], s[4 * j + 3]);
}

template <int MODEL, int INTEG, int CTRL, int MOTOR, bool PERSET, bool SYM = false>
__global__ void __launch_bounds__(256) step_kernel(StepArgs a, DevParams P0) {
  chain_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n) {
    if constexpr (PERSET) {
      const DevParams P = a.params[a.set_of_world[i / a.N]];
      run_drone<MODEL, INTEG, CTRL, MOTOR, false, SYM>(a, i, P);
    } else {
      run_drone<MODEL, INTEG, CTRL, MOTOR, false, SYM>(a, i, P0);
    }
  }
  chain_release();
}

// Uneven / mixed batches: warp w of the persistent grid takes tiles w, w + W,
// w + 2W, ... (W = warps in the grid).  A tile is up to 32 consecutive drones of
// one world (x = first drone, y = count, z = world, w = model), so the branch
// on the model is uniform across the warp and parameters are a broadcast load.
template <int INTEG, int CTRL, int MOTOR, bool SINGLE, bool SYM>
__device__ __forceinline__ void run_tile(const StepArgs& a, const int4& d, int lane) {
  if (lane < d.y) {
    const DevParams P = a.params[a.set_of_world[d.z]];
    if (d.w == SIM_FIRST_PRINCIPLES) {
      run_drone<SIM_FIRST_PRINCIPLES, INTEG, CTRL, MOTOR, SINGLE, SYM>(a, d.x + lane, P);
    } else if (d.w == SIM_ABSTRACTED) {
      run_drone<SIM_ABSTRACTED, INTEG, SIM_CTRL_ATTITUDE, MOTOR, SINGLE>(a, d.x + lane, P);
    } else {
      run_drone<SIM_ABSTRACTED_NOTHRUST, INTEG, SIM_CTRL_ATTITUDE, MOTOR, SINGLE>(a, d.x + lane, P);
    }
  }
}

// Tiles of 32 drones, one per warp at a time.  Single-step launches take them in a
// fixed stride (a launch is ~0.1 ms; a shared counter would serialise 10^5 atomics).
// Fused launches take the next tile from a device counter, the next index
// requested before the current tile's steps and read after them: tiles of the two models differ about
// threefold in cost, so a fixed stride leaves the warps that drew more
// first-principles tiles running alone at the end.  Which warp steps a tile does
// not change its result.  The grid's last warp resets the counters for the next
// launch (a chained launch waits for this grid's completion before its first access).
template <int INTEG, int CTRL, int MOTOR, bool SINGLE, bool SYM>
__device__ __forceinline__ void run_tiles(const StepArgs& a, const int4* __restrict__ tiles, int n_tiles) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if constexpr (SINGLE) {
    for (int t = warp; t < n_tiles; t += nwarps) run_tile<INTEG, CTRL, MOTOR, SINGLE, SYM>(a, tiles[t], lane);
  } else {
    const unsigned FULL = 0xffffffffu;
    unsigned raw = lane == 0 ? atomicAdd(&a.tile_ctr[0], 1u) : 0u;
    int cur = (int)__shfl_sync(FULL, raw, 0);
    while (cur < n_tiles) {
      // lane 0 asks for the next tile; its index is read after this tile's steps
      raw = lane == 0 ? atomicAdd(&a.tile_ctr[0], 1u) : 0u;
      run_tile<INTEG, CTRL, MOTOR, SINGLE, SYM>(a, tiles[cur], lane);
      cur = (int)__shfl_sync(FULL, raw, 0);
    }
    if (lane == 0 && atomicAdd(&a.tile_ctr[1], 1u) == (unsigned)nwarps - 1u) {
      a.tile_ctr[0] = 0u;
      a.tile_ctr[1] = 0u;
    }
  }
}

template <int INTEG, int CTRL, int MOTOR, bool SYM>
__global__ void __launch_bounds__(256) step_batched_kernel(StepArgs a, const int4* __restrict__ tiles,
                                                           int n_tiles) {
  chain_wait();
  chain_release();
  run_tiles<INTEG, CTRL, MOTOR, false, SYM>(a, tiles, n_tiles);
}

// One step per launch (HBM bound): compiled for four 256-thread CTAs per SM with
// lag rotors under Euler (three with the general rotor model, two under RK4, whose
// registers would spill beyond that) so that more state loads are in flight.
template <int INTEG, int CTRL, int MOTOR, bool SYM>
__global__ void __launch_bounds__(256, INTEG == SIM_EULER ? (MOTOR == MOTOR_LAG ? 4 : 3) : 2)
    step_batched_single_kernel(StepArgs a, const int4* __restrict__ tiles, int n_tiles) {
  chain_wait();
  chain_release();
  run_tiles<INTEG, CTRL, MOTOR, true, SYM>(a, tiles, n_tiles);
}

template <int INTEG, int CTRL, int MOTOR, bool SINGLE, bool SYM = false>
static cudaError_t launch_b(const StepArgs& a, const int4* tiles, int n_tiles, int tpb,
                            cudaStream_t st) {
  auto kernel = SINGLE ? step_batched_single_kernel<INTEG, CTRL, MOTOR, SYM>
                       : step_batched_kernel<INTEG, CTRL, MOTOR, SYM>;
  // occupancy per (device, block size), queried once per kernel variant
  static int cached[16][9] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int slot = tpb / 32;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = (dev < 16 && slot <= 8) ? cached[dev][slot] : 0;
  if (per_sm == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, tpb, 0);
    if (per_sm < 1) per_sm = 1;
    if (dev < 16 && slot <= 8) cached[dev][slot] = per_sm;
  }
  const int warps_per_block = tpb / 32;
  int grid = sms * per_sm;
  const int need = (n_tiles + warps_per_block - 1) / warps_per_block;
  if (grid > need) grid = need;
  return launch_chained(kernel, grid, tpb, st, a, tiles, n_tiles);
}

cudaError_t launch_step_batched(const StepArgs& a, const int4* tiles, int n_tiles, int integrator,
                                int ctrl, bool general_motor, bool sym, int tpb, cudaStream_t st) {
#define CF_L(I, C, S)                                                                       \
  (sym ? launch_b<I, C, MOTOR_LAG, S, true>(a, tiles, n_tiles, tpb, st)                      \
       : launch_b<I, C, MOTOR_LAG, S, false>(a, tiles, n_tiles, tpb, st))
#define CF_B(I, C)                                                                          \
  {                                                                                         \
    if (a.K == 1)                                                                           \
      return general_motor ? launch_b<I, C, MOTOR_GENERAL, true>(a, tiles, n_tiles, tpb, st) \
                           : CF_L(I, C, true);                                              \
    return general_motor ? launch_b<I, C, MOTOR_GENERAL, false>(a, tiles, n_tiles, tpb, st)  \
                         : CF_L(I, C, false);                                               \
  }
  if (integrator == SIM_RK4) {
    if (ctrl == SIM_CTRL_ROTOR_SPEED) CF_B(SIM_RK4, SIM_CTRL_ROTOR_SPEED);
    if (ctrl == SIM_CTRL_POSITION) CF_B(SIM_RK4, SIM_CTRL_POSITION);
    if (ctrl == SIM_CTRL_TORQUE) CF_B(SIM_RK4, SIM_CTRL_TORQUE);
    CF_B(SIM_RK4, SIM_CTRL_ATTITUDE);
  }
  if (ctrl == SIM_CTRL_ROTOR_SPEED) CF_B(SIM_EULER, SIM_CTRL_ROTOR_SPEED);
  if (ctrl == SIM_CTRL_POSITION) CF_B(SIM_EULER, SIM_CTRL_POSITION);
  if (ctrl == SIM_CTRL_TORQUE) CF_B(SIM_EULER, SIM_CTRL_TORQUE);
  CF_B(SIM_EULER, SIM_CTRL_ATTITUDE);
#undef CF_B
#undef CF_L
}

template <int MODEL, int INTEG, int CTRL, int MOTOR, bool PERSET, bool SYM = false>
static cudaError_t launch_t(const StepArgs& a, const DevParams& P, int tpb, cudaStream_t st) {
  const int grid = (a.n + tpb - 1) / tpb;
  return launch_chained(step_kernel<MODEL, INTEG, CTRL, MOTOR, PERSET, SYM>, grid, tpb, st, a, P);
}

template <int MODEL, int INTEG, int CTRL>
static cudaError_t launch_m(const StepArgs& a, const DevParams& P, bool gm, bool perset, int tpb,
                            cudaStream_t st) {
  if (gm) {
    return perset ? launch_t<MODEL, INTEG, CTRL, MOTOR_GENERAL, true>(a, P, tpb, st)
                  : launch_t<MODEL, INTEG, CTRL, MOTOR_GENERAL, false>(a, P, tpb, st);
  }
  // first-principles lag-rotor steps come in two forms: Jx = Jy in every set (the
  // union of the sets' flags lacks PF_ASYM_XY) or not
  if constexpr (MODEL == SIM_FIRST_PRINCIPLES) {
    if ((P.flags & PF_ASYM_XY) == 0)
      return perset ? launch_t<MODEL, INTEG, CTRL, MOTOR_LAG, true, true>(a, P, tpb, st)
                    : launch_t<MODEL, INTEG, CTRL, MOTOR_LAG, false, true>(a, P, tpb, st);
  }
  return perset ? launch_t<MODEL, INTEG, CTRL, MOTOR_LAG, true>(a, P, tpb, st)
                : launch_t<MODEL, INTEG, CTRL, MOTOR_LAG, false>(a, P, tpb, st);
}

template <int MODEL, int INTEG>
static cudaError_t launch_c(const StepArgs& a, const DevParams& P, int ctrl, bool gm, bool perset,
                            int tpb, cudaStream_t st) {
  if constexpr (MODEL != SIM_FIRST_PRINCIPLES) {
    // the abstracted models have no rotors: the general variant only adds drag
    return launch_m<MODEL, INTEG, SIM_CTRL_ATTITUDE>(a, P, gm, perset, tpb, st);
  } else {
    switch (ctrl) {
      case SIM_CTRL_ROTOR_SPEED:
        return launch_m<MODEL, INTEG, SIM_CTRL_ROTOR_SPEED>(a, P, gm, perset, tpb, st);
      case SIM_CTRL_POSITION:
        return launch_m<MODEL, INTEG, SIM_CTRL_POSITION>(a, P, gm, perset, tpb, st);
      case SIM_CTRL_TORQUE:
        return launch_m<MODEL, INTEG, SIM_CTRL_TORQUE>(a, P, gm, perset, tpb, st);
      default:
        return launch_m<MODEL, INTEG, SIM_CTRL_ATTITUDE>(a, P, gm, perset, tpb, st);
    }
  }
}

cudaError_t launch_step(const StepArgs& a, const DevParams& P, int model, int integrator, int ctrl,
                        bool general_motor, bool per_set, int tpb, cudaStream_t st) {
  if (model == SIM_FIRST_PRINCIPLES) {
    return integrator == SIM_RK4
               ? launch_c<SIM_FIRST_PRINCIPLES, SIM_RK4>(a, P, ctrl, general_motor, per_set, tpb, st)
               : launch_c<SIM_FIRST_PRINCIPLES, SIM_EULER>(a, P, ctrl, general_motor, per_set, tpb,
                                                           st);
  }
  if (model == SIM_ABSTRACTED_NOTHRUST) {
    return integrator == SIM_RK4
               ? launch_c<SIM_ABSTRACTED_NOTHRUST, SIM_RK4>(a, P, ctrl, general_motor, per_set, tpb,
                                                            st)
               : launch_c<SIM_ABSTRACTED_NOTHRUST, SIM_EULER>(a, P, ctrl, general_motor, per_set,
                                                              tpb, st);
  }
  return integrator == SIM_RK4
             ? launch_c<SIM_ABSTRACTED, SIM_RK4>(a, P, ctrl, general_motor, per_set, tpb, st)
             : launch_c<SIM_ABSTRACTED, SIM_EULER>(a, P, ctrl, general_motor, per_set, tpb, st);
}

}  // namespace cf
