// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace cf {

// Forward step launch (step.cu).  per_set: parameters per world from a.params.
cudaError_t launch_step(const StepArgs& a, const DevParams& P, int model, int integrator, int ctrl,
                        bool general_motor, bool per_set, int tpb, cudaStream_t st);

// Uneven / mixed batches (step.cu): tiles [n_tiles] of (first drone, count <= 32,
// world, model), one warp per tile, persistent grid.  sym: Jx = Jy in every
// parameter set.
cudaError_t launch_step_batched(const StepArgs& a, const int4* tiles, int n_tiles, int integrator,
                                int ctrl, bool general_motor, bool sym, int tpb, cudaStream_t st);

// Differentiable policy rollout (rollout.cu).  Workspace: checkpoints
// [ceil(H/C)][n][20], segment sub-step states [C R][n][20], per-drone loss [n], per-CTA dW
// partials; all fp32; with the tracking reward also the previous action at each
// checkpoint [ceil(H/C)][n] and segment step [C][n] (float4).
constexpr int POLICY_NPARAMS = 5316;
// Objective of the policy rollout (SIM_OBJ_*) with the tracking-reward weights.
struct RolloutObjective {
  int kind = SIM_OBJ_SQUARED;
  bool hilo = true;  // MLP operands as hi + lo bf16 pairs (SIM_MLP_HILO) or plain bf16
  float w_theta = 0.f, w_act[4] = {0.f, 0.f, 0.f, 0.f}, w_dact[4] = {0.f, 0.f, 0.f, 0.f};
};
size_t rollout_workspace_bytes(int n, int H, int C, int objective, int R);
cudaError_t launch_rollout_fwd(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                               int C, int R, float dt, float w_act, const RolloutObjective& obj,
                               const DevParams& P, void* ws,
                               float* loss, bool store_ckpt, cudaStream_t st);
// Self-test of the bounded in-kernel waits (rollout.cu): sets SIM_FLAG_TIMEOUT.
cudaError_t launch_wait_selftest(uint32_t* status, cudaStream_t st);
cudaError_t launch_rollout_bwd(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                               int C, int R, float dt, float w_act, const RolloutObjective& obj,
                               const DevParams& P, void* ws, const float* dL, float* dW, float* dx0,
                               uint32_t* status, cudaStream_t st);
// Forward and adjoint in one adjoint launch (its recompute warps run the forward
// pass first), then the loss and dW reductions.
cudaError_t launch_rollout_grad(const float* x0, const uint16_t* w, const float* p_ref, int n, int H,
                                int C, int R, float dt, float w_act, const RolloutObjective& obj,
                                const DevParams& P, void* ws, float* loss, const float* dL, float* dW,
                                float* dx0, uint32_t* status, cudaStream_t st);

// Batched sampling rollouts (sample.cu).
cudaError_t launch_sample(const float4* planes, int n, const int* offsets, int M, int N,
                          const float* goals, const float* nominal, const unsigned long long* seed,
                          const DevParams* params, const int32_t* set_of_world, const DevParams& P0,
                          bool per_set, bool general_motor, int integrator, const float* obstacles,
                          int n_obs, float w_obs, float sigma, float dt, int S, int H, float* cost,
                          int tpb, cudaStream_t st, int n_ctrl = 0, float rho = 0.f);
cudaError_t launch_mppi_update(const float* cost, float* mean, float* plan, float* best_cost,
                               const unsigned long long* seed, int n, int S, int H, int C, int n_e,
                               float sigma, float rho, float lambda, cudaStream_t st);

// The MPPI update and the elite selection run one warp per controller when a
// controller has at most 2048 samples and 32 elites (mppi.cu), else one thread
// block per controller (the update: a drone's controllers in one cluster).
bool mppi_uses_warp_path(int S_c, int n_e);
cudaError_t launch_elite_select(const float* cost, long long rows, int S_c, int n_e, int* idx,
                                float* jmin, cudaStream_t st);
cudaError_t launch_philox(const unsigned long long* seed, unsigned long long first_id, long long n,
                          int step, uint32_t* words, float* normals, cudaStream_t st);

cudaError_t launch_adam(const float* g, float* w, float* m, float* v, uint16_t* wb, int n, int* step,
                        float lr, float b1, float b2, float eps, cudaStream_t st);

// Depth rendering by ray casting (raycast.cu).
cudaError_t launch_depth(const float4* planes, int n, int H, int W, float hfov, float vfov,
                         float max_range, const float* spheres, int n_sph, const float* boxes,
                         int n_box, float* out, cudaStream_t st);

// Record a message as the handle's last error (sim.cu); used by entry points
// defined in other translation units.
void note_error(sim_h h, const char* fmt, ...);
// The device that holds the handle's workspace (-1 before sim_bind).
int handle_device(sim_h h);

// Row-major [n][20] floats <-> 5 float4 planes [5][n] (layout.cu).
cudaError_t launch_rows_to_planes(const float4* rows, float4* planes, int n, cudaStream_t st);
cudaError_t launch_planes_to_rows(const float4* planes, float4* rows, int n, cudaStream_t st);
// grid-stride 16-byte copy with at most max_blocks blocks of 256 threads
cudaError_t launch_copy16(const float4* src, float4* dst, int64_t n, int max_blocks, cudaStream_t st);

}  // namespace cf
