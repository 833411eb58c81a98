// The handle behind sim_h (private to the library's translation units).
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

struct sim_s {
  int64_t M = 0, N = 0, ntot = 0;
  bool batched = false;
  int model = SIM_FIRST_PRINCIPLES;  // uniform batches
  int integrator = SIM_EULER;
  int ctrl = SIM_CTRL_ATTITUDE;
  float dt = 0.f;
  int tpb = 128;         // threads per block of the step launches
  int tpb_sample = 128;  // and of the sampling launches
  std::vector<int64_t> n_per_world, offset;
  std::vector<int32_t> model_of_world;
  std::vector<int4> tiles;  // uneven batches: (first drone, count <= 32, world, model)
  std::vector<int32_t> offsets32;  // uneven batches: first drone of each world, [M + 1]
  // workspace (caller-owned device memory) and the device that holds it
  char* ws = nullptr;
  int device = -1;
  size_t ws_bytes = 0;
  int64_t max_blocks = 0;
  float4* planes = nullptr;
  cf::DevParams* params_dev = nullptr;
  int32_t* set_of_world_dev = nullptr;
  float4* cmd = nullptr;
  float4* staging = nullptr;
  uint32_t* status = nullptr;
  int4* tiles_dev = nullptr;
  int32_t* offsets_dev = nullptr;
  // host copies
  std::vector<cf::DevParams> params_host;
  cf::DevParams p0;  // the single set of a uniform batch, passed by value
  std::vector<int32_t> set_of_world_host;
  bool params_ok = false, per_set = false, general_motor = false, state_ok = false;
  int64_t n_blocks = 0;
  int hold = 1;
  int64_t t = 0;
  int64_t launches = 0;
  cf::RolloutObjective objective;
  int rollout_repeat = 1;
  char err[512] = {0};
};


namespace cf {
// The sampling launch behind sim_sample_rollouts and sim_mppi_iteration
// (sim.cu); n_ctrl = 0 for plain sampling.
int sample_launch(sim_h h, int S, int H, const uint64_t* seed, float sigma, const float* nominal,
                const float* goals, const float* obstacles, int n_obs, float w_obs, float* cost,
                void* stream, int n_ctrl, float rho);
}  // namespace cf
