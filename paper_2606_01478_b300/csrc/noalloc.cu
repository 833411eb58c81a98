// Policy-rollout gradient that needs no caller-provided workspace.
//
// The regular entry points take their scratch memory (checkpoints, segment
// states, per-drone losses, dW partials) from a workspace the caller allocates.
// Some callers cannot allocate device memory at the point where they need a
// gradient: a control loop with a hard deadline (cudaMalloc can synchronise the
// device and take milliseconds), or a plugin whose host framework owns every
// device allocation.  For them, sim_rollout_grad_noalloc runs the same kernels
// with their scratch in the fixed-size array below, which every GPU that loads
// this library holds until the process exits.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;  // 8 MiB

// File-scope device scratch.  In host code these names are host-side stand-ins,
// not device addresses: the address is resolved with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_rollout_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ __align__(16) float g_unit_seed = 1.0f;

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};
float* g_seed_ptr[MAX_DEVICES] = {};

// Resolve the device addresses once per device, with that device current.
cudaError_t device_pointers(void** scratch, const float** seed) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    e = cudaGetSymbolAddress(&p, g_rollout_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_unit_seed);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_seed_ptr[dev] = static_cast<float*>(q);
  }
  *scratch = g_scratch_ptr[dev];
  *seed = g_seed_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int sim_rollout_noalloc_max_bytes(size_t* bytes) {
  if (!bytes) return SIM_EINVAL;
  *bytes = NOALLOC_SCRATCH_BYTES;
  return SIM_OK;
}

extern "C" int sim_rollout_grad_noalloc(sim_h h, const float* x0, const uint16_t* w,
                                        const float* p_ref, int H, int C, float w_act,
                                        float* loss, float* dW, float* dx0, void* stream) {
  if (!h) return SIM_EINVAL;
  size_t need = 0;
  int r = sim_rollout_workspace_bytes(h, H, C, &need);
  if (r != SIM_OK) return r;
  if (need > NOALLOC_SCRATCH_BYTES) {
    cf::note_error(h, "sim_rollout_grad_noalloc: this batch needs %zu bytes of scratch, more "
                      "than the %zu-byte built-in scratch; use sim_rollout_grad with a workspace",
                   need, NOALLOC_SCRATCH_BYTES);
    return SIM_EINVAL;
  }
  // The array exists once per device and is looked up for the current one:
  // the handle's buffers must be on that same device.
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != cf::handle_device(h)) {
    cudaGetLastError();
    cf::note_error(h, "sim_rollout_grad_noalloc: device %d is current, the handle's workspace is "
                      "on device %d; make the handle's device current first",
                   cur, cf::handle_device(h));
    return SIM_EINVAL;
  }
  void* scratch = nullptr;
  const float* seed = nullptr;
  cudaError_t e = device_pointers(&scratch, &seed);
  if (e != cudaSuccess) {
    cf::note_error(h, "sim_rollout_grad_noalloc: resolving the built-in scratch failed: %s",
                   cudaGetErrorString(e));
    return SIM_ECUDA;
  }
  return sim_rollout_grad(h, x0, w, p_ref, H, C, w_act, scratch, NOALLOC_SCRATCH_BYTES, loss, seed,
                          dW, dx0, stream);
}
