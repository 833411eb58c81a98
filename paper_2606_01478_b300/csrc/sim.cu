// C-ABI of the B300 drone step: handle management, argument validation,
// workspace layout, host<->device transfers and kernel dispatch.
// Declarations and contracts: include/crazyflow.h.
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <initializer_list>
#include <new>
#include <vector>

#include "handle.h"
#include "internal.h"

using cf::DevParams;

namespace {

int fail(sim_h h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(sim_h h, cudaError_t e, const char* what) {
  return fail(h, SIM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t planes, params, set_of_world, cmd, staging, status, tiles, offsets, total;
};

Layout layout_of(const sim_s* h, int64_t max_blocks) {
  Layout L;
  size_t off = 0;
  L.planes = off;
  off = align256(off + (size_t)h->ntot * 5 * sizeof(float4));
  L.params = off;
  off = align256(off + (size_t)h->M * sizeof(DevParams));
  L.set_of_world = off;
  off = align256(off + (size_t)h->M * sizeof(int32_t));
  L.cmd = off;
  off = align256(off + (size_t)max_blocks * h->ntot * sizeof(float4));
  L.staging = off;
  off = align256(off + (size_t)h->ntot * SIM_STATE_DIM * sizeof(float));
  L.status = off;  // status word, then the two tile counters of the batched kernels
  off = align256(off + 3 * sizeof(uint32_t));
  L.tiles = off;
  off = align256(off + h->tiles.size() * sizeof(int4));
  L.offsets = off;
  off = align256(off + h->offsets32.size() * sizeof(int32_t));
  L.total = off;
  return L;
}

// Where kernels can reach a caller's buffer: itself for device memory, its device
// address for pinned host memory (kernels then move the data over the host link
// themselves), nullptr for pageable host memory (copy-engine transfers).
const void* kernel_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) return a.devicePointer;
  return nullptr;
}

bool valid_enums(int model, int integrator) {
  return (model == SIM_FIRST_PRINCIPLES || model == SIM_ABSTRACTED ||
          model == SIM_ABSTRACTED_NOTHRUST) &&
         (integrator == SIM_EULER || integrator == SIM_RK4);
}

// Host derivation of the kernel constants from one user parameter vector.
int derive_params(const float* p, DevParams* d, char* why, size_t why_n) {
  for (int k = 0; k < SIM_P_COUNT; ++k) {
    if (!isfinite(p[k])) {
      snprintf(why, why_n, "parameter %d is not finite", k);
      return SIM_EINVAL;
    }
  }
  const int pos[] = {SIM_P_MASS, SIM_P_JX, SIM_P_JY, SIM_P_JZ, SIM_P_ARM, SIM_P_KF, SIM_P_KM,
                     SIM_P_OMEGA_MAX};
  for (int k : pos) {
    if (!(p[k] > 0.f)) {
      snprintf(why, why_n, "parameter %d must be > 0", k);
      return SIM_EINVAL;
    }
  }
  const double m = p[SIM_P_MASS], g = p[SIM_P_G];
  const double Jx = p[SIM_P_JX], Jy = p[SIM_P_JY], Jz = p[SIM_P_JZ];
  const double a = p[SIM_P_ARM] / sqrt(2.0);
  const double kf = p[SIM_P_KF], km = p[SIM_P_KM], wmax = p[SIM_P_OMEGA_MAX];
  memset(d, 0, sizeof(*d));
  d->inv_m = (float)(1.0 / m);
  d->g = (float)g;
  d->mass = (float)m;
  d->inv_Jx = (float)(1.0 / Jx);
  d->inv_Jy = (float)(1.0 / Jy);
  d->inv_Jz = (float)(1.0 / Jz);
  d->cJx = (float)((Jy - Jz) / Jx);
  d->cJy = (float)((Jz - Jx) / Jy);
  d->cJz = (float)((Jx - Jy) / Jz);
  d->kf = (float)kf;
  d->kfa = (float)(kf * a);
  d->km = (float)km;
  d->cv_up = p[SIM_P_CV_UP];
  d->cd_up = p[SIM_P_CD_UP];
  d->cv_down = p[SIM_P_CV_DOWN];
  d->cd_down = p[SIM_P_CD_DOWN];
  d->Ca_x = p[SIM_P_CA_X];
  d->Ca_y = p[SIM_P_CA_Y];
  d->Ca_z = p[SIM_P_CA_Z];
  d->KRJh_x = (float)(0.5 * p[SIM_P_KR_X] * Jx);
  d->KRJh_y = (float)(0.5 * p[SIM_P_KR_Y] * Jy);
  d->KRJh_z = (float)(0.5 * p[SIM_P_KR_Z] * Jz);
  d->KwJ_x = (float)(p[SIM_P_KW_X] * Jx);
  d->KwJ_y = (float)(p[SIM_P_KW_Y] * Jy);
  d->KwJ_z = (float)(p[SIM_P_KW_Z] * Jz);
  d->Kp_x = p[SIM_P_KP_X];
  d->Kp_y = p[SIM_P_KP_Y];
  d->Kp_z = p[SIM_P_KP_Z];
  d->Kd_x = p[SIM_P_KD_X];
  d->Kd_y = p[SIM_P_KD_Y];
  d->Kd_z = p[SIM_P_KD_Z];
  d->Ki_x = p[SIM_P_KI_X];
  d->Ki_y = p[SIM_P_KI_Y];
  d->Ki_z = p[SIM_P_KI_Z];
  d->max_angle = p[SIM_P_MAX_ANGLE];
  d->half_max_angle = (float)(0.5 * p[SIM_P_MAX_ANGLE]);
  d->mg = (float)(m * g);
  d->ts_mg = (float)(p[SIM_P_THRUST_SCALE] * m * g);
  d->mix_a = (float)(1.0 / (4.0 * a));
  d->mix_k = (float)(kf / (4.0 * km));
  d->inv_kf = (float)(1.0 / kf);
  d->fmax = (float)(kf * wmax * wmax);
  d->omega_max = (float)wmax;
  d->c1_r = p[SIM_P_C1_R];
  d->c1_p = p[SIM_P_C1_P];
  d->c1_y = p[SIM_P_C1_Y];
  d->c2_r = p[SIM_P_C2_R];
  d->c2_p = p[SIM_P_C2_P];
  d->c2_y = p[SIM_P_C2_Y];
  d->c3_r = p[SIM_P_C3_R];
  d->c3_p = p[SIM_P_C3_P];
  d->c3_y = p[SIM_P_C3_Y];
  d->c_tau = p[SIM_P_C_TAU];
  d->cf_inv_m = (float)(p[SIM_P_C_F] / m);
  const double kf0 = p[SIM_P_KF0], kf1 = p[SIM_P_KF1];
  d->kf0 = (float)kf0;
  d->kf1 = (float)kf1;
  d->km1 = p[SIM_P_KM1];
  d->kf1sq = (float)(kf1 * kf1);
  d->four_kf = (float)(4.0 * kf);
  d->inv_2kf = (float)(1.0 / (2.0 * kf));
  d->Jpc = (float)(p[SIM_P_J_P] * 2.0 * M_PI / 60.0);
  d->fmax = (float)(kf * wmax * wmax + kf1 * wmax + kf0);
  {
    // lag-rotor step form (see DevParams)
    const double cv = p[SIM_P_CV_UP], cv2kf = cv * cv / kf;
    const double mix_a = 1.0 / (4.0 * a), mix_k = kf / (4.0 * km);
    d->kfm = (float)(kf / m);
    d->kfm2 = (float)(2.0 * kf / m);
    d->kfaJx = (float)(kf * a / Jx);
    d->kfaJy = (float)(kf * a / Jy);
    d->kmJz = (float)(km / Jz);
    d->ncv = (float)(-cv);
    d->cA = (float)(0.25 * cv2kf);
    d->cRx = (float)(0.5 * p[SIM_P_KR_X] * Jx * mix_a * cv2kf);
    d->cRy = (float)(0.5 * p[SIM_P_KR_Y] * Jy * mix_a * cv2kf);
    d->cRz = (float)(0.5 * p[SIM_P_KR_Z] * Jz * mix_k * cv2kf);
    d->cwx = (float)(p[SIM_P_KW_X] * Jx * mix_a * cv2kf);
    d->cwy = (float)(p[SIM_P_KW_Y] * Jy * mix_a * cv2kf);
    d->cwz = (float)(p[SIM_P_KW_Z] * Jz * mix_k * cv2kf);
    d->cXt = (float)(mix_a * cv2kf);
    d->cZt = (float)(mix_k * cv2kf);
    d->u2max = (float)(cv * cv * wmax * wmax);
  }
  int flags = 0;
  // drag also selects the general kernel variants: the lag-rotor variants carry
  // no drag term (and no branch on it in the hot loop)
  if (p[SIM_P_CA_X] != 0.f || p[SIM_P_CA_Y] != 0.f || p[SIM_P_CA_Z] != 0.f)
    flags |= cf::PF_DRAG | cf::PF_GENERAL_MOTOR;
  if (p[SIM_P_CV_UP] != p[SIM_P_CV_DOWN] || p[SIM_P_CD_UP] != 0.f || p[SIM_P_CD_DOWN] != 0.f ||
      p[SIM_P_J_P] != 0.f || kf0 != 0.0 || kf1 != 0.0 || p[SIM_P_KM1] != 0.f)
    flags |= cf::PF_GENERAL_MOTOR;
  if (Jx != Jy) flags |= cf::PF_ASYM_XY;
  d->flags = flags;
  return SIM_OK;
}

}  // namespace

namespace cf {
void note_error(sim_h h, const char* fmt, ...) {
  if (!h) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(h->err, sizeof(h->err), fmt, ap);
  va_end(ap);
}
int handle_device(sim_h h) { return h ? h->device : -1; }

int sample_launch(sim_h h, int S, int H, const uint64_t* seed, float sigma,
                       const float* nominal, const float* goals, const float* obstacles, int n_obs,
                       float w_obs, float* cost, void* stream, int n_ctrl, float rho) {
  if (!h) return SIM_EINVAL;
  if (!h->ws || !h->params_ok || !h->state_ok)
    return fail(h, SIM_ESTATE, "bind, parameters and state must be set before sampling");
  bool all_fp = h->batched ? true : h->model == SIM_FIRST_PRINCIPLES;
  for (int32_t m : h->model_of_world) all_fp &= (m == SIM_FIRST_PRINCIPLES);
  if (!all_fp) return fail(h, SIM_EINVAL, "sampling rollouts need first-principles drones");
  if (h->ctrl != SIM_CTRL_ATTITUDE)
    return fail(h, SIM_EINVAL, "sampling rollouts use the attitude interface");
  if (S < 1 || H < 1 || n_obs < 0 || n_obs > SIM_MAX_OBSTACLES || !(sigma >= 0.f) ||
      !isfinite(sigma) || !isfinite(w_obs))
    return fail(h, SIM_EINVAL, "need S, H >= 1, 0 <= n_obs <= %d, finite sigma >= 0",
                SIM_MAX_OBSTACLES);
  if ((double)h->ntot * S > 4.0e18) return fail(h, SIM_EINVAL, "too many rollouts");
  if (!seed || ((uintptr_t)seed & 7) || !goals || ((uintptr_t)goals & 3) || !cost ||
      ((uintptr_t)cost & 3) || (nominal && ((uintptr_t)nominal & 15)) || (n_obs > 0 && !obstacles))
    return fail(h, SIM_EINVAL, "bad or misaligned buffer");
  for (int o = 0; o < n_obs; ++o) {
    for (int j = 0; j < 4; ++j)
      if (!isfinite(obstacles[4 * o + j])) return fail(h, SIM_EINVAL, "obstacle %d not finite", o);
    if (obstacles[4 * o + 3] < 0.f) return fail(h, SIM_EINVAL, "obstacle %d has a negative radius", o);
  }
  // one parameter set for every world (uniform or batched): the parameters are
  // kernel arguments (constant bank); otherwise each rollout reads its world's set
  cudaError_t e = cf::launch_sample(
      h->planes, (int)h->ntot, h->batched ? h->offsets_dev : nullptr, (int)h->M, (int)h->N, goals,
      nominal, (const unsigned long long*)seed, h->params_dev, h->set_of_world_dev, h->p0,
      h->per_set, h->general_motor, h->integrator, obstacles, n_obs, w_obs, sigma,
      h->dt, S, H, cost, h->tpb_sample, (cudaStream_t)stream, n_ctrl, rho);
  if (e != cudaSuccess) return cuda_fail(h, e, "sampling launch");
  h->launches++;
  return SIM_OK;
}

}  // namespace cf

extern "C" {

int sim_create(sim_h* out, int64_t M, int64_t N, int model, int integrator, float dt) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (M < 1 || N < 1 || M * N > 0x7fffffffLL || !valid_enums(model, integrator) || !(dt > 0.f) ||
      !isfinite(dt))
    return SIM_EINVAL;
  sim_s* h = new (std::nothrow) sim_s();
  if (!h) return SIM_ENOMEM;
  h->M = M;
  h->N = N;
  h->ntot = M * N;
  h->model = model;
  h->integrator = integrator;
  h->dt = dt;
  *out = h;
  return SIM_OK;
}

int sim_create_batched(sim_h* out, int64_t M, const int64_t* n_per_world,
                       const int32_t* model_per_world, int integrator, float dt) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  if (M < 1 || !n_per_world || !model_per_world || !valid_enums(SIM_FIRST_PRINCIPLES, integrator) ||
      !(dt > 0.f) || !isfinite(dt))
    return SIM_EINVAL;
  int64_t tot = 0;
  for (int64_t w = 0; w < M; ++w) {
    if (n_per_world[w] < 1 || !valid_enums(model_per_world[w], integrator)) return SIM_EINVAL;
    tot += n_per_world[w];
    if (tot > 0x7fffffffLL) return SIM_EINVAL;
  }
  sim_s* h = new (std::nothrow) sim_s();
  if (!h) return SIM_ENOMEM;
  h->M = M;
  h->N = 0;
  h->ntot = tot;
  h->batched = true;
  h->integrator = integrator;
  h->dt = dt;
  h->n_per_world.assign(n_per_world, n_per_world + M);
  h->model_of_world.assign(model_per_world, model_per_world + M);
  h->offset.resize(M + 1);
  h->offset[0] = 0;
  for (int64_t w = 0; w < M; ++w) h->offset[w + 1] = h->offset[w] + n_per_world[w];
  for (int64_t w = 0; w < M; ++w) {
    for (int64_t s = 0; s < n_per_world[w]; s += 32) {
      const int64_t c = n_per_world[w] - s < 32 ? n_per_world[w] - s : 32;
      h->tiles.push_back(make_int4((int)(h->offset[w] + s), (int)c, (int)w, model_per_world[w]));
    }
  }
  h->offsets32.assign(h->offset.begin(), h->offset.end());
  *out = h;
  return SIM_OK;
}

int sim_set_control(sim_h h, int ctrl) {
  if (!h) return SIM_EINVAL;
  if (ctrl != SIM_CTRL_ROTOR_SPEED && ctrl != SIM_CTRL_ATTITUDE && ctrl != SIM_CTRL_POSITION &&
      ctrl != SIM_CTRL_TORQUE)
    return fail(h, SIM_EINVAL, "unknown control interface %d", ctrl);
  bool any_abs = h->batched ? false : h->model != SIM_FIRST_PRINCIPLES;
  for (int32_t m : h->model_of_world) any_abs |= (m != SIM_FIRST_PRINCIPLES);
  if (any_abs && ctrl != SIM_CTRL_ATTITUDE)
    return fail(h, SIM_EINVAL, "the abstracted model takes attitude commands only");
  h->ctrl = ctrl;
  return SIM_OK;
}

int sim_workspace_bytes(sim_h h, int64_t max_cmd_blocks, size_t* bytes) {
  if (!h || !bytes || max_cmd_blocks < 1) return h ? fail(h, SIM_EINVAL, "bad arguments") : SIM_EINVAL;
  *bytes = layout_of(h, max_cmd_blocks).total;
  return SIM_OK;
}

int sim_bind(sim_h h, void* workspace, size_t bytes, int64_t max_cmd_blocks, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!workspace || max_cmd_blocks < 1 || ((uintptr_t)workspace & 255))
    return fail(h, SIM_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  const Layout L = layout_of(h, max_cmd_blocks);
  if (bytes < L.total)
    return fail(h, SIM_ENOMEM, "workspace of %zu bytes is smaller than the %zu needed", bytes,
                L.total);
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, workspace) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(h, SIM_EINVAL, "workspace must be device memory");
  }
  char* ws = (char*)workspace;
  h->device = pa.device;
  h->ws = ws;
  h->ws_bytes = bytes;
  h->max_blocks = max_cmd_blocks;
  h->planes = (float4*)(ws + L.planes);
  h->params_dev = (DevParams*)(ws + L.params);
  h->set_of_world_dev = (int32_t*)(ws + L.set_of_world);
  h->cmd = (float4*)(ws + L.cmd);
  h->staging = (float4*)(ws + L.staging);
  h->status = (uint32_t*)(ws + L.status);
  h->tiles_dev = (int4*)(ws + L.tiles);
  h->offsets_dev = (int32_t*)(ws + L.offsets);
  h->params_ok = h->state_ok = false;
  h->n_blocks = 0;
  h->t = 0;
  cudaError_t e = cudaMemsetAsync(h->status, 0, 3 * sizeof(uint32_t), (cudaStream_t)stream);
  if (e == cudaSuccess && !h->tiles.empty())
    e = cudaMemcpyAsync(h->tiles_dev, h->tiles.data(), h->tiles.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e == cudaSuccess && !h->offsets32.empty())
    e = cudaMemcpyAsync(h->offsets_dev, h->offsets32.data(), h->offsets32.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "initialising the workspace");
  return SIM_OK;
}

int sim_set_params(sim_h h, const float* params, int64_t n_sets, const int32_t* set_of_world,
                   void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws) return fail(h, SIM_ESTATE, "sim_bind must come first");
  if (!params || n_sets < 1 || n_sets > h->M)
    return fail(h, SIM_EINVAL, "need 1 <= n_sets <= M and a parameter array");
  std::vector<DevParams> dp((size_t)n_sets);
  char why[128];
  for (int64_t s = 0; s < n_sets; ++s) {
    if (derive_params(params + s * SIM_NPARAMS, &dp[(size_t)s], why, sizeof(why)) != SIM_OK)
      return fail(h, SIM_EINVAL, "parameter set %lld: %s", (long long)s, why);
  }
  std::vector<int32_t> sow((size_t)h->M, 0);
  bool uniform = true;
  if (set_of_world) {
    for (int64_t w = 0; w < h->M; ++w) {
      if (set_of_world[w] < 0 || set_of_world[w] >= n_sets)
        return fail(h, SIM_EINVAL, "set_of_world[%lld] = %d out of range", (long long)w,
                    set_of_world[w]);
      sow[(size_t)w] = set_of_world[w];
      uniform &= (set_of_world[w] == set_of_world[0]);
    }
  }
  int flags = 0;
  for (const DevParams& d : dp) flags |= d.flags;
  h->params_host = dp;
  h->set_of_world_host = sow;
  h->per_set = !uniform;
  h->general_motor = (flags & cf::PF_GENERAL_MOTOR) != 0;
  // every set carries the union of the flags so one kernel variant serves all
  for (DevParams& d : h->params_host) d.flags = flags;
  h->p0 = h->params_host[(size_t)sow[0]];
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h->params_dev, h->params_host.data(),
                                  h->params_host.size() * sizeof(DevParams),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->set_of_world_dev, h->set_of_world_host.data(),
                        h->set_of_world_host.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "uploading parameters");
  h->params_ok = true;
  return SIM_OK;
}

int sim_set_state(sim_h h, const float* x, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws) return fail(h, SIM_ESTATE, "sim_bind must come first");
  if (!x || ((uintptr_t)x & 15)) return fail(h, SIM_EINVAL, "state pointer must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  const float4* rows = (const float4*)kernel_view(x);  // device or pinned host: read in place
  cudaError_t e;
  if (!rows) {
    e = cudaMemcpyAsync(h->staging, x, (size_t)h->ntot * SIM_STATE_DIM * sizeof(float),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying the state to the device");
    rows = h->staging;
  }
  e = cf::launch_rows_to_planes(rows, h->planes, (int)h->ntot, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "rows_to_planes launch");
  h->launches++;
  h->state_ok = true;
  return SIM_OK;
}

int sim_get_state(sim_h h, float* x, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws || !h->state_ok) return fail(h, SIM_ESTATE, "no state has been set");
  if (!x || ((uintptr_t)x & 15)) return fail(h, SIM_EINVAL, "state pointer must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  float4* view = (float4*)kernel_view(x);  // device or pinned host: written in place
  float4* rows = view ? view : h->staging;
  cudaError_t e = cf::launch_planes_to_rows(h->planes, rows, (int)h->ntot, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "planes_to_rows launch");
  h->launches++;
  if (!view) {
    e = cudaMemcpyAsync(x, h->staging, (size_t)h->ntot * SIM_STATE_DIM * sizeof(float),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying the state to the host");
  }
  return SIM_OK;
}

int sim_set_commands(sim_h h, const float* cmd, int64_t n_blocks, int hold, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws) return fail(h, SIM_ESTATE, "sim_bind must come first");
  if (!cmd || n_blocks < 1 || n_blocks > h->max_blocks || hold < 1 ||
      n_blocks * (int64_t)hold > 0x7fffffffLL)
    return fail(h, SIM_EINVAL, "need a command array, 1 <= n_blocks <= %lld, hold >= 1",
                (long long)h->max_blocks);
  const float4* view = (const float4*)kernel_view(cmd);
  cudaError_t e = view ? cf::launch_copy16(view, h->cmd, n_blocks * h->ntot, 592, (cudaStream_t)stream)
                       : cudaMemcpyAsync(h->cmd, cmd, (size_t)n_blocks * h->ntot * sizeof(float4),
                                         cudaMemcpyDefault, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "copying commands");
  h->n_blocks = n_blocks;
  h->hold = hold;
  h->t = 0;
  return SIM_OK;
}

int sim_set_block_size(sim_h h, int tpb) {
  if (!h) return SIM_EINVAL;
  if (tpb < 32 || tpb > 256 || (tpb & 31)) return fail(h, SIM_EINVAL, "bad block size %d", tpb);
  h->tpb = tpb;
  h->tpb_sample = tpb;
  return SIM_OK;
}

int sim_step(sim_h h, int K, void* stream) {
  if (!h) return SIM_EINVAL;
  if (K < 1 || K > 100000) return fail(h, SIM_EINVAL, "K = %d outside [1, 100000]", K);
  if (!h->ws || !h->params_ok || !h->state_ok || h->n_blocks < 1)
    return fail(h, SIM_ESTATE, "bind, parameters, state and commands must be set before stepping");
  cf::StepArgs a;
  a.planes = h->planes;
  a.cmd = h->cmd;
  a.params = h->params_dev;
  a.set_of_world = h->set_of_world_dev;
  a.status = h->status;
  a.tile_ctr = h->status + 1;
  a.n = (int)h->ntot;
  a.N = (int)h->N;
  a.n_blocks = (int)h->n_blocks;
  a.hold = h->hold;
  const int64_t tmax = (h->n_blocks - 1) * (int64_t)h->hold;
  a.t0 = (int)(h->t < tmax ? h->t : tmax);
  a.K = K;
  a.dt = h->dt;
  cudaError_t e =
      h->batched
          ? cf::launch_step_batched(a, h->tiles_dev, (int)h->tiles.size(), h->integrator, h->ctrl,
                                    h->general_motor, (h->p0.flags & cf::PF_ASYM_XY) == 0, h->tpb,
                                    (cudaStream_t)stream)
          : cf::launch_step(a, h->p0, h->model, h->integrator, h->ctrl, h->general_motor,
                            h->per_set, h->tpb, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
  h->launches++;
  h->t += K;
  return SIM_OK;
}

int sim_run(sim_h h, int64_t n_steps, int K, void* stream) {
  if (!h) return SIM_EINVAL;
  if (n_steps < 0 || K < 1) return fail(h, SIM_EINVAL, "need n_steps >= 0 and K >= 1");
  while (n_steps > 0) {
    const int k = (int)(n_steps < K ? n_steps : K);
    const int r = sim_step(h, k, stream);
    if (r != SIM_OK) return r;
    n_steps -= k;
  }
  return SIM_OK;
}

int sim_run_host(sim_h h, const float* x0, const float* cmd, int64_t n_blocks, int hold,
                 int64_t n_steps, int K, float* x_out, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws || !h->params_ok) return fail(h, SIM_ESTATE, "sim_bind and sim_set_params must come first");
  if (n_steps < 0 || K < 1 || K > 100000) return fail(h, SIM_EINVAL, "need n_steps >= 0 and 1 <= K <= 100000");
  // one stream, no copy engine for pinned or device buffers: measured on B300
  // systems whose host-to-device copy engine is several times slower than SM
  // loads over the host link, overlapping command copies with the step kernels
  // (copy engine or a concurrent gather kernel) lost to this sequence
  int r = sim_set_state(h, x0, stream);
  if (r == SIM_OK) r = sim_set_commands(h, cmd, n_blocks, hold, stream);
  if (r == SIM_OK) r = sim_run(h, n_steps, K, stream);
  if (r == SIM_OK) r = sim_get_state(h, x_out, stream);
  return r;
}

int sim_selftest_wait_timeout(sim_h h, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws) return fail(h, SIM_ESTATE, "sim_bind must come first");
  cudaError_t e = cf::launch_wait_selftest(h->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "wait self-test launch");
  h->launches++;
  return SIM_OK;
}

int sim_status(sim_h h, uint32_t* flags, void* stream) {
  if (!h || !flags) return h ? fail(h, SIM_EINVAL, "flags is NULL") : SIM_EINVAL;
  if (!h->ws) return fail(h, SIM_ESTATE, "sim_bind must come first");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t v = 0;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&v, h->status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "reading the status word");
  *flags = v;
  return SIM_OK;
}

// ---------------------------------------------------------------- sampling rollouts

int sim_sample_rollouts(sim_h h, int S, int H, const uint64_t* seed, float sigma,
                        const float* nominal, const float* goals, const float* obstacles,
                        int n_obs, float w_obs, float* cost, void* stream) {
  return cf::sample_launch(h, S, H, seed, sigma, nominal, goals, obstacles, n_obs, w_obs, cost, stream, 0,
                     0.f);
}

int sim_mppi_iteration(sim_h h, const sim_mppi_config* cfg, const uint64_t* seed,
                       const float* goals, const float* obstacles, int n_obs, float* mean,
                       float* plan, float* cost, float* best_cost, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!cfg) return fail(h, SIM_EINVAL, "cfg is NULL");
  const sim_mppi_config c = *cfg;
  if (c.S < 1 || c.H < 1 || c.n_ctrl < 1 || c.n_ctrl > 32 || c.S % c.n_ctrl != 0 ||
      !(c.rho >= 0.f && c.rho < 1.f) || !(c.lambda > 0.f) || !isfinite(c.lambda) ||
      c.n_elite < 1 || c.n_elite > SIM_MAX_ELITES || c.n_elite > c.S / c.n_ctrl)
    return fail(h, SIM_EINVAL,
                "MPPI config: need S %% n_ctrl == 0, 1 <= n_ctrl <= 32, 0 <= rho < 1, lambda > 0, "
                "1 <= n_elite <= min(S / n_ctrl, %d)", SIM_MAX_ELITES);
  const int S_c = c.S / c.n_ctrl;
  if (!cf::mppi_uses_warp_path(S_c, c.n_elite) &&
      (c.n_ctrl > SIM_MPPI_CLUSTER_MAX_CTRL || c.H > SIM_MPPI_CLUSTER_MAX_H ||
       h->ntot * c.n_ctrl >= ((int64_t)1 << 27)))
    return fail(h, SIM_EINVAL,
                "MPPI config: controllers of more than %d samples or %d elites need n_ctrl <= %d, "
                "H <= %d and Ntot n_ctrl < 2^27", SIM_MPPI_WARP_MAX_COSTS, SIM_MPPI_WARP_MAX_ELITES,
                SIM_MPPI_CLUSTER_MAX_CTRL, SIM_MPPI_CLUSTER_MAX_H);
  if (!mean || ((uintptr_t)mean & 15) || !plan || ((uintptr_t)plan & 15) || !best_cost ||
      ((uintptr_t)best_cost & 3))
    return fail(h, SIM_EINVAL, "bad or misaligned MPPI buffer");
  // sampling with per-(drone, controller) means and AR(1) noise
  int r = cf::sample_launch(h, c.S, c.H, seed, c.sigma, mean, goals, obstacles, n_obs, c.w_obs, cost,
                      stream, c.n_ctrl, c.rho);
  if (r != SIM_OK) return r;
  cudaError_t e = cf::launch_mppi_update(cost, mean, plan, best_cost,
                                         (const unsigned long long*)seed, (int)h->ntot, c.S, c.H,
                                         c.n_ctrl, c.n_elite, c.sigma, c.rho, c.lambda,
                                         (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "MPPI update launch");
  h->launches++;
  return SIM_OK;
}


int sim_render_depth(sim_h h, const sim_camera* cam, const float* spheres, int n_spheres,
                     const float* boxes, int n_boxes, float* depth, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!h->ws || !h->state_ok) return fail(h, SIM_ESTATE, "bind and state must be set before rendering");
  bool all_fp = h->batched ? true : h->model == SIM_FIRST_PRINCIPLES;
  for (int32_t m : h->model_of_world) all_fp &= (m == SIM_FIRST_PRINCIPLES);
  if (!all_fp) return fail(h, SIM_EINVAL, "depth rendering needs first-principles drones");
  if (!cam || cam->height < 1 || cam->width < 1 || (int64_t)cam->height * cam->width > (1 << 24) ||
      !(cam->hfov > 0.f && cam->hfov < 3.14159f) || !(cam->vfov > 0.f && cam->vfov < 3.14159f) ||
      !(cam->max_range > 0.f) || !isfinite(cam->max_range))
    return fail(h, SIM_EINVAL, "bad camera");
  if (n_spheres < 0 || n_spheres > SIM_MAX_SPHERES || n_boxes < 0 || n_boxes > SIM_MAX_BOXES ||
      (n_spheres > 0 && !spheres) || (n_boxes > 0 && !boxes))
    return fail(h, SIM_EINVAL, "at most %d spheres and %d boxes", SIM_MAX_SPHERES, SIM_MAX_BOXES);
  for (int i = 0; i < 4 * n_spheres; ++i)
    if (!isfinite(spheres[i])) return fail(h, SIM_EINVAL, "sphere values must be finite");
  for (int i = 0; i < 6 * n_boxes; ++i)
    if (!isfinite(boxes[i])) return fail(h, SIM_EINVAL, "box values must be finite");
  if (!depth || ((uintptr_t)depth & 3)) return fail(h, SIM_EINVAL, "bad depth buffer");
  if (h->ntot > 65535) return fail(h, SIM_EINVAL, "at most 65535 cameras per call");
  cudaError_t e = cf::launch_depth(h->planes, (int)h->ntot, cam->height, cam->width, cam->hfov,
                                   cam->vfov, cam->max_range, spheres, n_spheres, boxes, n_boxes,
                                   depth, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "depth launch");
  h->launches++;
  return SIM_OK;
}

int sim_mppi_select_elites(const float* cost, int64_t rows, int S_c, int n_e, int32_t* idx,
                           float* jmin, void* stream) {
  if (!cost || !idx || rows < 0 || S_c < 1 || n_e < 1 || n_e > SIM_MAX_ELITES ||
      ((uintptr_t)cost & 3) || ((uintptr_t)idx & 3) || ((uintptr_t)jmin & 3) ||
      rows >= ((int64_t)1 << 27))
    return SIM_EINVAL;
  if (rows == 0) return SIM_OK;
  cudaError_t e = cf::launch_elite_select(cost, (long long)rows, S_c, n_e, (int*)idx, jmin,
                                          (cudaStream_t)stream);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_philox_normals(const uint64_t* seed, uint64_t first_id, int64_t n, int step, uint32_t* words,
                       float* normals, void* stream) {
  if (!seed || ((uintptr_t)seed & 7) || n < 0 || step < 0 || (!words && !normals)) return SIM_EINVAL;
  if (n == 0) return SIM_OK;
  cudaError_t e = cf::launch_philox((const unsigned long long*)seed, first_id, n, step, words, normals,
                                    (cudaStream_t)stream);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

// ---------------------------------------------------------------- rollout (BPTT)

static int rollout_check(sim_h h, int H, int C, const void* ws, size_t ws_bytes,
                         std::initializer_list<const void*> dev_ptrs) {
  if (h->batched || h->model != SIM_FIRST_PRINCIPLES || h->integrator != SIM_EULER)
    return fail(h, SIM_EINVAL, "policy rollouts need a uniform first-principles Euler handle");
  if (!h->params_ok) return fail(h, SIM_ESTATE, "sim_set_params must come first");
  if (h->per_set || (h->p0.flags & (cf::PF_DRAG | cf::PF_GENERAL_MOTOR)))
    return fail(h, SIM_EINVAL, "policy rollouts need one parameter set, lag rotors and no drag");
  if (H < 1 || C < 1 || C > H) return fail(h, SIM_EINVAL, "need 1 <= C <= H");
  if (!ws || ((uintptr_t)ws & 255)) return fail(h, SIM_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < cf::rollout_workspace_bytes((int)h->ntot, H, C, h->objective.kind, h->rollout_repeat))
    return fail(h, SIM_ENOMEM, "rollout workspace too small");
  for (const void* p : dev_ptrs)
    if (!p || ((uintptr_t)p & 15)) return fail(h, SIM_EINVAL, "device buffers must be 16-byte aligned");
  return SIM_OK;
}

int sim_rollout_set_objective(sim_h h, const sim_objective* obj) {
  if (!h) return SIM_EINVAL;
  cf::RolloutObjective o;
  if (obj) {
    if (obj->kind != SIM_OBJ_SQUARED && obj->kind != SIM_OBJ_TRACKING_REWARD)
      return fail(h, SIM_EINVAL, "unknown objective kind %d", obj->kind);
    bool ok = isfinite(obj->w_theta) && obj->w_theta >= 0.f;
    for (int i = 0; i < 4; ++i)
      ok = ok && isfinite(obj->w_act[i]) && obj->w_act[i] >= 0.f && isfinite(obj->w_dact[i]) &&
           obj->w_dact[i] >= 0.f;
    if (!ok) return fail(h, SIM_EINVAL, "objective weights must be finite and non-negative");
    o.kind = obj->kind;
    o.w_theta = obj->w_theta;
    for (int i = 0; i < 4; ++i) {
      o.w_act[i] = obj->w_act[i];
      o.w_dact[i] = obj->w_dact[i];
    }
  }
  o.hilo = h->objective.hilo;  // the precision is a separate setting
  h->objective = o;
  return SIM_OK;
}

int sim_rollout_set_precision(sim_h h, int mode) {
  if (!h) return SIM_EINVAL;
  if (mode != SIM_MLP_HILO && mode != SIM_MLP_BF16) return fail(h, SIM_EINVAL, "unknown MLP precision %d", mode);
  h->objective.hilo = mode == SIM_MLP_HILO;
  return SIM_OK;
}

int sim_rollout_workspace_bytes(sim_h h, int H, int C, size_t* bytes) {
  if (!h || !bytes) return SIM_EINVAL;
  if (H < 1 || C < 1 || C > H) return fail(h, SIM_EINVAL, "need 1 <= C <= H");
  *bytes = cf::rollout_workspace_bytes((int)h->ntot, H, C, h->objective.kind, h->rollout_repeat);
  return SIM_OK;
}

int sim_rollout_set_action_repeat(sim_h h, int R) {
  if (!h) return SIM_EINVAL;
  if (R < 1 || R > SIM_MAX_ACTION_REPEAT)
    return fail(h, SIM_EINVAL, "action repeat must lie in [1, %d]", SIM_MAX_ACTION_REPEAT);
  h->rollout_repeat = R;
  return SIM_OK;
}

int sim_rollout_fwd(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                    float w_act, void* ws, size_t ws_bytes, float* loss, void* stream) {
  if (!h) return SIM_EINVAL;
  int r = rollout_check(h, H, C, ws, ws_bytes, {x0, w, p_ref, loss});
  if (r != SIM_OK) return r;
  cudaError_t e = cf::launch_rollout_fwd(x0, w, p_ref, (int)h->ntot, H, C, h->rollout_repeat, h->dt,
                                         w_act, h->objective,
                                         h->p0, ws, loss, true, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout forward launch");
  h->launches += 2;
  return SIM_OK;
}

int sim_rollout_bwd(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                    float w_act, void* ws, size_t ws_bytes, const float* dL, float* dW, float* dx0,
                    void* stream) {
  if (!h) return SIM_EINVAL;
  int r = rollout_check(h, H, C, ws, ws_bytes, {x0, w, p_ref, dL, dW, dx0});
  if (r != SIM_OK) return r;
  cudaError_t e = cf::launch_rollout_bwd(x0, w, p_ref, (int)h->ntot, H, C, h->rollout_repeat, h->dt,
                                         w_act, h->objective,
                                         h->p0, ws, dL, dW, dx0, h->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout backward launch");
  h->launches += 2;
  return SIM_OK;
}

int sim_rollout_grad(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                     float w_act, void* ws, size_t ws_bytes, float* loss, const float* dL_one,
                     float* dW, float* dx0, void* stream) {
  if (!h) return SIM_EINVAL;
  int r = rollout_check(h, H, C, ws, ws_bytes, {x0, w, p_ref, loss, dL_one, dW, dx0});
  if (r != SIM_OK) return r;
  // one adjoint launch whose recompute warps run the forward pass first: the
  // reverse sweep starts as soon as the last segment is stepped
  cudaError_t e = cf::launch_rollout_grad(x0, w, p_ref, (int)h->ntot, H, C, h->rollout_repeat, h->dt,
                                          w_act, h->objective, h->p0, ws, loss, dL_one, dW, dx0,
                                          h->status, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "rollout gradient launch");
  h->launches += 3;
  return SIM_OK;
}

int sim_adam_step(const float* grad, float* w, float* m, float* v, uint16_t* w_bf16, int64_t n,
                  int32_t* step, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!grad || !w || !m || !v || !w_bf16 || !step || n < 1 || n > (1 << 24) ||
      ((uintptr_t)grad & 3) || ((uintptr_t)w & 3) || ((uintptr_t)m & 3) || ((uintptr_t)v & 3) ||
      ((uintptr_t)w_bf16 & 1) || ((uintptr_t)step & 3) || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return SIM_EINVAL;
  cudaError_t e = cf::launch_adam(grad, w, m, v, w_bf16, (int)n, step, lr, beta1, beta2, eps,
                                  (cudaStream_t)stream);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int64_t sim_num_drones(sim_h h) { return h ? h->ntot : -1; }
int64_t sim_step_count(sim_h h) { return h ? h->t : -1; }
int sim_set_step_count(sim_h h, int64_t t) {
  if (!h) return SIM_EINVAL;
  if (t < 0) return fail(h, SIM_EINVAL, "negative step count");
  h->t = t;
  return SIM_OK;
}
int64_t sim_launch_count(sim_h h) { return h ? h->launches : -1; }
const char* sim_last_error(sim_h h) { return h ? h->err : "NULL handle"; }
void sim_destroy(sim_h h) { delete h; }

}  // extern "C"
