// Autotuner of the launch shapes: threads per block and steps per launch of
// the fused step, threads per block of the sampling launch.  Candidates are
// timed with CUDA events on the handle's own data and stream; the fastest is
// applied to the handle and cached under a key that names everything the
// timing depends on: the GPU, the operation, the batch shape and model mix,
// the integrator, the control interface, the rotor model and the run length.
//
// The cache is a file of JSON lines, {"key": ..., "tpb": ..., "K": ..., "ms": ...},
// at $CRAZYFLOW_AUTOTUNE_CACHE or ~/.cache/crazyflow_b300/autotune.jsonl; it is
// read on every cached lookup and appended to after every tuning, so handles
// in one process and runs in later processes share it.  Nothing is allocated
// on the device: the step trials save the state planes in the handle's staging
// region and restore them (and the command schedule) around every run.
#include <errno.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"

namespace {

std::mutex g_file_mu;

int tune_fail(sim_h h, int code, const char* fmt, ...) {
  char buf[400];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  cf::note_error(h, "sim_autotune: %s", buf);
  return code;
}

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

const char* name_of_integrator(int i) { return i == SIM_RK4 ? "rk4" : "euler"; }
const char* name_of_ctrl(int c) {
  switch (c) {
    case SIM_CTRL_ROTOR_SPEED: return "rotor_speed";
    case SIM_CTRL_ATTITUDE: return "attitude";
    case SIM_CTRL_POSITION: return "position";
    default: return "torque";
  }
}

std::string gpu_name() {
  int dev = -1;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
    cudaGetLastError();
    return "no-device";
  }
  char buf[300];
  snprintf(buf, sizeof(buf), "%s sm_%d%d x%d", p.name, p.major, p.minor, p.multiProcessorCount);
  std::string s(buf);
  for (char& c : s)
    if (c == '|' || c == '"' || c == '\\') c = '_';
  return s;
}

bool valid_op(int op) { return op == SIM_TUNE_STEP || op == SIM_TUNE_SAMPLE; }

std::string make_key(const sim_s* h, const sim_tune_request* r) {
  int n_model[3] = {0, 0, 0};
  if (h->batched) {
    for (int32_t m : h->model_of_world)
      if (m >= 0 && m < 3) ++n_model[m];
  } else if (h->model >= 0 && h->model < 3) {
    n_model[h->model] = (int)h->M;
  }
  uint64_t mix = 1469598103934665603ull;
  if (h->batched) {
    mix = fnv1a(mix, h->n_per_world.data(), h->n_per_world.size() * sizeof(int64_t));
    mix = fnv1a(mix, h->model_of_world.data(), h->model_of_world.size() * sizeof(int32_t));
  }
  char buf[512];
  int k = snprintf(buf, sizeof(buf),
                   "%s|op=%s|M=%lld|N=%lld|ntot=%lld|worlds=fp%d,abs%d,absnt%d|mix=%016llx|"
                   "integrator=%s|ctrl=%s|motor=%s|per_set=%d|dt=%.9g",
                   gpu_name().c_str(), r->op == SIM_TUNE_STEP ? "step" : "sample",
                   (long long)h->M, h->batched ? -1ll : (long long)h->N, (long long)h->ntot,
                   n_model[0], n_model[1], n_model[2], (unsigned long long)mix,
                   name_of_integrator(h->integrator), name_of_ctrl(h->ctrl),
                   h->general_motor ? "general"
                   : (h->p0.flags & cf::PF_ASYM_XY) ? "lag"
                                                    : "lag_jxy",  // the Jx = Jy kernel variants
                   h->per_set ? 1 : 0, (double)h->dt);
  if (r->op == SIM_TUNE_STEP)
    snprintf(buf + k, sizeof(buf) - k, "|steps=%lld", (long long)r->n_steps);
  else
    snprintf(buf + k, sizeof(buf) - k, "|S=%d|H=%d|n_obs=%d", r->S, r->H, r->n_obs);
  return std::string(buf);
}

std::string cache_path() {
  const char* e = getenv("CRAZYFLOW_AUTOTUNE_CACHE");
  if (e && *e) return std::string(e);
  const char* home = getenv("HOME");
  return std::string(home && *home ? home : ".") + "/.cache/crazyflow_b300/autotune.jsonl";
}

// Last line of the cache whose key matches (later lines win).
bool cache_lookup(const std::string& key, int* tpb, int* K, float* ms) {
  std::lock_guard<std::mutex> lock(g_file_mu);
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return false;
  const std::string want = "{\"key\": \"" + key + "\",";
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    if (strncmp(line, want.c_str(), want.size()) != 0) continue;
    int t = 0, kk = 0;
    float m = 0.f;
    if (sscanf(line + want.size(), " \"tpb\": %d, \"K\": %d, \"ms\": %g", &t, &kk, &m) == 3) {
      *tpb = t;
      *K = kk;
      *ms = m;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void mkdirs_for(const std::string& path) {
  for (size_t i = 1; i < path.size(); ++i) {
    if (path[i] != '/') continue;
    const std::string d = path.substr(0, i);
    if (mkdir(d.c_str(), 0755) != 0 && errno != EEXIST) return;
  }
}

bool cache_store(const std::string& key, int tpb, int K, float ms) {
  std::lock_guard<std::mutex> lock(g_file_mu);
  const std::string path = cache_path();
  mkdirs_for(path);
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return false;
  fprintf(f, "{\"key\": \"%s\", \"tpb\": %d, \"K\": %d, \"ms\": %.6g}\n", key.c_str(), tpb, K, ms);
  return fclose(f) == 0;
}

// A device-side pause of about 0.2 ms ahead of each timed run, so that the
// host enqueues the run's launches while the GPU is busy and the events time
// device execution rather than host launch latency.
__global__ void pause_kernel() {
  for (int i = 0; i < 200; ++i) __nanosleep(1000);
}

float median(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  const size_t n = v.size();
  return n % 2 ? v[n / 2] : 0.5f * (v[n / 2 - 1] + v[n / 2]);
}

}  // namespace

extern "C" {

int sim_autotune_key(sim_h h, const sim_tune_request* req, char* key, size_t n) {
  if (!h) return SIM_EINVAL;
  if (!req || !key || n == 0 || !valid_op(req->op)) return tune_fail(h, SIM_EINVAL, "bad request");
  const std::string k = make_key(h, req);
  if (k.size() + 1 > n) return tune_fail(h, SIM_EINVAL, "key buffer of %zu bytes is too small", n);
  memcpy(key, k.c_str(), k.size() + 1);
  return SIM_OK;
}

int sim_autotune(sim_h h, const sim_tune_request* req, sim_tune_result* out, void* stream) {
  if (!h) return SIM_EINVAL;
  if (!req || !out || !valid_op(req->op) || req->reps < 1 || req->reps > 100)
    return tune_fail(h, SIM_EINVAL, "need a request with op SIM_TUNE_STEP or SIM_TUNE_SAMPLE, "
                                    "1 <= reps <= 100, and a result");
  const bool step = req->op == SIM_TUNE_STEP;
  // candidates (defaults when none are given)
  static const int def_tpb[] = {32, 64, 128, 256};
  static const int def_K[] = {1, 5, 10, 25, 50, 100, 200};
  std::vector<int> tpbs, Ks;
  if (req->n_tpb < 0 || req->n_tpb > SIM_TUNE_MAX_CANDIDATES || req->n_K < 0 ||
      req->n_K > SIM_TUNE_MAX_CANDIDATES)
    return tune_fail(h, SIM_EINVAL, "at most %d candidates per list", SIM_TUNE_MAX_CANDIDATES);
  if (req->n_tpb == 0) tpbs.assign(def_tpb, def_tpb + 4);
  else tpbs.assign(req->tpb, req->tpb + req->n_tpb);
  for (int t : tpbs)
    if (t < 32 || t > 256 || (t & 31)) return tune_fail(h, SIM_EINVAL, "bad block size %d", t);
  if (step) {
    if (req->n_steps < 1) return tune_fail(h, SIM_EINVAL, "need n_steps >= 1");
    if (req->n_K == 0) Ks.assign(def_K, def_K + 7);
    else Ks.assign(req->K, req->K + req->n_K);
    for (int K : Ks)
      if (K < 1 || K > 100000) return tune_fail(h, SIM_EINVAL, "bad steps per launch %d", K);
    // a K beyond the run is the same run as K = n_steps
    std::vector<int> kept;
    for (int K : Ks)
      if (K <= req->n_steps) kept.push_back(K);
    if (kept.empty()) kept.push_back((int)std::min<int64_t>(req->n_steps, 100000));
    Ks = kept;
    if (!h->ws || !h->params_ok || !h->state_ok || h->n_blocks < 1)
      return tune_fail(h, SIM_ESTATE, "bind, parameters, state and commands must be set first");
  } else {
    Ks.assign(1, 1);
    if (!h->ws || !h->params_ok || !h->state_ok)
      return tune_fail(h, SIM_ESTATE, "bind, parameters and state must be set first");
  }
  memset(out, 0, sizeof(*out));
  const std::string key = make_key(h, req);
  snprintf(out->key, sizeof(out->key), "%s", key.c_str());
  int ctpb = 0, cK = 0;
  float cms = 0.f;
  if (req->use_cache && cache_lookup(key, &ctpb, &cK, &cms) && ctpb >= 32 && ctpb <= 256 &&
      !(ctpb & 31) && cK >= 1) {
    if (step) h->tpb = ctpb;
    else h->tpb_sample = ctpb;
    out->tpb = ctpb;
    out->K = cK;
    out->ms = cms;
    out->from_cache = 1;
    return SIM_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return tune_fail(h, SIM_ECUDA, "cudaEventCreate failed");
  }
  const int64_t t0 = h->t;
  const size_t plane_bytes = (size_t)h->ntot * 5 * sizeof(float4);
  int rc = SIM_OK;
  cudaError_t ce = cudaSuccess;
  if (step) ce = cudaMemcpyAsync(h->staging, h->planes, plane_bytes, cudaMemcpyDeviceToDevice, st);
  const int tpb0 = h->tpb, tpbs0 = h->tpb_sample;
  int best = -1;
  float best_ms = 0.f;
  int n_trials = 0;
  for (size_t i = 0; i < tpbs.size() && rc == SIM_OK && ce == cudaSuccess; ++i) {
    for (size_t j = 0; j < Ks.size() && rc == SIM_OK && ce == cudaSuccess; ++j) {
      if (step) h->tpb = tpbs[i];
      else h->tpb_sample = tpbs[i];
      std::vector<float> times;
      for (int r = 0; r <= req->reps && rc == SIM_OK; ++r) {
        if (step) {
          ce = cudaMemcpyAsync(h->planes, h->staging, plane_bytes, cudaMemcpyDeviceToDevice, st);
          h->t = t0;
          if (ce != cudaSuccess) break;
        }
        pause_kernel<<<1, 1, 0, st>>>();
        ce = cudaEventRecord(e0, st);
        if (ce != cudaSuccess) break;
        rc = step ? sim_run(h, req->n_steps, Ks[j], stream)
                  : cf::sample_launch(h, req->S, req->H, req->seed, req->sigma, req->nominal,
                                      req->goals, req->obstacles, req->n_obs, req->w_obs, req->cost,
                                      stream, 0, 0.f);
        if (rc != SIM_OK) break;
        ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) break;
        if (r > 0) times.push_back(ms);
      }
      if (rc != SIM_OK || ce != cudaSuccess) break;
      const float m = median(times);
      const int idx = (int)(i * SIM_TUNE_MAX_CANDIDATES + j);
      out->trial_ms[idx] = m;
      ++n_trials;
      if (best < 0 || m < best_ms) {
        best = idx;
        best_ms = m;
      }
    }
  }
  // restore the state and the command schedule the trials started from
  if (step) {
    const cudaError_t c2 =
        cudaMemcpyAsync(h->planes, h->staging, plane_bytes, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = c2;
    const cudaError_t c3 = cudaStreamSynchronize(st);
    if (ce == cudaSuccess) ce = c3;
    h->t = t0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SIM_OK || ce != cudaSuccess || best < 0) {
    h->tpb = tpb0;
    h->tpb_sample = tpbs0;
    if (rc != SIM_OK) return rc;  // the failing call recorded its message
    cudaGetLastError();
    return tune_fail(h, SIM_ECUDA, "timing failed: %s", cudaGetErrorString(ce));
  }
  const int bt = tpbs[best / SIM_TUNE_MAX_CANDIDATES], bK = Ks[best % SIM_TUNE_MAX_CANDIDATES];
  h->tpb = step ? bt : tpb0;
  h->tpb_sample = step ? tpbs0 : bt;
  out->tpb = bt;
  out->K = step ? bK : 1;
  out->ms = best_ms;
  out->n_trials = n_trials;
  out->cache_written = cache_store(key, out->tpb, out->K, best_ms) ? 1 : 0;
  return SIM_OK;
}

}  // extern "C"
