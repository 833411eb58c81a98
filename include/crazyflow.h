/*
 * crazyflow.h -- C-ABI of the B300 batched drone physics step.
 *
 * The library advances an M_worlds x N_drones batch of quadrotors through the
 * simulation step of Crazyflow (arXiv 2606.01478, Materials and Methods):
 * controller -> rotor dynamics -> rotor forces/torques -> rigid-body (or
 * abstracted) derivative -> Euler or RK4 integrator, with K steps fused into
 * one kernel launch (the paper fuses its step pipeline and scans it over
 * steps: Architecture section).
 *
 * Conventions shared by every call
 *   - Units: SI, rotor speeds in RPM.  World z up, gravity along -z.  Body x
 *     forward, y left, z up.  Quaternions scalar-last [x, y, z, w] (First
 *     Principles Modeling, after Eqs. 1-4).
 *   - State row (SIM_STATE_DIM = 20 floats per drone):
 *       first-principles: p(3) q(4) v(3) omega_body(3) Omega(4) I(3)
 *         (the paper's x = [p, q, v, omega, Omega], text after Eq. 6, plus the
 *          position-controller integrator I)
 *       abstracted: p(3) Psi(3: roll, pitch, yaw) v(3) Psidot(3) f_sigma(1),
 *         slots 13..19 unused (Abstracted Physics Modeling, state after Eq. 10)
 *   - Command row (SIM_CMD_DIM = 4 floats per drone), by control interface:
 *       SIM_CTRL_ROTOR_SPEED: Omega_cmd (RPM) per rotor
 *       SIM_CTRL_ATTITUDE:    a in [-1,1]^4 = (roll, pitch, yaw, thrust),
 *                             angles a*max_angle, thrust m g (1 + thrust_scale a4)
 *       SIM_CTRL_POSITION:    (x, y, z, yaw) setpoint
 *       SIM_CTRL_TORQUE:      (collective thrust N, body torque x, y, z N m)
 *     (the paper's control interfaces: text after Eq. 6)
 *   - Drone i of world w has global index w*N + i (uniform batches) or
 *     offset[w] + i with offset the exclusive prefix sum of n_per_world.
 *
 * Memory ownership
 *   The caller owns ALL device memory.  sim_workspace_bytes() reports the size
 *   of one device workspace; sim_bind() hands it to the handle, which keeps the
 *   pointer (not a copy) until sim_destroy() or the next sim_bind().  Inside it
 *   live the state (5 float4 planes of length Ntot: plane j holds state slots
 *   4j..4j+3 of every drone), the parameter sets, the command blocks, a staging
 *   area for host transfers and a 4-byte device status word.  The library
 *   itself allocates only the host-side handle (malloc) and never calls
 *   cudaMalloc/cudaFree.
 *
 * Streams and errors
 *   Every call that touches the device is asynchronous on the given stream
 *   (a cudaStream_t passed as void*; NULL = legacy default stream) and
 *   launches nothing when it returns an error.  Argument and call-order errors
 *   return SIM_EINVAL / SIM_ESTATE immediately; a failed CUDA launch or copy
 *   returns SIM_ECUDA.  sim_last_error() gives a message for the last failure
 *   on that handle.  Conditions detected on the device (a non-finite state)
 *   set bits in the device status word, read by sim_status().  No call traps,
 *   asserts on the device or aborts the process.
 */
#ifndef CRAZYFLOW_B300_H
#define CRAZYFLOW_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SIM_OK 0
#define SIM_EINVAL (-1)  /* bad argument (size, enum, NULL, unsupported combination) */
#define SIM_ENOMEM (-2)  /* host allocation of the handle failed / workspace too small */
#define SIM_ECUDA (-3)   /* a CUDA call failed; see sim_last_error */
#define SIM_ESTATE (-4)  /* call order: e.g. sim_step before sim_bind / sim_set_params */

/* device status word bits (sim_status) */
#define SIM_FLAG_NONFINITE 1u /* some drone's state became NaN/Inf after a launch */
#define SIM_FLAG_TIMEOUT 2u   /* a bounded in-kernel wait gave up (that call's results are invalid) */

/* physics models (First Principles Modeling, Eqs. 1-6; Abstracted Physics Modeling, Eqs. 7-10;
 * the abstracted variant without thrust dynamics and drag, last sentence of that section:
 * f_sigma follows f_cmd at once, the drag term is dropped) */
#define SIM_FIRST_PRINCIPLES 0
#define SIM_ABSTRACTED 1
#define SIM_ABSTRACTED_NOTHRUST 2

/* integrators: explicit Euler, classic RK4 (controller output held over the stages) */
#define SIM_EULER 0
#define SIM_RK4 1

/* control interfaces (text after Eq. 6); the abstracted model takes attitude commands only */
#define SIM_CTRL_ROTOR_SPEED 0
#define SIM_CTRL_ATTITUDE 1
#define SIM_CTRL_POSITION 2
#define SIM_CTRL_TORQUE 3

#define SIM_STATE_DIM 20
#define SIM_CMD_DIM 4
#define SIM_NPARAMS 48

/* Per-platform parameter vector (float[SIM_NPARAMS]); indices below.  Per-rotor
 * thrust kf W^2 + kf1 W + kf0 and drag torque km W^2 + km1 W ("second-order
 * polynomials", text before Eq. 5; W in RPM); the rotor model is Eq. 6 with
 * coefficients (cv_up, cd_up) for spin-up and (cv_down, cd_down) for spin-down;
 * J_p (kg m^2) is the rotor + motor inertia of Eq. 5's gyroscopic and reaction
 * torques; C_a is the diagonal of the body-frame linear drag matrix (text after
 * Eq. 5); gains are those of the geometric attitude/position controller;
 * c1..c3 (roll, pitch, yaw), c_tau and c_f are the abstracted-model
 * coefficients of Eqs. 8-10. */
enum sim_param_index {
  SIM_P_MASS = 0, SIM_P_JX, SIM_P_JY, SIM_P_JZ, SIM_P_ARM, SIM_P_KF, SIM_P_KM,
  SIM_P_CV_UP, SIM_P_CD_UP, SIM_P_CV_DOWN, SIM_P_CD_DOWN, SIM_P_OMEGA_MAX,
  SIM_P_CA_X, SIM_P_CA_Y, SIM_P_CA_Z,
  SIM_P_KR_X, SIM_P_KR_Y, SIM_P_KR_Z, SIM_P_KW_X, SIM_P_KW_Y, SIM_P_KW_Z,
  SIM_P_KP_X, SIM_P_KP_Y, SIM_P_KP_Z, SIM_P_KD_X, SIM_P_KD_Y, SIM_P_KD_Z,
  SIM_P_KI_X, SIM_P_KI_Y, SIM_P_KI_Z,
  SIM_P_MAX_ANGLE, SIM_P_THRUST_SCALE, SIM_P_G,
  SIM_P_C1_R, SIM_P_C1_P, SIM_P_C1_Y, SIM_P_C2_R, SIM_P_C2_P, SIM_P_C2_Y,
  SIM_P_C3_R, SIM_P_C3_P, SIM_P_C3_Y, SIM_P_C_TAU, SIM_P_C_F,
  SIM_P_J_P, SIM_P_KF0, SIM_P_KF1, SIM_P_KM1,
  SIM_P_COUNT /* = 48 = SIM_NPARAMS */
};

typedef struct sim_s* sim_h;

/* Create a handle for a uniform batch of M worlds x N drones, one model, one
 * integrator, step dt (s).  Control interface defaults to SIM_CTRL_ATTITUDE.
 * Returns SIM_EINVAL for M, N < 1, M*N > 2^31-1, unknown enums, dt <= 0. */
int sim_create(sim_h* out, int64_t M, int64_t N, int model, int integrator, float dt);

/* Create a handle for uneven / mixed batches: world w holds n_per_world[w]
 * drones of model model_per_world[w] (both host arrays of length M, read
 * during the call only).  Drones are laid out world after world. */
int sim_create_batched(sim_h* out, int64_t M, const int64_t* n_per_world,
                       const int32_t* model_per_world, int integrator, float dt);

/* Select the control interface (SIM_CTRL_*).  SIM_EINVAL if the batch holds
 * abstracted-model drones and ctrl is not SIM_CTRL_ATTITUDE. */
int sim_set_control(sim_h h, int ctrl);

/* Bytes of device workspace needed when up to max_cmd_blocks command blocks
 * will be set (see sim_set_commands).  256-byte alignment required. */
int sim_workspace_bytes(sim_h h, int64_t max_cmd_blocks, size_t* bytes);

/* Give the handle its device workspace (caller-owned device memory, >= the
 * reported size, 256-byte aligned; SIM_EINVAL for host memory).  The device
 * that holds it is the handle's device: make it current for every later call
 * on the handle.  Clears nothing; sim_set_state / sim_set_params /
 * sim_set_commands fill it.  Resets the status word (async on stream). */
int sim_bind(sim_h h, void* workspace, size_t bytes, int64_t max_cmd_blocks, void* stream);

/* Parameter sets: params is a host array [n_sets][SIM_NPARAMS] (floats in the
 * order of enum sim_param_index), set_of_world a host array [M] of indices into
 * it (NULL: every world uses set 0).  Both are read during the call only;
 * derived constants are computed on the host in double precision and copied
 * to the workspace with cudaMemcpyAsync on stream.  1 <= n_sets <= M. */
int sim_set_params(sim_h h, const float* params, int64_t n_sets, const int32_t* set_of_world,
                   void* stream);

/* Load / read the state as rows [Ntot][SIM_STATE_DIM].  x may be device
 * memory or pinned host memory, both read/written in place by the layout
 * kernel (pinned host rows travel over the host link as that kernel's own loads
 * and stores), or pageable host memory (copied through the workspace staging
 * area).  Asynchronous on stream: x must stay valid and unchanged until stream
 * reaches the end of the call's work (for pageable memory CUDA makes the copy
 * synchronous with respect to the host). */
int sim_set_state(sim_h h, const float* x, void* stream);
int sim_get_state(sim_h h, float* x, void* stream);

/* Commands: cmd is [n_blocks][Ntot][SIM_CMD_DIM] (device or pinned host memory,
 * copied into the workspace by a kernel; pageable host memory, by the copy
 * engine).  Asynchronous on stream, as for sim_set_state.  Step s after this call (s = 0, 1, ...) uses
 * block min(s / hold, n_blocks - 1).  1 <= n_blocks <= max_cmd_blocks, hold >= 1. */
int sim_set_commands(sim_h h, const float* cmd, int64_t n_blocks, int hold, void* stream);

/* Advance every drone by K steps in ONE kernel launch (state kept in
 * registers across the K steps).  1 <= K <= 100000.  Consecutive step launches
 * on a stream are chained as programmatically dependent launches (the next is
 * scheduled while the previous one drains); with CRAZYFLOW_SERIAL_LAUNCH=1 in
 * the environment they are plain stream-ordered launches instead (same
 * kernels, same results), for profilers that do not follow the chained form. */
int sim_step(sim_h h, int K, void* stream);

/* Advance n_steps steps as ceil(n_steps / K) launches of at most K steps. */
int sim_run(sim_h h, int64_t n_steps, int K, void* stream);

/* One rollout from host memory to host memory on `stream`: sim_set_state(x0),
 * sim_set_commands(cmd, n_blocks, hold), sim_run(n_steps, K) and
 * sim_get_state(x_out) in one call.  With pinned (or device) buffers no copy
 * engine is involved: the layout kernels read and write the state rows in place
 * and a gather kernel moves the commands, SM loads crossing the host link (on
 * B300 systems measured several times faster host-to-device than the copy
 * engine).  The paper has no counterpart; it serves callers whose states and
 * commands live on the host.
 *   x0, x_out [Ntot][SIM_STATE_DIM] float, cmd [n_blocks][Ntot][4] float:
 *   16-byte aligned, caller-owned, valid and unchanged until `stream` reaches
 *   the end of the call's work (x_out is complete then).
 * Errors as for the four calls it stands for. */
int sim_run_host(sim_h h, const float* x0, const float* cmd, int64_t n_blocks, int hold,
                 int64_t n_steps, int K, float* x_out, void* stream);

/* Threads per block of the step and the sampling launches (default 128;
 * 32..256, multiple of 32). */
int sim_set_block_size(sim_h h, int threads_per_block);

/* ---------------------------------------------------------------------------
 * Autotuner of the launch shapes (the batching plan's autotuner: threads per
 * block and steps per launch of the fused step, threads per block of the
 * sampling launch).  The library times every candidate on the handle's own
 * data with CUDA events on `stream` (after one untimed run, the median of
 * `reps` runs), applies the fastest to the handle (SIM_TUNE_STEP sets the
 * step launches' block size, SIM_TUNE_SAMPLE the sampling launches'), and
 * returns it.  The caller passes the chosen K to sim_run / sim_step.
 * Cache: one JSON line per tuning, {"key", "tpb", "K", "ms"}, appended to
 * $CRAZYFLOW_AUTOTUNE_CACHE (default ~/.cache/crazyflow_b300/autotune.jsonl);
 * with use_cache = 1 a matching key (the last one in the file) is returned
 * without timing.  The key names the GPU (name, compute capability, SM count),
 * the operation, M, N (or -1 for uneven batches), Ntot, the number of worlds of
 * each model and a hash of the per-world drone counts and models, the
 * integrator, the control interface, the rotor model (general, lag, or lag with
 * Jx = Jy in every parameter set: each has kernel variants of its own),
 * per-world parameters, dt, and n_steps (step) or S, H and the obstacle count
 * (sample).
 * Step trials restore the state planes (saved in the handle's staging region)
 * and the command schedule around every run and at the end: the handle's
 * state is the same after the call.  Sampling trials write `cost`.  The call
 * synchronises `stream`; do not call it during stream capture.  Nothing is
 * allocated on the device.  Errors: SIM_EINVAL (bad request), SIM_ESTATE
 * (call order), SIM_ECUDA; on an error the block sizes are left unchanged. */
#define SIM_TUNE_STEP 0
#define SIM_TUNE_SAMPLE 1
#define SIM_TUNE_MAX_CANDIDATES 16
typedef struct {
  int op;        /* SIM_TUNE_STEP or SIM_TUNE_SAMPLE */
  int reps;      /* timed runs per candidate, 1..100 */
  int use_cache; /* 1: a cached result for the same key is returned without timing */
  int n_tpb;     /* candidate block sizes (0: 32, 64, 128, 256) */
  int tpb[SIM_TUNE_MAX_CANDIDATES];
  int n_K;       /* SIM_TUNE_STEP: candidate steps per launch (0: 1, 5, 10, 25, 50, 100, 200;
                    candidates above n_steps are dropped) */
  int K[SIM_TUNE_MAX_CANDIDATES];
  int64_t n_steps; /* SIM_TUNE_STEP: steps of each timed run (sim_run(n_steps, K)) */
  /* SIM_TUNE_SAMPLE: the sim_sample_rollouts call to time (arguments as there) */
  int S, H;
  const uint64_t* seed;
  float sigma;
  const float* nominal;
  const float* goals;
  const float* obstacles;
  int n_obs;
  float w_obs;
  float* cost;
} sim_tune_request;

typedef struct {
  int tpb;           /* chosen block size (applied to the handle) */
  int K;             /* SIM_TUNE_STEP: chosen steps per launch; 1 for SIM_TUNE_SAMPLE */
  float ms;          /* its time (median over reps), or the cached time */
  int from_cache;    /* 1 when the result came from the cache */
  int n_trials;      /* candidates timed */
  int cache_written; /* 1 when the result was appended to the cache file */
  /* median time of candidate (tpb[i], K[j]) at [i * SIM_TUNE_MAX_CANDIDATES + j]
     (0 where not timed) */
  float trial_ms[SIM_TUNE_MAX_CANDIDATES * SIM_TUNE_MAX_CANDIDATES];
  char key[512];     /* the cache key */
} sim_tune_result;

int sim_autotune(sim_h h, const sim_tune_request* req, sim_tune_result* out, void* stream);
/* The cache key sim_autotune would use for this handle and request (no timing,
 * no device work); SIM_EINVAL if key[n] cannot hold it. */
int sim_autotune_key(sim_h h, const sim_tune_request* req, char* key, size_t n);

/* Failure-detection self-test of the library's bounded in-kernel waits (the
 * rollout adjoint's warp hand-off uses them): one small kernel waits on a barrier
 * phase that never completes, gives up after the wait's limit (about a second on
 * B300) and sets SIM_FLAG_TIMEOUT in the handle's status word, as a real
 * hand-off failure would.  Nothing faults, traps or hangs, and the context stays
 * usable.  Read the flag with sim_status.  Errors: SIM_EINVAL (h NULL),
 * SIM_ESTATE (not bound), SIM_ECUDA (launch). */
int sim_selftest_wait_timeout(sim_h h, void* stream);

/* Synchronise stream, read and clear the device status word (SIM_FLAG_*). */
int sim_status(sim_h h, uint32_t* flags, void* stream);

int64_t sim_num_drones(sim_h h);     /* Ntot, or -1 for a NULL handle */
int64_t sim_step_count(sim_h h);     /* steps taken since the last sim_set_commands */
/* Set that step counter (it selects the command block of the next launch), e.g.
 * to undo the advance made while capturing launches into a CUDA graph. */
int sim_set_step_count(sim_h h, int64_t t);
const char* sim_last_error(sim_h h); /* message of the last failure ("" if none) */
void sim_destroy(sim_h h);           /* frees the host handle; the workspace stays the caller's */

/* ---------------------------------------------------------------------------
 * Batched sampling rollouts: the forward model of the paper's MPPI / iCEM
 * sampling controller (Materials and Methods, Model Predictive Path Integral;
 * Results, Control in Cluttered Environments).  Every drone of the handle
 * expands S sampled command sequences over H steps, starting from its current
 * state (the state is read, not modified).  For drone d of world w, sample s,
 * step k = 0 .. H-1:
 *   xi  = 4 standard normals: Philox4x32-10 (Salmon et al., SC'11) with counter
 *         (id mod 2^32, id / 2^32, k, 0), key (seed mod 2^32, seed / 2^32),
 *         id = d*S + s; u = ((word >> 9) + 0.5) 2^-23; Box-Muller on word pairs
 *         (0,1) and (2,3)
 *   a   = clip(nominal[w][k] + sigma xi, -1, 1)   (attitude interface)
 *   x   <- one step of the handle's integrator (first-principles model)
 *   cost[d][s] += |p - goal[w]| + w_obs sum_o max(0, r_o - |p - c_o|)
 * Requires every drone to be first-principles and the attitude interface.
 *   seed      device uint64 (read by the kernel: a captured graph replays with
 *             whatever the device word holds)
 *   nominal   device [M][H][4] float, or NULL for zero (hover)
 *   goals     device [M][3] float
 *   obstacles HOST [n_obs][4] float (centre xyz, radius >= 0), read during the
 *             call and passed by value; 0 <= n_obs <= SIM_MAX_OBSTACLES
 *   cost      device [Ntot][S] float (output)
 * One persistent kernel launch; no scratch memory. */
#define SIM_MAX_OBSTACLES 64
/* The sampling noise on its own: for ids first_id .. first_id + n - 1 at step
 * `step`, writes the four Philox4x32-10 words (device uint32 [n][4], or NULL)
 * and the four normals (device float [n][4], or NULL) exactly as the sampling
 * kernel draws them.  seed: device uint64.  Needs no handle. */
int sim_philox_normals(const uint64_t* seed, uint64_t first_id, int64_t n, int step, uint32_t* words,
                       float* normals, void* stream);
int sim_sample_rollouts(sim_h h, int S, int H, const uint64_t* seed, float sigma,
                        const float* nominal, const float* goals, const float* obstacles,
                        int n_obs, float w_obs, float* cost, void* stream);

/* ---------------------------------------------------------------------------
 * One MPPI / iCEM control iteration (Materials and Methods, Model Predictive
 * Path Integral: parallel controllers, the top fraction of each controller's
 * trajectories as elites, temporally correlated noise, warm start from the
 * previous mean, exponential weighting of the elites, best controller applied).
 * For every drone d of the handle:
 *   sample s (0 <= s < S) belongs to controller c = s / S_c, S_c = S / n_ctrl;
 *   its actions are clip(mean[d][c][k] + sigma eps_k, -1, 1) with the noise of
 *   sim_sample_rollouts made AR(1): eps_0 = xi_0,
 *   eps_k = rho eps_{k-1} + sqrt(1 - rho^2) xi_k
 *   cost[d][s] as in sim_sample_rollouts (goal of the drone's world, obstacles)
 *   elites of controller c: its n_elite lowest costs (ties: lower sample index;
 *   NaN costs never selected).  The paper keeps the top 1 % of each
 *   controller's samples: n_elite = ceil(S_c / 100).
 *   mean'[d][c] = sum_e w_e a_e / sum_e w_e,  w_e = exp(-(J_e - J_min,c) / lambda)
 *   plan[d] = mean'[d][c*], c* = argmin_c J_min,c (ties: lower c);
 *   best_cost[d] = J_min,c*
 *   mean[d][c][k] <- mean'[d][c][k+1] (warm start; the last step repeated)
 * Buffers (device): mean [Ntot][n_ctrl][H][4] float (in/out, 16-byte aligned),
 * plan [Ntot][H][4] float, cost [Ntot][S] float (written), best_cost [Ntot]
 * float; goals, obstacles and seed as for sim_sample_rollouts.
 * Constraints: S % n_ctrl == 0, 1 <= n_ctrl <= 32, 0 <= rho < 1, lambda > 0,
 * 1 <= n_elite <= min(S_c, SIM_MAX_ELITES).  Controllers with more than
 * SIM_MPPI_WARP_MAX_COSTS samples or more than SIM_MPPI_WARP_MAX_ELITES elites
 * take the cluster update (one thread-block cluster of up to 16 blocks per
 * controller -- 16 where the device places clusters of that size, else 8 --
 * the controller's costs split over its blocks), which needs
 * n_ctrl <= SIM_MPPI_CLUSTER_MAX_CTRL, H <= SIM_MPPI_CLUSTER_MAX_H and
 * Ntot n_ctrl < 2^27.  Two launches (sampling, update); no scratch memory. */
#define SIM_MAX_ELITES 4096
#define SIM_MPPI_WARP_MAX_COSTS 2048
#define SIM_MPPI_WARP_MAX_ELITES 32
#define SIM_MPPI_CLUSTER_MAX_CTRL 8
#define SIM_MPPI_CLUSTER_MAX_H 1024
typedef struct {
  int S;            /* samples per drone, all controllers */
  int H;            /* horizon (steps of the handle's dt and integrator) */
  int n_ctrl;       /* parallel controllers per drone */
  int n_elite;      /* elites per controller */
  float sigma;      /* noise scale */
  float rho;        /* AR(1) temporal correlation of the noise */
  float lambda;     /* temperature of the exponential weights */
  float w_obs;      /* obstacle penalty weight */
} sim_mppi_config;

int sim_mppi_iteration(sim_h h, const sim_mppi_config* cfg, const uint64_t* seed,
                       const float* goals, const float* obstacles, int n_obs, float* mean,
                       float* plan, float* cost, float* best_cost, void* stream);

/* The elite selection of sim_mppi_iteration on its own (Materials and Methods,
 * Model Predictive Path Integral: the top fraction of each controller's
 * samples).  cost: device float [rows][S_c]; for every row, the n_e smallest
 * (cost, sample index) pairs in lexicographic order, i.e. ties to the lower
 * index, NaN costs never selected.  idx: device int32 [rows][n_e], the elites'
 * sample indices in increasing index order, -1 in the slots past the row's
 * number of non-NaN costs; jmin: device float [rows] (or NULL), the row's
 * smallest cost (INFINITY if every cost is NaN).  1 <= n_e <= SIM_MAX_ELITES,
 * S_c >= 1, 0 <= rows < 2^27, 4-byte aligned buffers.  One launch, no handle.
 * Returns SIM_EINVAL on bad arguments (nothing launched), SIM_ECUDA if the
 * launch fails. */
int sim_mppi_select_elites(const float* cost, int64_t rows, int S_c, int n_e, int32_t* idx,
                           float* jmin, void* stream);

/* ---------------------------------------------------------------------------
 * Batched depth images by ray casting (the paper's parallel depth rendering,
 * Results, Computation Performance; here as CUDA arithmetic, no graphics API).
 * Every drone of the handle carries a pinhole camera at its centre looking
 * along body +x; pixel (row i, column j) casts the ray
 *   normalise(1, -tan(hfov/2) (2 (j + 0.5) / W - 1), -tan(vfov/2) (2 (i + 0.5) / H - 1))
 * in the body frame, rotated by the drone's current attitude; depth = range to
 * the first hit among the spheres, the axis-aligned boxes and the ground plane
 * z = 0, clipped to max_range.  spheres: HOST [n_spheres][4] (centre, radius);
 * boxes: HOST [n_boxes][6] (min corner, max corner); both read during the call
 * (passed by value).  depth: device [Ntot][height][width] float.  Requires
 * first-principles drones (quaternion attitude).  One launch. */
#define SIM_MAX_SPHERES 64
#define SIM_MAX_BOXES 32
typedef struct {
  int height, width;     /* pixels */
  float hfov, vfov;      /* full fields of view, radians, in (0, pi) */
  float max_range;       /* metres */
} sim_camera;
int sim_render_depth(sim_h h, const sim_camera* cam, const float* spheres, int n_spheres,
                     const float* boxes, int n_boxes, float* depth, void* stream);

/* ---------------------------------------------------------------------------
 * Differentiable policy rollout (backpropagation through time; Materials and
 * Methods, Backpropagation Through Time).  For every drone of the handle,
 * independently:
 *   obs_k = [p_k - r_k, q_k, v_k, omega_k]                         (13)
 *   a_k   = tanh(W3 tanh(W2 tanh(W1 obs_k + b1) + b2) + b3)        (4, attitude action)
 *   x_{k+1} = R Euler steps of the first-principles model under the attitude
 *             interface with command a_k held, k = 0 .. H-1 (R = 1 unless set
 *             by sim_rollout_set_action_repeat; R = 10 runs a 50 Hz policy on
 *             500 Hz physics, the paper's recommended attitude-interface rate)
 *   L = (1/Ntot) sum_drones sum_k |p_{k+1} - r_{k+1}|^2 + w_act |a_k|^2
 * (the squared objective, default) or, after sim_rollout_set_objective with
 * SIM_OBJ_TRACKING_REWARD, the paper's tracking reward (Backpropagation Through
 * Time, reward equation; discount 1) negated as a loss:
 *   L = (1/Ntot) sum_drones sum_k [ -exp(-2 |p_{k+1} - r_{k+1}|) + w_theta theta_{k+1}
 *         + sum_i w_act[i] a_k,i^2 + w_dact[i] (a_k,i - a_{k-1},i)^2 ]
 * with theta the tilt from upright (angle between body z and world z),
 * a_{-1} = 0 = the hover action of the attitude map, and gradient 0 at the
 * kinks of |p - r| and theta.  The w_act argument of the calls below is then
 * unused.
 * Requires a handle created with SIM_FIRST_PRINCIPLES and SIM_EULER, one
 * parameter set with a first-order-lag rotor model (cv_up = cv_down, cd = 0)
 * and zero drag.  The policy MLP runs on tensor cores with bf16 weights and
 * fp32 accumulation.
 *
 * Device buffers (all caller-owned, 16-byte aligned):
 *   x0    [Ntot][SIM_STATE_DIM] float   initial states (slots 17..19 ignored)
 *   w     [SIM_POLICY_NPARAMS] bf16 bit patterns, packed row-major
 *         W1[64][13] b1[64] W2[64][64] b2[64] W3[4][64] b3[4]
 *   p_ref [H+1][Ntot][3] float          reference positions r_k (at policy steps)
 *   ws    rollout workspace of sim_rollout_workspace_bytes(h, H, C) bytes:
 *         checkpoints every C steps, per-drone losses, dW partials and two
 *         segment buffers (the recomputed states and activation cache of the
 *         segment being swept and of the one recomputed beside it), and the
 *         previous actions under the tracking reward: the size depends on the
 *         objective and the action repeat set on the handle; a segment buffer
 *         holds C R + 1 sub-step states
 *   loss  [1] float; dL [1] float (upstream gradient, read on the device);
 *   dW    [SIM_POLICY_NPARAMS] float = dL * dL/dw (in the packed order of w)
 *   dx0   [Ntot][SIM_STATE_DIM] float = dL * dL/dx0 (slots 17..19 = 0)
 * sim_rollout_fwd writes the loss and the checkpoints; sim_rollout_bwd must
 * follow it with the same x0, w, p_ref, H, C, w_act and workspace.  Gradients
 * are deterministic (fixed-order reductions).  1 <= C <= H.
 */
#define SIM_POLICY_NPARAMS 5316
#define SIM_OBJ_SQUARED 0
#define SIM_OBJ_TRACKING_REWARD 1
/* Weights of the tracking reward (the paper's BPTT table: w_theta 0.1,
 * w_act (0.12, 0.12, 0, 0.02), w_dact (1.4, 1.4, 0, 0.8)); action order
 * roll, pitch, yaw, thrust. */
typedef struct sim_objective {
  int kind;            /* SIM_OBJ_SQUARED or SIM_OBJ_TRACKING_REWARD */
  float w_theta;       /* tilt weight */
  float w_act[4];      /* action (distance from hover) weights */
  float w_dact[4];     /* action smoothness weights */
} sim_objective;
/* Objective of every later rollout call on the handle (host-side setting; obj
 * NULL restores SIM_OBJ_SQUARED).  SIM_EINVAL for an unknown kind or a weight
 * that is negative or not finite. */
int sim_rollout_set_objective(sim_h h, const sim_objective* obj);
/* Tensor-core operand precision of the policy MLP in every later rollout call
 * on the handle (host-side setting).  SIM_MLP_HILO (default): activations and
 * adjoints enter the MMAs as hi + lo bf16 pairs (~2^-16 relative; weight
 * gradients as hi*hi + hi*lo + lo*hi), within the 1e-3 gradient bar against
 * FP64.  SIM_MLP_BF16: plain bf16 operands (~2^-8 relative; half the forward
 * and input-adjoint MMAs, a third of the weight-gradient ones), the paper's
 * "BF16 weights, FP32 accumulate" policy taken literally.  Weights are bf16
 * values in both; accumulation is fp32.  SIM_EINVAL for another mode. */
#define SIM_MLP_HILO 0
#define SIM_MLP_BF16 1
int sim_rollout_set_precision(sim_h h, int mode);
/* Physics steps per policy action (R) of every later rollout call on the
 * handle (host-side setting; default 1).  H and C count policy steps, p_ref
 * holds the reference at policy steps, and the loss is evaluated after every
 * R-th physics step.  SIM_EINVAL unless 1 <= R <= SIM_MAX_ACTION_REPEAT. */
#define SIM_MAX_ACTION_REPEAT 100
int sim_rollout_set_action_repeat(sim_h h, int R);
int sim_rollout_workspace_bytes(sim_h h, int H, int C, size_t* bytes);
int sim_rollout_fwd(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                    float w_act, void* ws, size_t ws_bytes, float* loss, void* stream);
int sim_rollout_bwd(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                    float w_act, void* ws, size_t ws_bytes, const float* dL, float* dW, float* dx0,
                    void* stream);
/* Forward and backward in one call with dL = 1 (dL_one: device scalar holding 1.0f).
 * One adjoint launch whose recompute warps run the forward pass first, then the
 * loss and dW reductions: loss, dW and dx0 equal those of sim_rollout_fwd followed
 * by sim_rollout_bwd bit for bit, and the workspace holds the same checkpoints
 * afterwards (sim_rollout_bwd may follow with another dL). */
int sim_rollout_grad(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H, int C,
                     float w_act, void* ws, size_t ws_bytes, float* loss, const float* dL_one,
                     float* dW, float* dx0, void* stream);

/* One Adam step (Kingma & Ba, ICLR 2015) on n parameters, in place -- the
 * optimiser of the BPTT training loop (Materials and Methods, Backpropagation
 * Through Time: rollouts and optimisation fused on the device).  With
 * t = *step + 1 (step: device int32, incremented by the call):
 *   m <- b1 m + (1-b1) g;  v <- b2 v + (1-b2) g^2;
 *   w <- w - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps);  w_bf16 <- bf16_rn(w)
 * grad, w, m, v: device float [n]; w_bf16: device bf16 bits [n] (the weights the
 * next rollout reads).  One single-block launch; 1 <= n <= 2^24. */
int sim_adam_step(const float* grad, float* w, float* m, float* v, uint16_t* w_bf16, int64_t n,
                  int32_t* step, float lr, float beta1, float beta2, float eps, void* stream);

/* sim_rollout_grad without a workspace argument.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory when
 * they need a gradient -- a control loop with a hard deadline (cudaMalloc can
 * synchronise the device and take milliseconds) or a plugin whose host
 * framework owns every device allocation.  It allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call): the scratch lives in a fixed 8 MiB
 * device array inside the library, which every GPU that loads the library holds
 * until the process exits (sim_rollout_noalloc_max_bytes reports the size).
 * Batches whose rollout workspace (sim_rollout_workspace_bytes) exceeds it are
 * rejected with SIM_EINVAL and a message, before anything is launched.
 * The caller still passes inputs and outputs (as for sim_rollout_grad; dL is
 * fixed to 1), on the device that holds the handle's workspace, which must be
 * the current device (SIM_EINVAL otherwise).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it for the life of the process; make that first call
 * before any stream capture.  A device reset (cudaDeviceReset) invalidates the
 * kept addresses: do not call this entry point again in a process that reset
 * a device after its first call there.  All calls share the one array and nothing in it needs
 * to start at zero (every byte a call reads, the same call wrote first), but
 * calls that overlap on the GPU -- on different streams or threads -- race on it
 * and must be serialised by the caller. */
int sim_rollout_grad_noalloc(sim_h h, const float* x0, const uint16_t* w, const float* p_ref, int H,
                             int C, float w_act, float* loss, float* dW, float* dx0, void* stream);
int sim_rollout_noalloc_max_bytes(size_t* bytes);

/* Number of kernel launches issued on this handle since creation (all calls). */
int64_t sim_launch_count(sim_h h);

#ifdef __cplusplus
}
#endif
#endif /* CRAZYFLOW_B300_H */
