/*
 * cvba.h - C ABI of the GB300 sliding-window bundle-adjustment library.
 *
 * The library solves the local sparse bundle adjustment (SBA) problem of cuVSLAM
 * (arXiv 2506.04359, Sec. 2.2 "3D module"):
 *
 *   r_ijk = pi(T^cb_k T^bw_i p^w_j) - o_{j,k}                          (Eq. r^repr)
 *   argmin over T^bw_{1:N}, p^w_{1:M} of  sum_i sum_j sum_k ||r_ijk||^2_Sigma   (Eq. argmin)
 *
 * with keyframe poses T^bw_i (base-from-world), a rig of cameras with fixed
 * camera-from-base extrinsics T^cb_k and pinhole intrinsics, landmarks p^w_j and pixel
 * observations o_{j,k}.  As in Sec. 2.2, the linear system of each Levenberg-Marquardt
 * (LM) step is solved with the Schur complement: poses first (dense Cholesky of the
 * reduced camera system), landmarks afterwards.
 *
 * Readings fixed by this library where the paper is silent: pinhole projection without
 * distortion; Sigma = I (pixels); Huber robust kernel on the per-observation residual
 * norm with IRLS weights; left SE(3) update T <- Exp(xi) T with xi = (rho, phi); Euclidean
 * landmark update; one keyframe fixed (gauge); observations with camera depth <= z_min
 * are invalid; Marquardt scaling D = diag(H) floored at 1e-12 max(diag H); Nielsen's
 * lambda update; exactly `iters` iterations, each one linear solve, accepted or not.
 *
 * Conventions
 *  - Poses are (3 x 4) row-major [R | t] with X_b = R X_w + t (12 doubles each).
 *  - Rig extrinsics T_cb are (3 x 4) row-major [R | t] with X_c = R X_b + t.
 *  - Intrinsics are fx, fy, cx, cy (4 doubles per camera); camera axes x right, y down,
 *    z forward; u = fx X/Z + cx, v = fy Y/Z + cy.
 *  - All host arrays are owned by the caller; setters copy them (host -> device) at the
 *    call, getters copy out into caller-owned arrays.  No pointer is retained.
 *  - Every call returns a status; no C++ exception crosses the ABI.  The message of the
 *    last failure on a context is available from cvba_last_error().
 *  - A context is bound to one CUDA device and one stream; calls on one context must not
 *    overlap in time.  Different contexts are independent.
 */
#ifndef CVBA_H
#define CVBA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cvba_ctx cvba_ctx;

typedef enum {
  CVBA_OK = 0,
  CVBA_ERR_INVALID_ARG = 1,  /* bad size, NULL pointer, unsupported option */
  CVBA_ERR_INDEX = 2,        /* observation index out of range */
  CVBA_ERR_NONFINITE = 3,    /* NaN / Inf in an input array */
  CVBA_ERR_CUDA = 4,         /* a CUDA runtime call failed (message has the detail) */
  CVBA_ERR_OOM = 5,          /* device allocation failed */
  CVBA_ERR_NOT_PD = 6,       /* reserved: a system was not positive definite (solve
                                reports this per iteration in cvba_iter.nonpd instead) */
  CVBA_ERR_TIMEOUT = 7,      /* reserved: a bounded device-side wait gave up (no call of this
                                library waits on the device without a bound today) */
  CVBA_ERR_STATE = 8         /* call out of order (e.g. solve before all setters) */
} cvba_status;

typedef enum {
  CVBA_FP64 = 0,   /* every step in FP64 */
  CVBA_MIXED = 1   /* residuals, Jacobians and Schur products in FP32 with FP64
                      accumulation; RCS Cholesky, refinement and gain ratio in FP64 */
} cvba_precision;

typedef struct {
  int iters;            /* LM iterations to run (>= 0) */
  double huber_delta;   /* Huber threshold in pixels (> 0) */
  double lambda0;       /* initial LM damping (> 0); used when reset_lambda != 0 */
  double z_min;         /* minimum camera depth of a valid observation (metres) */
  int reset_lambda;     /* 1: start from lambda0, nu = 2; 0: continue the context's
                           lambda and nu (after cvba_set_damping or a previous solve) */
  int refine;           /* FP64 iterative-refinement corrections allowed per reduced-camera-
                           system solve (0..8; each is taken only while the residual fails
                           the backward-error test |r| <= |A| |dc| 2^-53 sqrt(n_c), infinity
                           norms); < 0 selects the precision's default: 1 for CVBA_MIXED,
                           0 for CVBA_FP64.  The single-CTA fallback factorisations used for
                           systems too large for a cluster's shared memory do not refine. */
} cvba_opts;

typedef struct {
  double cost0;      /* F = 1/2 sum rho(||r||^2) at the linearisation point */
  double cost1;      /* F at the candidate (NaN if the system was not PD) */
  double lambda;     /* damping used for this iteration's solve */
  double gain;       /* (cost0 - cost1) / pred */
  double pred;       /* predicted reduction L = 1/2 d^T (lambda D d - g) */
  double step_norm;  /* ||delta|| over all free coordinates */
  double rms_px;     /* unweighted RMS reprojection error at the linearisation point */
  int accepted;      /* 1 if the candidate became the new state */
  int nonpd;         /* 1 if a 3x3 landmark block or the RCS was not PD (step rejected) */
  int n_valid;       /* observations with camera depth > z_min */
  int n_inlier;      /* valid observations with ||r|| <= huber_delta */
  double berr;       /* backward error |r|/(|A| |dc| + |b|) of the reduced-camera-system
                        solve before refinement (NaN when refine == 0 or not PD) */
  int refined;       /* refinement corrections applied */
  int reserved;
} cvba_iter;

/* Library / context lifetime ---------------------------------------------------- */

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = a new non-blocking stream owned by the context). */
cvba_status cvba_create(cvba_ctx** out, int device, void* cuda_stream, cvba_precision precision);
void cvba_destroy(cvba_ctx* ctx);
const char* cvba_status_string(cvba_status s);
const char* cvba_last_error(const cvba_ctx* ctx);

/* Problem definition (Sec. 2.2: rig T^cb_k and intrinsics, poses T^bw_i, landmarks
 * p^w_j, observations o_{j,k}) ---------------------------------------------------- */

/* n_cams >= 1 cameras: intr[n_cams*4] (fx, fy, cx, cy), T_cb[n_cams*12], and optionally
 * each camera's image width and height wh[n_cams*2] (> 0; NULL = not given).  The image size
 * plays no part in the objective (an observation outside its image is still a residual; the
 * paper's Eq. r^repr has no bounds), so the solve does not use it: it is kept with the rig
 * and returned by cvba_get_rig. */
cvba_status cvba_set_rig(cvba_ctx* ctx, int n_cams, const double* intr, const double* T_cb, const int32_t* wh);

/* The rig as set: intr[n_cams*4], T_cb[n_cams*12], wh[n_cams*2] (zeros when not given).
 * Any pointer may be NULL. */
cvba_status cvba_get_rig(cvba_ctx* ctx, double* intr, double* T_cb, int32_t* wh);

/* n_kf >= 2 keyframe poses T_bw[n_kf*12]; keyframe `fixed_kf` is held constant.  Once a
 * layout exists (cvba_set_observations), the poses of the current state are replaced and the
 * landmarks keep their current values. */
cvba_status cvba_set_poses(cvba_ctx* ctx, int n_kf, const double* T_bw, int fixed_kf);

/* n_lm >= 1 landmarks p_w[n_lm*3] in world coordinates.  Once a layout exists, the
 * landmarks of the current state are replaced and the poses keep their current values. */
cvba_status cvba_set_landmarks(cvba_ctx* ctx, int n_lm, const double* p_w);

/* n_obs observations: keyframe kf[n], camera cam[n], landmark lm[n] and pixel uv[2n..2n+1].
 * Indices are validated (CVBA_ERR_INDEX); every landmark needs >= 2 observations and every
 * keyframe except the fixed one >= 1 (otherwise its columns of the normal equations are
 * zero and no damping makes the system well posed): CVBA_ERR_INVALID_ARG.  Must follow
 * set_rig, set_poses and set_landmarks.
 * This call builds the device layout: observations sorted by (landmark, keyframe,
 * camera), landmarks reordered by keyframe span, and the solve's work tiles. */
cvba_status cvba_set_observations(cvba_ctx* ctx, int n_obs, const int32_t* kf, const int32_t* cam,
                                  const int32_t* lm, const double* uv);

/* Solve ---------------------------------------------------------------------------- */

/* Run opts->iters LM iterations from the current state.  trace (caller-owned,
 * opts->iters entries, may be NULL) receives one record per iteration.  The whole solve
 * runs on the device; the host waits once at the end. */
cvba_status cvba_solve(cvba_ctx* ctx, const cvba_opts* opts, cvba_iter* trace);

/* Cost, counts and RMS at the current state (cost = 1/2 sum rho). */
cvba_status cvba_evaluate(cvba_ctx* ctx, double huber_delta, double z_min, double* cost,
                          double* rms_px, int* n_valid, int* n_inlier);

/* Results and state ------------------------------------------------------------------ */

cvba_status cvba_get_poses(cvba_ctx* ctx, double* T_bw /* n_kf*12 */);
cvba_status cvba_get_landmarks(cvba_ctx* ctx, double* p_w /* n_lm*3, caller's order */);

/* Increment solved in the last iteration, accepted or not: the free keyframes' twists in
 * keyframe order (6 each, fixed keyframe skipped), then landmark steps in the caller's
 * landmark order (3 each).  dx[6*(n_kf-1) + 3*n_lm]. */
cvba_status cvba_get_increment(cvba_ctx* ctx, double* dx);

/* Current LM damping state (lambda, nu) and its replacement. */
cvba_status cvba_get_damping(cvba_ctx* ctx, double* lambda, double* nu);
cvba_status cvba_set_damping(cvba_ctx* ctx, double lambda, double nu);

/* Checkpoint of the solve state: everything a later solve depends on besides the problem
 * itself, i.e. the current poses, the landmarks (caller order) and the LM damping (lambda,
 * nu), in an opaque, versioned byte buffer (a fixed header with the window's sizes, then
 * FP64 values).  With buf == NULL, cvba_get_state only writes the size needed to *bytes;
 * otherwise *bytes must be at least that size (CVBA_ERR_INVALID_ARG) and receives it.
 * cvba_set_state restores a buffer into a context holding the same problem (same keyframe,
 * landmark and observation counts and fixed keyframe: CVBA_ERR_INVALID_ARG otherwise).
 * Resuming is exact: on the FP64 path, a solve of N iterations gives bit-identical results
 * to a solve of k iterations, a checkpoint, a restore (into this or another context with the
 * same problem) and a solve of N - k iterations with reset_lambda = 0.  Requires a layout
 * (CVBA_ERR_STATE). */
cvba_status cvba_get_state(cvba_ctx* ctx, void* buf, size_t* bytes);
cvba_status cvba_set_state(cvba_ctx* ctx, const void* buf, size_t bytes);

/* Device layout, for exact integer checks: lm_order[n_lm] = caller landmark index of each
 * internal landmark; obs_order[n_obs] = caller observation index of each internal slot;
 * lm_off[n_lm+1] = internal landmark segment offsets into the slots.  Any may be NULL. */
cvba_status cvba_get_layout(cvba_ctx* ctx, int32_t* lm_order, int32_t* obs_order, int32_t* lm_off);

/* Sizes: n_kf, n_cams, n_lm, n_obs, n_pairs ((landmark, keyframe) pairs). Any may be NULL. */
cvba_status cvba_get_sizes(cvba_ctx* ctx, int* n_kf, int* n_cams, int* n_lm, int* n_obs, int* n_pairs);

/* Number of kernel launches one solve of `iters` iterations issues (graph nodes that
 * are kernels of this library). */
cvba_status cvba_solve_launch_count(cvba_ctx* ctx, int iters, int* n_launches);

/* Asynchronous solve: enqueue the solve on the context's stream and return without
 * waiting.  The iteration records stay on the device until cvba_get_trace. */
cvba_status cvba_solve_async(cvba_ctx* ctx, const cvba_opts* opts);

/* Copy the first n iteration records of the last solve (waits for the stream). */
cvba_status cvba_get_trace(cvba_ctx* ctx, cvba_iter* trace, int n);

/* Device-pointer variants (e.g. torch tensors' data_ptr()): same layouts as the host
 * setters / getters, copied on the context's stream without a host synchronisation.
 * Require a layout (cvba_set_observations).  The caller keeps the arrays alive until the
 * stream has consumed them. */
cvba_status cvba_set_poses_dev(cvba_ctx* ctx, const double* T_bw /* device, n_kf*12 */);
cvba_status cvba_set_landmarks_dev(cvba_ctx* ctx, const double* p_w /* device, n_lm*3 */);
cvba_status cvba_get_poses_dev(cvba_ctx* ctx, double* T_bw /* device, n_kf*12 */);
cvba_status cvba_get_landmarks_dev(cvba_ctx* ctx, double* p_w /* device, n_lm*3 */);

/* Profiling: run `reps` one-iteration solves from the current state (each relinearises;
 * opts->reset_lambda as given) with CUDA events around each kernel of the iteration (part
 * names: cvba_profile_names(), comma separated) and return the mean milliseconds per part
 * in ms[*n_parts].  With ms == NULL only *n_parts is set.  The state advances as the
 * accepted steps of those solves take it. */
cvba_status cvba_profile_iteration(cvba_ctx* ctx, const cvba_opts* opts, int reps, float* ms, int* n_parts);
const char* cvba_profile_names(void);

/* Batched windows (independent BA problems) ---------------------------------------------
 *
 * Solves many independent windows together (the batched form of the hot path): every
 * phase of an LM iteration is one kernel launch over all windows' work tiles, the
 * reduced-system Cholesky runs one thread-block cluster per window, and the whole
 * multi-iteration solve is one CUDA graph.  Windows keep their own state, damping and
 * iteration records (each is an ordinary context, created with the same device and
 * precision; the batch uses the first context's stream).  A batch holds no copy of the
 * windows' data: a window whose observations are replaced is re-planned on the next
 * solve. */
typedef struct cvba_batch cvba_batch;
cvba_status cvba_batch_create(cvba_batch** out, int n_win, cvba_ctx* const* ctxs);
void cvba_batch_destroy(cvba_batch* batch);
const char* cvba_batch_last_error(const cvba_batch* batch);

/* opts->iters LM iterations in every window; traces (may be NULL) receives n_win * iters
 * records, window-major.  The async form only enqueues (records stay on the device). */
cvba_status cvba_batch_solve(cvba_batch* batch, const cvba_opts* opts, cvba_iter* traces);
cvba_status cvba_batch_solve_async(cvba_batch* batch, const cvba_opts* opts);
cvba_status cvba_batch_launch_count(cvba_batch* batch, const cvba_opts* opts, int* n_launches);

/* Tuning.  cvba_set_tuning re-plans one window's tiles (pairs per linearisation tile,
 * landmarks per Schur tile; 0 = size-based default) keeping its state.
 * cvba_batch_set_chol_cluster picks the CTAs per window of the batched Cholesky (2, 4, 8
 * or 16).  cvba_batch_autotune times short batched solves over a grid of these sizes
 * (pairs per linearisation tile 32, 64, 128, 256; landmarks per Schur tile 8 to 128; cluster
 * sizes 2 to 16), keeps the fastest, restores every window's state and reports the choice.
 * Choices are cached per device (name, SM count, compute capability) and batch
 * configuration (precision and every window's keyframe, camera, landmark, observation and
 * pair counts) for the life of the process: a later call for the same configuration applies
 * the cached choice without timing.  cvba_batch_autotune_clear empties the cache. */
cvba_status cvba_set_tuning(cvba_ctx* ctx, int lin_tile_pairs, int schur_tile_landmarks);
/* How the reduced camera system is factored (re-plans the window, keeping its state):
 * 0 = by size (the default): systems of 320 rows or more take the blocked form, smaller ones
 *     the cluster form;
 * 1 = cluster form: one thread-block cluster factors A = L L^T in shared memory, 8-row
 *     block steps, with the forward substitution fused;
 * 2 = blocked form: right-looking by 32-column panels, the diagonal block of each panel
 *     factored by one CTA and the panel solve and trailing update spread over the GPU (the
 *     factor and y = L^-1 b in global memory); the cluster then runs the backward
 *     substitution, the refinement and the candidate step from the factor.
 * Both compute the FP64 Cholesky factorisation of the same damped reduced camera system
 * (the pose system left by the Schur complement of Sec. 2.2) and differ in rounding order
 * only.  Windows in a batch always use the cluster form.  CVBA_ERR_INVALID_ARG for another
 * mode. */
cvba_status cvba_set_chol_mode(cvba_ctx* ctx, int mode);
cvba_status cvba_batch_set_chol_cluster(cvba_batch* batch, int cluster_size);
cvba_status cvba_batch_autotune(cvba_batch* batch, const cvba_opts* opts, int* lin_tile_pairs,
                                int* schur_tile_landmarks, int* cluster_size);
void cvba_batch_autotune_clear(void);

/* Differentiable cost -------------------------------------------------------------------
 *
 * The robust objective of Sec. 2.2 (Eq. r^repr summed with the Huber kernel) as a
 * differentiable function of the keyframe poses, landmarks and intrinsics, for training
 * and analysis loops (the binding wraps it as a torch.autograd.Function).  Context-free:
 * every array is a caller-owned DEVICE array in the caller's order, all floating arrays of
 * one type: dtype 0 = FP64, 1 = FP32 (the arithmetic runs in that type; the keyframe
 * exponentials in FP64).  Arrays: intr[C*4], T_cb[C*12], xi[K*6] (left tangent
 * perturbation, translation first), T_bw[K*12], p_w[M*3], kf/cam/lm[N] (int32), uv[N*2].
 * Keyframe i is evaluated at Exp(xi_i) T_bw_i.  Observations with an index out of range
 * or camera depth <= z_min contribute nothing.  Limits: K <= 256, C <= 64.
 *
 * `work` is a caller-allocated device workspace of at least
 * cvba_cost_workspace_bytes(N, K, C) bytes (per-block partial sums).  Both calls are
 * asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream). */
size_t cvba_cost_workspace_bytes(int n_obs, int n_kf, int n_cams);

/* cost[0] = 1/2 sum_n rho(|r_n|^2) (device scalar of the dtype). */
cvba_status cvba_cost_forward(int dtype, int n_obs, int n_kf, int n_cams, int n_lm, const void* intr,
                              const void* T_cb, const void* xi, const void* T_bw, const void* p_w,
                              const int32_t* kf, const int32_t* cam, const int32_t* lm, const void* uv,
                              double huber_delta, double z_min, void* cost, void* work, size_t work_bytes,
                              void* stream);

/* Adjoint: with g = grad_cost[0] (device scalar), writes g dF/dxi (K*6, through the left
 * Jacobian of SE(3)), g dF/dT_bw (K*12), g dF/dp_w (M*3) and g dF/dintr (C*4); any output
 * may be NULL.  Jacobians are recomputed, not stored by the forward call. */
cvba_status cvba_cost_backward(int dtype, int n_obs, int n_kf, int n_cams, int n_lm, const void* intr,
                               const void* T_cb, const void* xi, const void* T_bw, const void* p_w,
                               const int32_t* kf, const int32_t* cam, const int32_t* lm, const void* uv,
                               double huber_delta, double z_min, const void* grad_cost, void* g_xi,
                               void* g_T_bw, void* g_p_w, void* g_intr, void* work, size_t work_bytes,
                               void* stream);

/* Motion-only bundle adjustment (multi-camera PnP) ---------------------------------------
 *
 * The pose of a tracked frame from its observations of map landmarks (Sec. 2.2.1 stereo,
 * Eq. PnP over k in [1, 2]; Sec. 2.2.2 multi-stereo, the same sum over every camera k of
 * the rig):  T^bw = argmin sum_j sum_k rho(|pi(T^cb_k T^bw p^w_j) - o_{j,k}|^2)  over the one
 * base pose, the landmarks p^w_j held fixed.  Same readings as the window solve: Huber IRLS
 * weights at the linearisation point, left SE(3) update, Marquardt diagonal floored at
 * 1e-12 max, Nielsen's damping update, accept iff the predicted reduction and the gain are
 * positive, exactly opts->iters iterations (opts->reset_lambda and opts->refine are
 * ignored: every frame starts from opts->lambda0, nu = 2).
 *
 * Many independent frames are solved in one launch (one thread block per frame, every
 * iteration inside it).  Context-free; DEVICE arrays in the caller's order:
 *   intr[n_cams*4], T_cb[n_cams*12], p_w[n_lm*3] and uv[n_obs*2] of type dtype
 *     (0 = FP64: all arithmetic in FP64; 1 = FP32 inputs, per-observation arithmetic in FP32
 *     with two-float block sums, the 6 x 6 solve, the pose and the decision in FP64),
 *   frame_off[n_frames+1] (int32): frame f owns observations [frame_off[f], frame_off[f+1]),
 *     non-decreasing from 0 to n_obs (read back to the host and checked:
 *     CVBA_ERR_INVALID_ARG; the call therefore waits for the stream to reach it),
 *   cam[n_obs], lm[n_obs] (int32): an observation with an index out of range is skipped and
 *     counted in n_bad_index,
 *   T_bw[n_frames*12] (FP64, in: initial poses, out: solved poses),
 *   trace (may be NULL): n_frames * opts->iters records, frame-major.
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream) after the check.
 * n_cams <= 64. */
/* One iteration of a small LM solve (one frame's pose, one landmark, ...): the fields of
 * cvba_iter for that solve, plus the count of its observations skipped for an index out of
 * range. */
typedef struct {
  double cost0, cost1, lambda, gain, pred, step_norm, rms_px;   /* as in cvba_iter */
  int accepted, nonpd, n_valid, n_inlier;
  int n_bad_index;   /* observations of the solve skipped for an index out of range */
  int reserved;
} cvba_lm_record;

cvba_status cvba_pnp_solve(int dtype, int n_frames, int n_cams, int n_lm, int n_obs, const void* intr,
                           const void* T_cb, const void* p_w, const int32_t* frame_off, const int32_t* cam,
                           const int32_t* lm, const void* uv, double* T_bw, const cvba_opts* opts,
                           cvba_lm_record* trace, void* stream);

/* Loop-closure relative pose (Sec. 2.3, relative pose estimation): for each query frame,
 * T^bm = argmin sum_j sum_k rho(|pi(T^cb_k T^bm T^mw p^w_j) - o_{j,k}|^2) with the map pose
 * T^mw (world to map frame) fixed: the landmarks are shifted into the map frame and the
 * pose is solved exactly as by cvba_pnp_solve.  Arguments as cvba_pnp_solve, plus
 * T_mw[n_frames*12] (DEVICE, FP64, [R | t] row-major, one per frame; NULL is
 * CVBA_ERR_INVALID_ARG) and T_bm[n_frames*12] (in: initial relative poses, out: solved). */
cvba_status cvba_relpose_solve(int dtype, int n_frames, int n_cams, int n_lm, int n_obs, const void* intr,
                               const void* T_cb, const void* p_w, const int32_t* frame_off, const int32_t* cam,
                               const int32_t* lm, const void* uv, const double* T_mw, double* T_bm,
                               const cvba_opts* opts, cvba_lm_record* trace, void* stream);

/* Kernel launches of one cvba_pnp_solve or cvba_relpose_solve call (1). */
int cvba_pnp_kernels_per_solve(void);

/* Pose-graph optimisation ----------------------------------------------------------------
 *
 * Sec. 2.3, Eq. PGO: T_{1:N} = argmin sum_{(i,j) in E} |Log(D_ij^-1 T_i^-1 T_j)|^2 over the
 * keyframe poses, from the pose deltas D_ij of odometry and loop-closure edges.  Readings:
 * T_i are WORLD-FROM-BASE poses (T_i^-1 T_j is pose j seen from i, what D_ij measures; the
 * inverse of the window solve's T^bw); Log is the SE(3) logarithm with the twist (rho, phi),
 * translation first; the norm is plain (no weights, no robust kernel); pose `fixed` is held
 * (gauge); left updates T_i <- Exp(xi_i) T_i; LM as the window solve (Marquardt diagonal
 * floored at 1e-12 max, Nielsen's update, accept iff L > 0 and gain > 0, opts->iters
 * iterations; huber_delta, z_min, reset_lambda and refine are ignored).  FP64 throughout; the
 * normal equations are factored densely (6 (n_poses - 1) unknowns).
 * DEVICE arrays: edges[n_edges*2] (int32 i, j: distinct, in range: CVBA_ERR_INDEX),
 * deltas[n_edges*12] ([R | t] row-major), poses[n_poses*12] (in: initial, out: solved),
 * trace (opts->iters records or NULL; n_valid = n_edges, rms_px = sqrt(2 F / n_edges)), and a
 * caller-allocated workspace `work` (256-byte aligned) of at least
 * cvba_pgo_workspace_bytes(n_poses, n_edges) bytes.  The edge list is read back to the host
 * (every free pose needs an edge: CVBA_ERR_INVALID_ARG), so the call waits for the stream to
 * reach it; the solve itself is then asynchronous on `stream`. */
size_t cvba_pgo_workspace_bytes(int n_poses, int n_edges);
cvba_status cvba_pgo_solve(int n_poses, int n_edges, const int32_t* edges, const double* deltas, double* poses,
                           int fixed, const cvba_opts* opts, cvba_lm_record* trace, void* work, size_t work_bytes,
                           void* stream);

/* Multi-view landmark triangulation ------------------------------------------------------
 *
 * The new landmarks of a keyframe from their multi-view observations, the keyframe poses and
 * the rig held fixed (Sec. 2.2 "3D module": triangulation on keyframe creation, whose output
 * the bundle adjustment refines).  The paper names the step without a method; this library
 * computes, for each landmark j:
 *   1. the linear point: with x = ((u - cx)/fx, (v - cy)/fy) and [R | t] = T^cb_k T^bw_i,
 *      the least-squares solution of x (R_3 p + t_3) = R_1 p + t_1, y (R_3 p + t_3) = R_2 p + t_2
 *      over its observations (inhomogeneous DLT), in FP64 (normal equations with one step of
 *      iterative refinement);
 *   2. opts->iters LM iterations on the point alone: the window solve's step restricted to
 *      one landmark (Huber IRLS weights, Marquardt diagonal, Nielsen's update, accept iff the
 *      predicted reduction and the gain are positive).
 * Context-free; DEVICE arrays: intr[n_cams*4], T_cb[n_cams*12], uv[n_obs*2] of type dtype
 * (0 = FP64; 1 = FP32: the refinement's per-observation arithmetic in FP32, the linear step,
 * the 3 x 3 solves, the point and the decisions in FP64), T_bw[n_kf*12] (FP64),
 * lm_off[n_lm+1] (int32; landmark j owns observations [lm_off[j], lm_off[j+1]), checked on the
 * host as for cvba_pnp_solve), kf[n_obs], cam[n_obs] (int32; out-of-range observations are
 * skipped and counted in the records).  Outputs: p_w[n_lm*3] (FP64; NaN where status != 0),
 * p_lin[n_lm*3] (the linear points, may be NULL), status[n_lm] (may be NULL: 0 = solved,
 * 1 = fewer than 2 usable observations, 2 = the linear system is rank deficient, a pivot of
 * its normal equations below 1e-14 of their largest diagonal entry) and trace
 * (n_lm * opts->iters records, landmark-major, written for status 0 only; may be NULL).
 * n_kf <= 256, n_cams <= 64.  Asynchronous on `stream` after the check. */
cvba_status cvba_triangulate(int dtype, int n_lm, int n_kf, int n_cams, int n_obs, const void* intr,
                             const void* T_cb, const double* T_bw, const int32_t* lm_off, const int32_t* kf,
                             const int32_t* cam, const void* uv, const cvba_opts* opts, double* p_lin, double* p_w,
                             int32_t* status, cvba_lm_record* trace, void* stream);

/* Allocation-free evaluation ----------------------------------------------------------
 *
 * The paper has no counterpart to this call; it exists for callers that cannot allocate
 * device memory while running (a tracking thread whose GPU memory is fixed at start-up,
 * where an allocation could block or fail and may be forbidden after initialisation, or
 * a program whose GPU memory belongs to another allocator).  Such callers cannot create a
 * cvba_ctx, so this call needs none.
 *
 * Computes, on the calling thread's current device and on `stream` (a cudaStream_t;
 * NULL = the legacy default stream), the same quantities as cvba_evaluate for a window
 * given as plain DEVICE arrays in the caller's layouts and order: intr[n_cams*4],
 * T_cb[n_cams*12], T_bw[n_kf*12], p_w[n_lm*3], kf/cam/lm[n_obs] (int32), uv[n_obs*2].
 * Writes out[5] (device doubles): cost = 1/2 sum rho(|r|^2) over valid observations,
 * sum |r|^2, n_valid, n_inlier, and the number of observations skipped because an index
 * was out of range.  The call is asynchronous: out is ready when the stream reaches it.
 *
 * It allocates nothing on the device while running: its scratch (per-block partial sums)
 * is a fixed 640 KB device array inside the library's device module.  With lazy module
 * loading (the CUDA default) that module, and the array with it, is loaded onto a device
 * by the first call there, so the FIRST call on each device may allocate: make it during
 * initialisation, before any stream capture (CUDA_MODULE_LOADING=EAGER loads it with the
 * context instead).  The array stays until the context is destroyed.  Its device address
 * is looked up on every call, so a module reloaded after a device reset is found again.
 * n_obs is limited to 4,194,304 (CVBA_ERR_INVALID_ARG beyond), as are a huber_delta that
 * is not a finite positive number, a non-finite z_min and NULL pointers.  If the calling
 * thread already has a CUDA error pending, the call launches nothing, leaves that error
 * pending and returns CVBA_ERR_CUDA.  All calls on a device share the array: calls whose
 * kernels overlap on the GPU race on it and must be serialised by the caller. */
cvba_status cvba_evaluate_noalloc(int n_obs, int n_kf, int n_cams, int n_lm, const double* intr,
                                  const double* T_cb, const double* T_bw, const double* p_w,
                                  const int32_t* kf, const int32_t* cam, const int32_t* lm,
                                  const double* uv, double huber_delta, double z_min, double* out,
                                  void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CVBA_H */
