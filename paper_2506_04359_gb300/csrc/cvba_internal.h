// Internal definitions shared by the host layer (cvba_host.cpp) and the CUDA kernels
// (cvba_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/cvba.h"

namespace cvba {

constexpr int RIG_STRIDE = 16;      // fx fy cx cy | R_cb (9, row-major) | t_cb (3)
constexpr int POSE_STRIDE = 12;     // R (9, row-major) | t (3)
constexpr int PAIR_LIN = 9;         // per (landmark, keyframe) pair: M3 (6 sym) | X_b (3)
constexpr int VINV_STRIDE = 8;      // per landmark: V^-1 (6 sym) | tau | unused
constexpr int K_MAX = 256;          // keyframes per window (sliding-window sizes)
constexpr int C_MAX = 64;           // cameras per rig
constexpr int LIN_THREADS = 256;
constexpr int SCHUR_THREADS = 256;
constexpr int CHOL_THREADS = 1024;
constexpr int DECIDE_THREADS = 256;
constexpr int KDECIDE_THREADS = 1024;  // k_decide: many loads in flight over the tile partials
constexpr int LIN_TILE_PAIRS = 256;     // pairs per linearisation / back-substitution tile
constexpr int LIN_TILE_LMS = 256;       // landmarks per linearisation tile
constexpr int LIN_TILE_OBS = 1024;      // observations a tile stages in shared memory (more: read in place)
constexpr int SCHUR_TILE_PAIRS = 256;   // pairs staged in shared memory per Schur tile
constexpr int SCHUR_TILE_LMS = 128;
constexpr int SPAN_MAX = 22;            // free keyframes in one Schur tile's window (<= 253 blocks)
constexpr int kCholBlockedMinN = 320;   // RCS size from which the blocked factorisation runs (mode 0)
constexpr int kMaxPanels = (6 * (K_MAX - 1) + 31) / 32;   // 32-column panels of the largest system

// Host threads (cvba_layout.cpp): fn(t) for t in [0, n) on n threads; fn(begin, end, thread)
// over [0, n) split in contiguous ranges over up to `threads` threads (one thread per 4096
// items at most); parallel_ranges splits [0, n) over up to all host threads whatever n is,
// for loops whose items are each large (tiles of many pairs).
int host_threads();
void parallel_tasks(int n, const std::function<void(int)>& fn);
void parallel_for(int64_t n, int threads, const std::function<void(int64_t, int64_t, int)>& fn);
void parallel_ranges(int64_t n, const std::function<void(int64_t, int64_t, int)>& fn);

// Host part of a window's layout (cvba_layout.cpp): landmark order and rank, observation
// slots (caller index per slot, camera per slot), landmark slot offsets, and the (landmark,
// keyframe) pairs with their slot offsets and the landmarks' pair offsets.
struct HostLayout {
  std::vector<int32_t> lm_order, lm_rank, obs_order, lm_off, obs_cam;
  std::vector<int32_t> pair_kf, pair_lm, pair_obs, lm_pair;
  // work arrays, kept for the next layout of the same context
  std::vector<uint64_t> rec_key, grp;
  std::vector<int64_t> goff;
  std::vector<int32_t> first, last, npair_of, by_first;
};
// False (with a message) if a landmark has fewer than 2 observations or a free keyframe has
// none.  Indices must be valid.
bool compute_host_layout(int K, int C, int M, int N, int fixed_kf, const int32_t* kf, const int32_t* cam,
                         const int32_t* lm, HostLayout& L, std::string& err);

// Device-resident LM control block.  Written only by the solve's kernels.
struct Ctrl {
  int cur;            // state buffer (0/1) holding the current iterate x
  int need_lin;       // 1: the linearisation buffers must be rebuilt at x
  int it;             // iterations done in this solve
  int nonpd;          // set when a landmark block or the RCS is not positive definite
  int iters;          // iterations requested (trace capacity)
  int pad_;
  double lam, nu;     // LM damping state
  double huber, zmin; // solve options
  double pred_part[16];   // pose part of d^T (lam D d - g), one partial per Cholesky CTA
  double step2_part[16];  // ||dc||^2, likewise
  int n_parts;            // partials written by this iteration's factorisation
  int pad2_;
  unsigned long long maxdiag_lm;   // bit pattern of max landmark diag(H) (non-negative double)
  unsigned long long maxdiag_kf;   // bit pattern of max keyframe diag(H), set by k_kf_reduce
  int refine_max;     // iterative-refinement corrections allowed per RCS solve
  int refined;        // corrections applied in this iteration
  double berr;        // backward error |r| / (|A| |dc| + |b|) of the first RCS solve (NaN: not formed)
};

// Landmark range [l0, l1) with its pairs [p0, p1); used by linearisation,
// back-substitution and evaluation.
struct LinTile {
  int l0, l1, p0, p1;
  int kf_lo, kf_n, part_off;   // keyframes [kf_lo, kf_lo + kf_n) touched; part_off unused (-1)
  int kfl_off;                 // offset in lin_kf_off of this tile's kf_n + 1 list offsets
  int o0, o1;                  // observations [o0, o1) of the tile's pairs
  int kfi0, kfi_n;             // the tile's entries [kfi0, kfi0 + kfi_n) of lin_kf_idx
};

// Landmark range for the Schur kernel: pairs [p0, p1), off-diagonal block work items
// [b0, b1), and the window of free keyframe blocks [k_lo, k_lo + span) whose part of the
// reduced camera system is accumulated in shared memory (direct = 1: straight to global).
struct SchurTile {
  int l0, l1, p0, p1, b0, b1, k_lo, span, direct;
  int part_off;                // offset of the window partial in schur_part (-1: direct)
};

struct Dev {
  int K, C, M, N, P, n_c, fixed_kf, mixed;
  int n_lin_tiles, n_schur_tiles;
  // problem
  const double* rig;          // C * RIG_STRIDE
  double* pose[2];            // K * POSE_STRIDE, double-buffered state
  double* lm[2];              // M * 3 (internal landmark order)
  // FP32 mirrors of the state for the mixed path (written wherever the FP64 state is
  // written; FP64<->FP32 conversions run on the slow FP64 pipe, so hot loops avoid them)
  const float* rig_f;         // C * RIG_STRIDE
  float* pose_f[2];           // K * POSE_STRIDE
  float* lm_f[2];             // M * 3
  float* dc_f;                // n_c
  const void* obs_uv;         // N * 2, double (FP64) or float (mixed)
  const int32_t* obs_cam;     // N
  const int32_t* pair_kf;     // P
  const int32_t* pair_lm;     // P
  const int32_t* pair_obs;    // P + 1 observation offsets
  const int32_t* lm_pair;     // M + 1 pair offsets
  const int32_t* lm_blk;      // M + 1 off-diagonal block offsets, m(m-1)/2 per landmark
  const int32_t* kf_pb;       // K: free block index or -1 for the fixed keyframe
  const LinTile* lin_tiles;
  const SchurTile* schur_tiles;    // landmarks sharing one window of <= SPAN_MAX free keyframes
  const SchurTile* direct_tiles;   // landmarks spanning more (atomics into S)
  int n_direct_tiles, max_span;
  int chol_fallback;               // batched solves: 1 = factor with the single-CTA kernel
  // linearisation
  void* pair_lin;             // P * PAIR_LIN (double or float)
  double* lm_H;               // M * 6  (Hll: 00 01 02 11 12 22)
  double* lm_g;               // M * 3
  double* kf_gp;              // K * 6  pose gradient
  double* kf_dp;              // K * 6  diag of Hpp
  // Schur / solve
  double* lm_Vinv;            // M * VINV_STRIDE
  double* S;                  // n_c * n_c, both triangles (the factorisations read the lower one)
  double* bS;                 // n_c   sum of W V^-1 g_l
  double* dc;                 // n_c   pose increment
  double* dp;                 // M * 3 landmark increment
  // blocked factorisation of large systems (chol_blocked = 1): the factor L (npw x npw, row
  // stride npw, lower triangle; npw = n_c rounded up to whole 32-column panels), the
  // reciprocals of its diagonal and y = L^-1 (rhs), read back by the cluster kernel
  double* Lw;
  double* Ldinv;
  double* yw;
  int npw, chol_blocked;
  // envelope of the factor by 32-column panel: rows [32 (p + 1), panel_end[p]) are the only
  // rows below panel p with nonzeros in its columns (first coupled keyframe of each row's
  // keyframe at or before the panel; the Cholesky fill stays inside this envelope)
  int16_t panel_end[kMaxPanels];
  // per-tile partials and the lists of tiles covering each keyframe / RCS block
  double* kf_part;            // keyframe-major slots of 12 (g_p 6, diag Hpp 6), one per covering lin
                              // tile (kf_tiles_off); mixed: float (hi, lo) pairs
  const int32_t* lin_kf_off;  // per lin tile, per keyframe of its range: start in lin_kf_idx (kf_n + 1)
  const int32_t* lin_kf_idx;  // tile-local indices of each keyframe's free pairs, in pair order
  const int32_t* lin_kf_slot; // per lin tile, per keyframe of its range: its slot in kf_part (kf_n + 1)
  double* schur_part;         // per Schur tile: window (rows (rows + 1) / 2) then b (rows)
  const int32_t* kf_tiles_off;   // K + 1: each keyframe's slots in kf_part
  const int32_t* blk_tiles_off;  // n_blk + 1, blocks (a >= b) of free keyframes
  const int32_t* blk_part_at;    // per block, per covering Schur tile: start of its 36 values in schur_part
  int n_blk;
  const int32_t* act_blk;        // blocks some tile touches, plus the diagonal ones
  int n_act;
  // partial sums per linearisation tile
  double* lin_part;           // n_lin_tiles * 4: cost, sum r^2, n_valid, n_inlier
  double* bs_part;            // n_lin_tiles * 4: candidate cost, pred_l, step2_l, unused
  cvba_iter* trace;           // iteration records (ctrl->iters entries)
  Ctrl* ctrl;
};

// Batched solve of independent windows: each phase is one launch over a work list of
// (window, item) pairs; the Cholesky runs one cluster of chol_cs CTAs per window.
struct BatchLaunch {
  const Dev* wins = nullptr;       // device array of per-window views
  int n_win = 0, mixed = 0;
  const int2* lin_items = nullptr;   int n_lin = 0;      // (window, lin tile)
  const int2* kf_items = nullptr;    int n_kf = 0;       // (window, keyframe)
  const int2* schur_items = nullptr; int n_schur = 0;    // (window, group tile)
  const int2* blk_items = nullptr;   int n_blkit = 0;    // (window, RCS block)
  const int2* direct_items = nullptr; int n_direct = 0;  // (window, direct tile)
  const int2* win_items = nullptr;                       // (window, 0)
  size_t lin_smem = 0, backsub_smem = 0, group_smem = 0, direct_smem = 0, chol_smem = 0;
  int chol_cs = 4;
  int n_fallback = 0;
  const Dev* fallback_host = nullptr;                   // host copies of windows that do not fit
};
// Fill the shared-memory maxima and fallback flags of `b` from host copies of the views
// (chol_fallback is written into host_devs before they are uploaded).
void batch_plan_sizes(Dev* host_devs, int n_win, BatchLaunch& b);
cudaError_t enqueue_batch_init(const BatchLaunch& b, double lam0, double huber, double zmin, int iters, int reset,
                               int refine, cudaStream_t s);
cudaError_t enqueue_batch_iteration(const BatchLaunch& b, cudaStream_t s);
int batch_kernels_per_iteration(const BatchLaunch& b);
int solve_kernels_per_iteration(const Dev& d);

// Launchers (cvba_kernels.cu).  All enqueue on `s` and return the launch status.
cudaError_t enqueue_solve_init(const Dev& d, double lam0, double huber, double zmin, int iters,
                               int reset_lambda, int refine, cudaStream_t s);
// A second stream and two events of the context, for work of an iteration that overlaps the
// main stream (the blocked factorisation's trailing updates).  Null members: no overlap.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// One LM iteration.  With ev != nullptr, profile_parts() + 1 events are recorded around
// the iteration's parts (for cvba_profile_iteration).
cudaError_t enqueue_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev, const SideStream* side = nullptr);
int profile_parts();
const char* profile_names();
// State transfer between a caller's device array (caller layout and landmark order) and
// the current state buffer: mode 0 poses in, 1 landmarks in, 2 poses out, 3 landmarks out.
cudaError_t enqueue_state_io(const Dev& d, int mode, double* user, const int32_t* lm_order, cudaStream_t s);
int kernels_per_iteration();
int kernels_per_solve_init();
cudaError_t enqueue_evaluate(const Dev& d, double huber, double zmin, double* out4, cudaStream_t s);
cudaError_t set_kernel_attributes();

}  // namespace cvba
