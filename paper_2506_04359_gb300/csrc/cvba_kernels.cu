// CUDA kernels of one Levenberg-Marquardt iteration of sliding-window bundle adjustment
// (cuVSLAM, arXiv 2506.04359, Sec. 2.2: reprojection residual Eq. r^repr, objective
// Eq. argmin, Schur complement "poses first, points afterwards").
//
// One iteration, all on the device (the accept/reject decision included):
//   k_lin      linearise at x: per (landmark, keyframe) pair the camera-frame information
//              M3 = sum_k w A_k^T A_k and a3 = sum_k w A_k^T r_k (A = d pi / d X_b); per
//              landmark Hll, g_l; per keyframe g_p and diag(Hpp); cost, counts.  Skipped
//              when the previous step was rejected (x unchanged).
//   k_schur    V_j = Hll_j + lam D_l,j, closed-form V_j^-1, W_ja, Y_ja = W_ja V_j^-1 and the
//              reduced camera system S = Hpp - sum_j W_j V_j^-1 W_j^T, b = sum_j Y_j g_l,j,
//              accumulated per tile in a shared-memory window of S.
//   k_chol     S + lam D_p = L L^T (FP64), dc = solve(-g_p + b); pose part of the predicted
//              reduction; candidate poses Exp(dxi) T.
//   k_backsub  dp_j = -V_j^-1 (g_l,j + sum_a W_ja^T dc_a); candidate landmarks; candidate
//              cost F'.
//   k_decide   gain ratio, accept/reject, Nielsen lambda update, iteration record.
//
// Compute type T: double (FP64 path) or float (mixed path).  All sums of the normal
// equations, the Schur window and the costs are accumulated in double.
#include <cfloat>
#include <math_constants.h>
#include <cmath>

#include "cvba_internal.h"

namespace cvba {
namespace {

constexpr double kDiagFloor = 1e-12;   // Marquardt floor relative to max(diag H)
constexpr double kTaylorTheta = 1e-4;  // Exp uses its Taylor series below this angle

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of four per-thread values over the block, in a fixed order.  Result valid in
// thread 0.  `red` holds at least 4 * 32 doubles.
__device__ void block_sum4(double v[4], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double x = lane < nw ? red[k * 32 + lane] : 0.0;
      v[k] = warp_sum(x);
    }
  }
  __syncthreads();
}

__device__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    double x = lane < nw ? red[lane] : 0.0;
    r = warp_max(x);
    if (lane == 0) red[0] = r;
  }
  __syncthreads();
  r = red[0];
  __syncthreads();
  return r;
}

// Marquardt floor 1e-12 * max(diag H) over landmarks (atomic max by k_lin) and poses.
__device__ double diag_floor(const Dev& d, double* red) {
  double m = 0.0;
  for (int i = threadIdx.x; i < d.K * 6; i += blockDim.x) m = fmax(m, d.kf_dp[i]);
  m = block_max(m, red);
  m = fmax(m, __longlong_as_double((long long)d.ctrl->maxdiag_lm));
  return kDiagFloor * m;
}

// -------------------------------------------------------------- observations

__device__ __forceinline__ void load_uv(const double* uv, int n, double& u, double& v) {
  const double2 x = reinterpret_cast<const double2*>(uv)[n];
  u = x.x;
  v = x.y;
}
__device__ __forceinline__ void load_uv(const float* uv, int n, float& u, float& v) {
  const float2 x = reinterpret_cast<const float2*>(uv)[n];
  u = x.x;
  v = x.y;
}

struct PairStats {
  double cost = 0.0, sq = 0.0;
  int nv = 0, ni = 0;
};

// Residuals of the observations [o0, o1) of one (landmark, keyframe) pair at pose P
// and landmark pw; with JAC also the pair's camera-frame information M3 (sym 00 01 02 11
// 12 22) and a3 = sum w A^T r, A = d pi(X_c) / d X_b = J_pi R_cb.
template <typename T, bool JAC>
__device__ __forceinline__ void eval_pair(const double* __restrict__ P, const double* pw, int o0, int o1,
                                          const int32_t* __restrict__ obs_cam, const T* __restrict__ uv,
                                          const double* rig, T hub, T zmin, T X[3], T M3[6], T a3[3],
                                          PairStats& st) {
  T R[9], t[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = (T)P[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) t[k] = (T)P[9 + k];
  const T px = (T)pw[0], py = (T)pw[1], pz = (T)pw[2];
#pragma unroll
  for (int r = 0; r < 3; ++r) X[r] = fma(R[3 * r], px, fma(R[3 * r + 1], py, fma(R[3 * r + 2], pz, t[r])));
  if (JAC) {
#pragma unroll
    for (int k = 0; k < 6; ++k) M3[k] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) a3[k] = 0;
  }
  for (int n = o0; n < o1; ++n) {
    const double* rg = rig + obs_cam[n] * RIG_STRIDE;
    const T fx = (T)rg[0], fy = (T)rg[1], cx = (T)rg[2], cy = (T)rg[3];
    T Rc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Rc[k] = (T)rg[4 + k];
    const T xc = fma(Rc[0], X[0], fma(Rc[1], X[1], fma(Rc[2], X[2], (T)rg[13])));
    const T yc = fma(Rc[3], X[0], fma(Rc[4], X[1], fma(Rc[5], X[2], (T)rg[14])));
    const T zc = fma(Rc[6], X[0], fma(Rc[7], X[1], fma(Rc[8], X[2], (T)rg[15])));
    if (!(zc > zmin)) continue;
    const T iz = (T)1 / zc;
    const T xn = xc * iz, yn = yc * iz;
    T uo, vo;
    load_uv(uv, n, uo, vo);
    const T r0 = fma(fx, xn, cx) - uo;
    const T r1 = fma(fy, yn, cy) - vo;
    const T s = fma(r0, r0, r1 * r1);
    const T e = sqrt(s);
    const bool inl = e <= hub;
    const T rho = inl ? s : fma((T)2 * hub, e, -hub * hub);
    st.cost += 0.5 * (double)rho;
    st.sq += (double)s;
    st.nv += 1;
    st.ni += inl ? 1 : 0;
    if (JAC) {
      const T w = inl ? (T)1 : hub / e;
      const T f0 = fx * iz, f1 = fy * iz;
      T A0[3], A1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        A0[k] = f0 * fma(-xn, Rc[6 + k], Rc[k]);
        A1[k] = f1 * fma(-yn, Rc[6 + k], Rc[3 + k]);
      }
      T wA0[3], wA1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        wA0[k] = w * A0[k];
        wA1[k] = w * A1[k];
      }
      M3[0] += fma(wA0[0], A0[0], wA1[0] * A1[0]);
      M3[1] += fma(wA0[0], A0[1], wA1[0] * A1[1]);
      M3[2] += fma(wA0[0], A0[2], wA1[0] * A1[2]);
      M3[3] += fma(wA0[1], A0[1], wA1[1] * A1[1]);
      M3[4] += fma(wA0[1], A0[2], wA1[1] * A1[2]);
      M3[5] += fma(wA0[2], A0[2], wA1[2] * A1[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) a3[k] += fma(wA0[k], r0, wA1[k] * r1);
    }
  }
}

template <typename T>
__device__ __forceinline__ void sym3_full(const T s[6], T m[9]) {
  m[0] = s[0]; m[1] = s[1]; m[2] = s[2];
  m[3] = s[1]; m[4] = s[3]; m[5] = s[4];
  m[6] = s[2]; m[7] = s[4]; m[8] = s[5];
}

// U = B^T M3 B with B = [I | -[X]x] (6 x 6, row-major), i.e. J_pose^T W J_pose summed
// over the pair's observations.
template <typename T>
__device__ __forceinline__ void pose_info(const T M[9], const T X[3], T U[36]) {
  T B[18];   // 3 x 6
#pragma unroll
  for (int k = 0; k < 18; ++k) B[k] = 0;
  B[0] = 1; B[7] = 1; B[14] = 1;
  // -[X]x in columns 3..5
  B[0 * 6 + 4] = X[2];  B[0 * 6 + 5] = -X[1];
  B[1 * 6 + 3] = -X[2]; B[1 * 6 + 5] = X[0];
  B[2 * 6 + 3] = X[1];  B[2 * 6 + 4] = -X[0];
  T MB[18];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) MB[r * 6 + c] = M[r * 3] * B[c] + M[r * 3 + 1] * B[6 + c] + M[r * 3 + 2] * B[12 + c];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) U[r * 6 + c] = B[r] * MB[c] + B[6 + r] * MB[6 + c] + B[12 + r] * MB[12 + c];
}

// --------------------------------------------------------------- SE(3) update

__device__ void pose_plus(const double* T0, const double* xi, double* T1) {
  const double rho[3] = {xi[0], xi[1], xi[2]};
  const double ph[3] = {xi[3], xi[4], xi[5]};
  const double th2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
  const double th = sqrt(th2);
  double A, B, C;
  if (th < kTaylorTheta) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    C = 1.0 / 6.0 - th2 / 120.0;
  } else {
    const double s = sin(th), c = cos(th);
    A = s / th;
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
  }
  const double P[9] = {0.0, -ph[2], ph[1], ph[2], 0.0, -ph[0], -ph[1], ph[0], 0.0};
  double P2[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) P2[r * 3 + c] = P[r * 3] * P[c] + P[r * 3 + 1] * P[3 + c] + P[r * 3 + 2] * P[6 + c];
  double Re[9], V[9];
  for (int k = 0; k < 9; ++k) {
    const double I = (k % 4 == 0) ? 1.0 : 0.0;
    Re[k] = I + A * P[k] + B * P2[k];
    V[k] = I + B * P[k] + C * P2[k];
  }
  double te[3];
  for (int r = 0; r < 3; ++r) te[r] = V[r * 3] * rho[0] + V[r * 3 + 1] * rho[1] + V[r * 3 + 2] * rho[2];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      T1[r * 3 + c] = Re[r * 3] * T0[c] + Re[r * 3 + 1] * T0[3 + c] + Re[r * 3 + 2] * T0[6 + c];
    T1[9 + r] = Re[r * 3] * T0[9] + Re[r * 3 + 1] * T0[10] + Re[r * 3 + 2] * T0[11] + te[r];
  }
}

// =================================================================== kernels

__global__ void k_solve_init(Dev d, double lam0, double huber, double zmin, int iters, int reset) {
  Ctrl* c = d.ctrl;
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    c->need_lin = 1;
    c->it = 0;
    c->nonpd = 0;
    c->iters = iters;
    if (reset) {
      c->lam = lam0;
      c->nu = 2.0;
    }
    c->huber = huber;
    c->zmin = zmin;
    c->pred_p = 0.0;
    c->step2_p = 0.0;
    c->maxdiag_lm = 0ull;
  }
  for (int i = threadIdx.x; i < d.K * 6; i += blockDim.x) {
    d.kf_gp[i] = 0.0;
    d.kf_dp[i] = 0.0;
  }
}

// ----------------------------------------------------------------- k_lin
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_lin(Dev d) {
  Ctrl* ctrl = d.ctrl;
  if (!ctrl->need_lin) return;
  extern __shared__ __align__(16) double smem[];
  const LinTile tile = d.lin_tiles[blockIdx.x];
  const int nl = tile.l1 - tile.l0;
  double* s_rig = smem;                                // C * 16
  double* s_lm = s_rig + d.C * RIG_STRIDE;             // LIN_TILE_LMS * 9
  double* s_kf = s_lm + LIN_TILE_LMS * 9;              // K * 12
  double* s_red = s_kf + d.K * 12;                     // 128
  int* s_flag = reinterpret_cast<int*>(s_red + 128);   // K
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = d.rig[i];
  for (int i = threadIdx.x; i < nl * 9; i += blockDim.x) s_lm[i] = 0.0;
  for (int i = threadIdx.x; i < d.K * 12; i += blockDim.x) s_kf[i] = 0.0;
  for (int i = threadIdx.x; i < d.K; i += blockDim.x) s_flag[i] = 0;
  __syncthreads();

  const int cur = ctrl->cur;
  const double* pose = d.pose[cur];
  const double* lmp = d.lm[cur];
  const T hub = (T)ctrl->huber, zmin = (T)ctrl->zmin;
  PairStats st;
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int a = d.pair_kf[q], j = d.pair_lm[q];
    T X[3], M3[6], a3[3];
    eval_pair<T, true>(pose + a * POSE_STRIDE, lmp + 3 * j, d.pair_obs[q], d.pair_obs[q + 1], d.obs_cam,
                       reinterpret_cast<const T*>(d.obs_uv), s_rig, hub, zmin, X, M3, a3, st);
    T* pl = reinterpret_cast<T*>(d.pair_lin) + (size_t)q * PAIR_LIN;
#pragma unroll
    for (int k = 0; k < 6; ++k) pl[k] = M3[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) pl[6 + k] = X[k];
    // landmark block: J_lm = A R  ->  Hll += R^T M3 R, g_l += R^T a3
    T R[9], M[9], G[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = (T)pose[a * POSE_STRIDE + k];
    sym3_full(M3, M);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) G[r * 3 + c] = M[r * 3] * R[c] + M[r * 3 + 1] * R[3 + c] + M[r * 3 + 2] * R[6 + c];
    double* L = s_lm + (j - tile.l0) * 9;
    const int si[6] = {0, 0, 0, 1, 1, 2}, sj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int r = si[k], c = sj[k];
      const T h = R[r] * G[c] + R[3 + r] * G[3 + c] + R[6 + r] * G[6 + c];
      atomicAdd(L + k, (double)h);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) atomicAdd(L + 6 + r, (double)(R[r] * a3[0] + R[3 + r] * a3[1] + R[6 + r] * a3[2]));
    if (d.kf_pb[a] >= 0) {
      // pose gradient B^T a3 = (a3, X x a3); diag of B^T M3 B
      double* Kf = s_kf + a * 12;
      atomicAdd(Kf + 0, (double)a3[0]);
      atomicAdd(Kf + 1, (double)a3[1]);
      atomicAdd(Kf + 2, (double)a3[2]);
      atomicAdd(Kf + 3, (double)(X[1] * a3[2] - X[2] * a3[1]));
      atomicAdd(Kf + 4, (double)(X[2] * a3[0] - X[0] * a3[2]));
      atomicAdd(Kf + 5, (double)(X[0] * a3[1] - X[1] * a3[0]));
      atomicAdd(Kf + 6, (double)M3[0]);
      atomicAdd(Kf + 7, (double)M3[3]);
      atomicAdd(Kf + 8, (double)M3[5]);
      atomicAdd(Kf + 9, (double)(M3[3] * X[2] * X[2] - 2 * M3[4] * X[1] * X[2] + M3[5] * X[1] * X[1]));
      atomicAdd(Kf + 10, (double)(M3[0] * X[2] * X[2] - 2 * M3[2] * X[0] * X[2] + M3[5] * X[0] * X[0]));
      atomicAdd(Kf + 11, (double)(M3[0] * X[1] * X[1] - 2 * M3[1] * X[0] * X[1] + M3[3] * X[0] * X[0]));
      s_flag[a] = 1;
    }
  }
  double v[4] = {st.cost, st.sq, (double)st.nv, (double)st.ni};
  block_sum4(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) d.lin_part[blockIdx.x * 4 + k] = v[k];
  }
  __syncthreads();
  double mx = 0.0;
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int j = tile.l0 + l;
#pragma unroll
    for (int k = 0; k < 6; ++k) d.lm_H[j * 6 + k] = s_lm[l * 9 + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) d.lm_g[j * 3 + k] = s_lm[l * 9 + 6 + k];
    mx = fmax(mx, fmax(s_lm[l * 9], fmax(s_lm[l * 9 + 3], s_lm[l * 9 + 5])));
  }
  mx = block_max(mx, s_red);
  if (threadIdx.x == 0 && mx > 0.0)
    atomicMax(&ctrl->maxdiag_lm, (unsigned long long)__double_as_longlong(mx));
  for (int a = threadIdx.x; a < d.K; a += blockDim.x) {
    if (!s_flag[a]) continue;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      atomicAdd(d.kf_gp + a * 6 + k, s_kf[a * 12 + k]);
      atomicAdd(d.kf_dp + a * 6 + k, s_kf[a * 12 + 6 + k]);
    }
  }
}

// ---------------------------------------------------------------- k_schur
template <typename T>
struct SchurSmem {
  static constexpr int WIN = 6 * SPAN_MAX;
  static constexpr int WIN_ENTRIES = WIN * (WIN + 1) / 2;
  static constexpr size_t bytes() {
    return sizeof(double) * (WIN_ENTRIES + WIN + SCHUR_TILE_LMS * 9 + 64) +
           sizeof(T) * (SCHUR_TILE_PAIRS * 36) + sizeof(int) * (SCHUR_TILE_LMS + 1);
  }
};

template <typename T>
__global__ void __launch_bounds__(SCHUR_THREADS) k_schur(Dev d) {
  using SM = SchurSmem<T>;
  extern __shared__ __align__(16) double smem[];
  double* s_win = smem;                               // WIN_ENTRIES
  double* s_b = s_win + SM::WIN_ENTRIES;              // WIN
  double* s_vinv = s_b + SM::WIN;                     // SCHUR_TILE_LMS * 6
  double* s_gl = s_vinv + SCHUR_TILE_LMS * 6;         // SCHUR_TILE_LMS * 3
  double* s_red = s_gl + SCHUR_TILE_LMS * 3;          // 64
  T* s_W = reinterpret_cast<T*>(s_red + 64);          // SCHUR_TILE_PAIRS * 18
  T* s_Y = s_W + SCHUR_TILE_PAIRS * 18;               // SCHUR_TILE_PAIRS * 18
  int* s_blk = reinterpret_cast<int*>(s_Y + SCHUR_TILE_PAIRS * 18);  // SCHUR_TILE_LMS + 1

  Ctrl* ctrl = d.ctrl;
  const SchurTile tile = d.schur_tiles[blockIdx.x];
  const int nl = tile.l1 - tile.l0;
  const int n_c = d.n_c;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);
  const int rows = 6 * tile.span;
  if (!tile.direct) {
    for (int i = threadIdx.x; i < rows * (rows + 1) / 2; i += blockDim.x) s_win[i] = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s_b[i] = 0.0;
  }
  // phase 1: closed-form inverse of V_j = Hll_j + lam D_l,j (adjugate / determinant).
  // Mixed path only: Hll_j is summed from FP32 products, so information below ~2^-23 of
  // its trace is rounding noise (a landmark drifting to infinity along its ray has an
  // eigenvalue ~1e-15 of the others).  If V_j then fails the positive-definite test, the
  // block is retried with tau = 2^-20 tr(Hll_j) added to its diagonal; tau enters the
  // predicted reduction in k_backsub.  The FP64 path never adds tau.
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int j = tile.l0 + l;
    const double* H = d.lm_H + 6 * j;
    double inv[6];
    double tau = 0.0;
    bool ok = false;
    for (int attempt = 0; attempt < (sizeof(T) == 4 ? 2 : 1) && !ok; ++attempt) {
      if (attempt == 1) tau = 0x1p-20 * (H[0] + H[3] + H[5]);
      const double a = H[0] + lam * fmax(H[0], floor_) + tau;
      const double b = H[1], c = H[2];
      const double dd = H[3] + lam * fmax(H[3], floor_) + tau;
      const double e = H[4];
      const double f = H[5] + lam * fmax(H[5], floor_) + tau;
      const double A = dd * f - e * e, Bc = c * e - b * f, Cc = b * e - c * dd;
      const double det = a * A + b * Bc + c * Cc;
      const double m2 = a * dd - b * b;
      if (a > 0.0 && m2 > 0.0 && det > 0.0 && isfinite(det)) {
        const double id = 1.0 / det;
        inv[0] = A * id;
        inv[1] = Bc * id;
        inv[2] = Cc * id;
        inv[3] = (a * f - c * c) * id;
        inv[4] = (b * c - a * e) * id;
        inv[5] = m2 * id;
        ok = true;
      }
    }
    if (!ok) {
      for (int k = 0; k < 6; ++k) inv[k] = 0.0;
      tau = 0.0;
      ctrl->nonpd = 1;
    }
    for (int k = 0; k < 6; ++k) {
      s_vinv[l * 6 + k] = inv[k];
      d.lm_Vinv[j * VINV_STRIDE + k] = inv[k];
    }
    d.lm_Vinv[j * VINV_STRIDE + 6] = tau;
    for (int k = 0; k < 3; ++k) s_gl[l * 3 + k] = d.lm_g[j * 3 + k];
  }
  for (int l = threadIdx.x; l <= nl; l += blockDim.x) s_blk[l] = d.lm_blk[tile.l0 + l] - tile.b0;
  __syncthreads();

  auto acc_S = [&](int pr, int pc, int r, int c, double v) {
    if (tile.direct) {
      atomicAdd(d.S + (size_t)(6 * pr + r) * n_c + 6 * pc + c, v);
    } else {
      const int wr = 6 * (pr - tile.k_lo) + r, wc = 6 * (pc - tile.k_lo) + c;
      atomicAdd(s_win + wr * (wr + 1) / 2 + wc, v);
    }
  };

  // phase 2: per pair W = [G; [X]x G] with G = M3 R, Y = W V^-1; diagonal block and b
  const double* pose = d.pose[ctrl->cur];
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int l = d.pair_lm[q] - tile.l0;
    const int a = d.pair_kf[q];
    const T* pl = reinterpret_cast<const T*>(d.pair_lin) + (size_t)q * PAIR_LIN;
    T M3[6], X[3], M[9], R[9], G[9];
#pragma unroll
    for (int k = 0; k < 6; ++k) M3[k] = pl[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) X[k] = pl[6 + k];
    sym3_full(M3, M);
#pragma unroll
    for (int k = 0; k < 9; ++k) R[k] = (T)pose[a * POSE_STRIDE + k];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) G[r * 3 + c] = M[r * 3] * R[c] + M[r * 3 + 1] * R[3 + c] + M[r * 3 + 2] * R[6 + c];
    T W[18];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = G[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      W[9 + c] = X[1] * G[6 + c] - X[2] * G[3 + c];
      W[12 + c] = X[2] * G[c] - X[0] * G[6 + c];
      W[15 + c] = X[0] * G[3 + c] - X[1] * G[c];
    }
    T Vi[9];
    {
      T s6[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) s6[k] = (T)s_vinv[l * 6 + k];
      sym3_full(s6, Vi);
    }
    T Y[18];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[r * 3 + c] = W[r * 3] * Vi[c] + W[r * 3 + 1] * Vi[3 + c] + W[r * 3 + 2] * Vi[6 + c];
    T* sw = s_W + (q - tile.p0) * 18;
    T* sy = s_Y + (q - tile.p0) * 18;
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      sw[k] = W[k];
      sy[k] = Y[k];
    }
    const int pb = d.kf_pb[a];
    if (pb >= 0) {
      T U[36];
      pose_info(M, X, U);
#pragma unroll
      for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) {
          const T v = U[r * 6 + c] - (Y[r * 3] * W[c * 3] + Y[r * 3 + 1] * W[c * 3 + 1] + Y[r * 3 + 2] * W[c * 3 + 2]);
          acc_S(pb, pb, r, c, (double)v);
        }
      const T g0 = (T)s_gl[l * 3], g1 = (T)s_gl[l * 3 + 1], g2 = (T)s_gl[l * 3 + 2];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const double v = (double)(Y[r * 3] * g0 + Y[r * 3 + 1] * g1 + Y[r * 3 + 2] * g2);
        if (tile.direct)
          atomicAdd(d.bS + 6 * pb + r, v);
        else
          atomicAdd(s_b + 6 * (pb - tile.k_lo) + r, v);
      }
    }
  }
  __syncthreads();

  // phase 3: off-diagonal blocks S_ba -= Y_b W_a^T for pairs a < b of one landmark
  const int nb = tile.b1 - tile.b0;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) {
    int lo = 0, hi = nl - 1;      // largest l with s_blk[l] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_blk[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int l = lo;
    const int lt = t - s_blk[l];
    int ib = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)lt)) * 0.5f);
    while (ib * (ib - 1) / 2 > lt) --ib;
    while ((ib + 1) * ib / 2 <= lt) ++ib;
    const int ia = lt - ib * (ib - 1) / 2;
    const int q0 = d.lm_pair[tile.l0 + l];
    const int qa = q0 + ia, qb = q0 + ib;
    const int pa = d.kf_pb[d.pair_kf[qa]], pbb = d.kf_pb[d.pair_kf[qb]];
    if (pa < 0 || pbb < 0) continue;
    const T* Yb = s_Y + (qb - tile.p0) * 18;
    const T* Wa = s_W + (qa - tile.p0) * 18;
    T yb[18], wa[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      yb[k] = Yb[k];
      wa[k] = Wa[k];
    }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        const T v = yb[r * 3] * wa[c * 3] + yb[r * 3 + 1] * wa[c * 3 + 1] + yb[r * 3 + 2] * wa[c * 3 + 2];
        acc_S(pbb, pa, r, c, -(double)v);
      }
  }
  __syncthreads();

  // phase 4: flush the window into the global reduced camera system
  if (!tile.direct) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int base = 6 * tile.k_lo;
    for (int wr = warp; wr < rows; wr += nw) {
      for (int wc = lane; wc <= wr; wc += 32) {
        const double v = s_win[wr * (wr + 1) / 2 + wc];
        if (v != 0.0) atomicAdd(d.S + (size_t)(base + wr) * n_c + base + wc, v);
      }
    }
    for (int r = threadIdx.x; r < rows; r += blockDim.x)
      if (s_b[r] != 0.0) atomicAdd(d.bS + base + r, s_b[r]);
  }
}

// ----------------------------------------------------------------- k_chol
// Dense FP64 Cholesky of the damped reduced camera system, then the two triangular
// solves.  One CTA; the matrix lives in shared memory when it fits (SMEM) else in global.
template <bool SMEM>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol(Dev d) {
  extern __shared__ __align__(16) double smem[];
  __shared__ double s_red[128];
  __shared__ double s_piv;
  __shared__ int s_bad;
  Ctrl* ctrl = d.ctrl;
  if (ctrl->nonpd) return;
  const int n = d.n_c;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double* A = SMEM ? smem : d.S;
  double* x = SMEM ? smem + n * n : d.dc;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);
  if (tid == 0) s_bad = 0;
  if (SMEM) {
    for (int i = tid; i < n * n; i += nt) {
      const int r = i / n, c = i % n;
      if (c <= r) A[i] = d.S[i];
    }
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    const int pb = i / 6, comp = i % 6;
    const int kf = pb < d.fixed_kf ? pb : pb + 1;
    A[(size_t)i * n + i] += lam * fmax(d.kf_dp[kf * 6 + comp], floor_);
    x[i] = d.bS[i] - d.kf_gp[kf * 6 + comp];
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double v = A[(size_t)k * n + k];
      if (!(v > 0.0) || !isfinite(v)) {
        s_bad = 1;
      } else {
        const double l = sqrt(v);
        A[(size_t)k * n + k] = l;
        s_piv = 1.0 / l;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const double ip = s_piv;
    for (int i = k + 1 + tid; i < n; i += nt) A[(size_t)i * n + k] *= ip;
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nw) {
      const double lik = A[(size_t)i * n + k];
      for (int j = k + 1 + lane; j <= i; j += 32) A[(size_t)i * n + j] -= lik * A[(size_t)j * n + k];
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) ctrl->nonpd = 1;
    return;
  }
  // forward: L y = rhs
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      x[k] /= A[(size_t)k * n + k];
      s_piv = x[k];
    }
    __syncthreads();
    const double yk = s_piv;
    for (int i = k + 1 + tid; i < n; i += nt) x[i] -= A[(size_t)i * n + k] * yk;
    __syncthreads();
  }
  // backward: L^T dc = y
  for (int k = n - 1; k >= 0; --k) {
    if (tid == 0) {
      x[k] /= A[(size_t)k * n + k];
      s_piv = x[k];
    }
    __syncthreads();
    const double xk = s_piv;
    for (int i = tid; i < k; i += nt) x[i] -= A[(size_t)k * n + i] * xk;
    __syncthreads();
  }
  // predicted-reduction and step-norm parts; candidate poses
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = tid; i < n; i += nt) {
    const int pb = i / 6, comp = i % 6;
    const int kf = pb < d.fixed_kf ? pb : pb + 1;
    const double D = fmax(d.kf_dp[kf * 6 + comp], floor_);
    const double xi = x[i];
    v[0] += xi * (lam * D * xi - d.kf_gp[kf * 6 + comp]);
    v[1] += xi * xi;
    if (SMEM) d.dc[i] = xi;
  }
  block_sum4(v, s_red);
  if (tid == 0) {
    ctrl->pred_p = v[0];
    ctrl->step2_p = v[1];
  }
  __syncthreads();
  const int cur = ctrl->cur;
  for (int a = tid; a < d.K; a += nt) {
    const double* T0 = d.pose[cur] + a * POSE_STRIDE;
    double* T1 = d.pose[cur ^ 1] + a * POSE_STRIDE;
    const int pb = d.kf_pb[a];
    if (pb < 0) {
      for (int k = 0; k < POSE_STRIDE; ++k) T1[k] = T0[k];
    } else {
      pose_plus(T0, d.dc + 6 * pb, T1);
    }
  }
}

// --------------------------------------------------------------- k_backsub
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_backsub(Dev d) {
  extern __shared__ __align__(16) double smem[];
  Ctrl* ctrl = d.ctrl;
  const LinTile tile = d.lin_tiles[blockIdx.x];
  if (ctrl->nonpd) {
    if (threadIdx.x < 4) d.bs_part[blockIdx.x * 4 + threadIdx.x] = 0.0;
    return;
  }
  const int nl = tile.l1 - tile.l0;
  double* s_rig = smem;                              // C * 16
  double* s_acc = s_rig + d.C * RIG_STRIDE;          // LIN_TILE_LMS * 3
  double* s_new = s_acc + LIN_TILE_LMS * 3;          // LIN_TILE_LMS * 3
  double* s_red = s_new + LIN_TILE_LMS * 3;          // 128
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = d.rig[i];
  for (int i = threadIdx.x; i < nl * 3; i += blockDim.x) s_acc[i] = 0.0;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);   // contains __syncthreads
  const int cur = ctrl->cur;
  const double* pose = d.pose[cur];
  // phase 1: W_ja^T dc_a = R_a^T M3 (rho + phi x X) accumulated per landmark
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int a = d.pair_kf[q];
    const int pb = d.kf_pb[a];
    if (pb < 0) continue;
    const T* pl = reinterpret_cast<const T*>(d.pair_lin) + (size_t)q * PAIR_LIN;
    const double* xi = d.dc + 6 * pb;
    T X[3] = {pl[6], pl[7], pl[8]};
    T u[3];
    u[0] = (T)xi[0] + ((T)xi[4] * X[2] - (T)xi[5] * X[1]);
    u[1] = (T)xi[1] + ((T)xi[5] * X[0] - (T)xi[3] * X[2]);
    u[2] = (T)xi[2] + ((T)xi[3] * X[1] - (T)xi[4] * X[0]);
    T M[9];
    {
      T s6[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) s6[k] = pl[k];
      sym3_full(s6, M);
    }
    T w3[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) w3[r] = M[r * 3] * u[0] + M[r * 3 + 1] * u[1] + M[r * 3 + 2] * u[2];
    const double* R = pose + a * POSE_STRIDE;
    double* acc = s_acc + (d.pair_lm[q] - tile.l0) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c)
      atomicAdd(acc + c, (double)((T)R[c] * w3[0] + (T)R[3 + c] * w3[1] + (T)R[6 + c] * w3[2]));
  }
  __syncthreads();
  // phase 2: dp_j = -V_j^-1 (g_l + acc); candidate landmark; predicted-reduction part
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int j = tile.l0 + l;
    const double* Vi = d.lm_Vinv + VINV_STRIDE * j;
    const double tau = Vi[6];
    const double* g = d.lm_g + 3 * j;
    const double t0 = g[0] + s_acc[l * 3], t1 = g[1] + s_acc[l * 3 + 1], t2 = g[2] + s_acc[l * 3 + 2];
    const double dp0 = -(Vi[0] * t0 + Vi[1] * t1 + Vi[2] * t2);
    const double dp1 = -(Vi[1] * t0 + Vi[3] * t1 + Vi[4] * t2);
    const double dp2 = -(Vi[2] * t0 + Vi[4] * t1 + Vi[5] * t2);
    const double* H = d.lm_H + 6 * j;
    const double D0 = fmax(H[0], floor_), D1 = fmax(H[3], floor_), D2 = fmax(H[5], floor_);
    v[1] += dp0 * ((lam * D0 + tau) * dp0 - g[0]) + dp1 * ((lam * D1 + tau) * dp1 - g[1]) +
            dp2 * ((lam * D2 + tau) * dp2 - g[2]);
    v[2] += dp0 * dp0 + dp1 * dp1 + dp2 * dp2;
    d.dp[j * 3] = dp0;
    d.dp[j * 3 + 1] = dp1;
    d.dp[j * 3 + 2] = dp2;
    const double* p = d.lm[cur] + 3 * j;
    double* pn = d.lm[cur ^ 1] + 3 * j;
    const double n0 = p[0] + dp0, n1 = p[1] + dp1, n2 = p[2] + dp2;
    pn[0] = n0; pn[1] = n1; pn[2] = n2;
    s_new[l * 3] = n0; s_new[l * 3 + 1] = n1; s_new[l * 3 + 2] = n2;
  }
  __syncthreads();
  // phase 3: candidate cost, same arithmetic and order as k_lin's cost
  const double* pnew = d.pose[cur ^ 1];
  const T hub = (T)ctrl->huber, zmin = (T)ctrl->zmin;
  PairStats st;
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int a = d.pair_kf[q], j = d.pair_lm[q];
    T X[3];
    eval_pair<T, false>(pnew + a * POSE_STRIDE, s_new + 3 * (j - tile.l0), d.pair_obs[q], d.pair_obs[q + 1],
                        d.obs_cam, reinterpret_cast<const T*>(d.obs_uv), s_rig, hub, zmin, X, nullptr, nullptr, st);
  }
  v[0] = st.cost;
  block_sum4(v, s_red);
  if (threadIdx.x == 0) {
    d.bs_part[blockIdx.x * 4 + 0] = v[0];
    d.bs_part[blockIdx.x * 4 + 1] = v[1];
    d.bs_part[blockIdx.x * 4 + 2] = v[2];
    d.bs_part[blockIdx.x * 4 + 3] = 0.0;
  }
}

// --------------------------------------------------------------- k_decide
// Fixed-order sum of tile partials (thread t takes tiles t, t+256, ...; then a tree).
__device__ void reduce_parts(const double* part, int n_tiles, double out[4], double* red) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
    for (int k = 0; k < 4; ++k) v[k] += part[t * 4 + k];
  block_sum4(v, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) red[64 + k] = v[k];
  __syncthreads();
  for (int k = 0; k < 4; ++k) out[k] = red[64 + k];
  __syncthreads();
}

__global__ void __launch_bounds__(DECIDE_THREADS) k_decide(Dev d) {
  __shared__ double s_red[128];
  Ctrl* ctrl = d.ctrl;
  double lin[4], bs[4];
  reduce_parts(d.lin_part, d.n_lin_tiles, lin, s_red);
  reduce_parts(d.bs_part, d.n_lin_tiles, bs, s_red);
  const int nonpd = ctrl->nonpd;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double F = lin[0];
    const double lam = ctrl->lam, nu = ctrl->nu;
    cvba_iter rec;
    rec.cost0 = F;
    rec.lambda = lam;
    rec.rms_px = lin[2] > 0.0 ? sqrt(lin[1] / lin[2]) : 0.0;
    rec.n_valid = (int)lin[2];
    rec.n_inlier = (int)lin[3];
    rec.nonpd = nonpd;
    bool acc = false;
    if (nonpd) {
      rec.cost1 = rec.gain = rec.pred = rec.step_norm = CUDART_NAN;
    } else {
      const double F1 = bs[0];
      const double L = 0.5 * (ctrl->pred_p + bs[1]);
      rec.cost1 = F1;
      rec.pred = L;
      rec.step_norm = sqrt(ctrl->step2_p + bs[2]);
      rec.gain = L != 0.0 ? (F - F1) / L : CUDART_NAN;
      acc = L > 0.0 && isfinite(F1) && rec.gain > 0.0;
    }
    rec.accepted = acc ? 1 : 0;
    if (ctrl->it < ctrl->iters) d.trace[ctrl->it] = rec;
    ctrl->it += 1;
    if (acc) {
      const double g = 2.0 * rec.gain - 1.0;
      ctrl->lam = lam * fmax(1.0 / 3.0, 1.0 - g * g * g);
      ctrl->nu = 2.0;
      ctrl->cur ^= 1;
      ctrl->need_lin = 1;
      ctrl->maxdiag_lm = 0ull;
    } else {
      ctrl->lam = lam * nu;
      ctrl->nu = 2.0 * nu;
      ctrl->need_lin = 0;
    }
    ctrl->nonpd = 0;
    s_red[0] = acc ? 1.0 : 0.0;
  }
  __syncthreads();
  if (s_red[0] != 0.0) {
    for (int i = threadIdx.x; i < d.K * 6; i += blockDim.x) {
      d.kf_gp[i] = 0.0;
      d.kf_dp[i] = 0.0;
    }
  }
}

// ------------------------------------------------------------- evaluation
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_eval(Dev d, double huber, double zmin, double* part) {
  extern __shared__ __align__(16) double smem[];
  const LinTile tile = d.lin_tiles[blockIdx.x];
  double* s_rig = smem;
  double* s_red = s_rig + d.C * RIG_STRIDE;
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = d.rig[i];
  __syncthreads();
  const int cur = d.ctrl->cur;
  const double* pose = d.pose[cur];
  const double* lmp = d.lm[cur];
  PairStats st;
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int a = d.pair_kf[q], j = d.pair_lm[q];
    T X[3];
    eval_pair<T, false>(pose + a * POSE_STRIDE, lmp + 3 * j, d.pair_obs[q], d.pair_obs[q + 1], d.obs_cam,
                        reinterpret_cast<const T*>(d.obs_uv), s_rig, (T)huber, (T)zmin, X, nullptr, nullptr, st);
  }
  double v[4] = {st.cost, st.sq, (double)st.nv, (double)st.ni};
  block_sum4(v, s_red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) part[blockIdx.x * 4 + k] = v[k];
}

__global__ void k_eval_reduce(const double* part, int n_tiles, double* out) {
  __shared__ double s_red[128];
  double v[4];
  reduce_parts(part, n_tiles, v, s_red);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) out[k] = v[k];
}

// Caller layout <-> state buffer d.*[ctrl->cur]: poses (3 x 4 row-major) <-> (R, t);
// landmarks in the caller's order <-> internal order lm_order[internal] = caller index.
__global__ void k_state_io(Dev d, int mode, double* user, const int32_t* lm_order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int cur = d.ctrl->cur;
  if (mode == 0 || mode == 2) {
    if (i >= d.K) return;
    double* P = d.pose[cur] + i * POSE_STRIDE;
    double* U = user + i * 12;
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) {
        if (mode == 0) P[r * 3 + c] = U[r * 4 + c]; else U[r * 4 + c] = P[r * 3 + c];
      }
      if (mode == 0) P[9 + r] = U[r * 4 + 3]; else U[r * 4 + 3] = P[9 + r];
    }
  } else {
    if (i >= d.M) return;
    double* L = d.lm[cur] + 3 * i;
    double* U = user + 3 * (size_t)lm_order[i];
    for (int k = 0; k < 3; ++k) {
      if (mode == 1) L[k] = U[k]; else U[k] = L[k];
    }
  }
}

size_t lin_smem(const Dev& d) {
  return sizeof(double) * (d.C * RIG_STRIDE + LIN_TILE_LMS * 9 + d.K * 12 + 128) + sizeof(int) * d.K;
}
size_t backsub_smem(const Dev& d) { return sizeof(double) * (d.C * RIG_STRIDE + LIN_TILE_LMS * 6 + 128); }
size_t eval_smem(const Dev& d) { return sizeof(double) * (d.C * RIG_STRIDE + 128); }
constexpr int kCholSmemMaxN = 160;
size_t chol_smem(int n) { return sizeof(double) * ((size_t)n * n + n); }

}  // namespace

// ================================================================ launchers

cudaError_t set_kernel_attributes() {
  cudaError_t e;
  const int big = 227 * 1024;
  e = cudaFuncSetAttribute(k_lin<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_lin<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_schur<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SchurSmem<double>::bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_schur<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)SchurSmem<float>::bytes());
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_chol<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)chol_smem(kCholSmemMaxN));
  return e;
}

int kernels_per_iteration() { return 5; }
int kernels_per_solve_init() { return 1; }

cudaError_t enqueue_solve_init(const Dev& d, double lam0, double huber, double zmin, int iters, int reset,
                               cudaStream_t s) {
  k_solve_init<<<1, 256, 0, s>>>(d, lam0, huber, zmin, iters, reset);
  return cudaGetLastError();
}

int profile_parts() { return 6; }
const char* profile_names() { return "lin,memset,schur,chol,backsub,decide"; }

cudaError_t enqueue_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e;
  auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
  if ((e = mark(0)) != cudaSuccess) return e;
  if (d.mixed)
    k_lin<float><<<d.n_lin_tiles, LIN_THREADS, lin_smem(d), s>>>(d);
  else
    k_lin<double><<<d.n_lin_tiles, LIN_THREADS, lin_smem(d), s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(1)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.S, 0, sizeof(double) * (size_t)d.n_c * d.n_c, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d.bS, 0, sizeof(double) * (size_t)d.n_c, s)) != cudaSuccess) return e;
  if ((e = mark(2)) != cudaSuccess) return e;
  if (d.mixed)
    k_schur<float><<<d.n_schur_tiles, SCHUR_THREADS, SchurSmem<float>::bytes(), s>>>(d);
  else
    k_schur<double><<<d.n_schur_tiles, SCHUR_THREADS, SchurSmem<double>::bytes(), s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(3)) != cudaSuccess) return e;
  if (d.n_c <= kCholSmemMaxN)
    k_chol<true><<<1, CHOL_THREADS, chol_smem(d.n_c), s>>>(d);
  else
    k_chol<false><<<1, CHOL_THREADS, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(4)) != cudaSuccess) return e;
  if (d.mixed)
    k_backsub<float><<<d.n_lin_tiles, LIN_THREADS, backsub_smem(d), s>>>(d);
  else
    k_backsub<double><<<d.n_lin_tiles, LIN_THREADS, backsub_smem(d), s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(5)) != cudaSuccess) return e;
  k_decide<<<1, DECIDE_THREADS, 0, s>>>(d);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return mark(6);
}

cudaError_t enqueue_state_io(const Dev& d, int mode, double* user, const int32_t* lm_order, cudaStream_t s) {
  const int n = (mode == 0 || mode == 2) ? d.K : d.M;
  const int blocks = (n + 255) / 256;
  k_state_io<<<blocks, 256, 0, s>>>(d, mode, user, lm_order);
  return cudaGetLastError();
}

cudaError_t enqueue_evaluate(const Dev& d, double huber, double zmin, double* out4, cudaStream_t s) {
  // partials go to the tail of bs_part's twin buffer: a dedicated region after lin_part
  double* part = d.bs_part + 4 * d.n_lin_tiles;
  if (d.mixed)
    k_eval<float><<<d.n_lin_tiles, LIN_THREADS, eval_smem(d), s>>>(d, huber, zmin, part);
  else
    k_eval<double><<<d.n_lin_tiles, LIN_THREADS, eval_smem(d), s>>>(d, huber, zmin, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_eval_reduce<<<1, DECIDE_THREADS, 0, s>>>(part, d.n_lin_tiles, out4);
  return cudaGetLastError();
}

}  // namespace cvba
