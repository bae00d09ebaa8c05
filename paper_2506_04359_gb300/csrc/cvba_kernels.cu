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
#include <cooperative_groups.h>
#include <math_constants.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <type_traits>

#include "cvba_internal.h"

namespace cvba {
namespace {

constexpr double kDiagFloor = 1e-12;   // Marquardt floor relative to max(diag H)

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

// Block maximum of non-negative floats (result in every thread).  Contains barriers.
__device__ float block_max_f(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float r = 0.0f;
  for (int w = 0; w < nw; ++w) r = fmaxf(r, red[w]);
  __syncthreads();
  return r;
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

// Marquardt floor 1e-12 * max(diag H) over landmarks (atomic max by k_lin) and poses
// (atomic max by k_kf_reduce).  Starts with a block barrier, which callers rely on.
__device__ double diag_floor(const Dev& d, double* /*red*/) {
  __syncthreads();
  const double m = fmax(__longlong_as_double((long long)d.ctrl->maxdiag_lm),
                        __longlong_as_double((long long)d.ctrl->maxdiag_kf));
  return kDiagFloor * m;
}

// ---------------------------------------------------------- compensated FP32 sums
// A value hi + lo held in two floats (about 48 significant bits).  The mixed path keeps
// its sums in this form and converts to FP64 once per tile: on GB300 every FP64
// operation, conversions included, issues at 1/64 of the FP32 rate.
struct DF {
  float hi, lo;
};

// Error-free sum of the high parts (Knuth's TwoSum), low parts added, renormalised
// (Dekker's Fast2Sum).  Symmetric in its arguments.
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}

__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const DF w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, w);
  }
  return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum of NV compensated values; thread 0 gets the FP64 results.
// `red` holds >= 2 * NV * 32 floats.  Contains barriers.
template <int NV>
__device__ void block_sum_df(DF v[NV], double out[NV], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum_df(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      red[(2 * k) * 32 + warp] = v[k].hi;
      red[(2 * k + 1) * 32 + warp] = v[k].lo;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      DF x{lane < nw ? red[(2 * k) * 32 + lane] : 0.0f, lane < nw ? red[(2 * k + 1) * 32 + lane] : 0.0f};
      x = warp_sum_df(x);
      out[k] = (double)x.hi + (double)x.lo;
    }
  }
  __syncthreads();
}

// As block_sum_df, but thread 0 gets the compensated (hi, lo) results themselves.
template <int NV>
__device__ void block_sum_df_pair(DF v[NV], DF out[NV], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum_df(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      red[(2 * k) * 32 + warp] = v[k].hi;
      red[(2 * k + 1) * 32 + warp] = v[k].lo;
    }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      DF x{lane < nw ? red[(2 * k) * 32 + lane] : 0.0f, lane < nw ? red[(2 * k + 1) * 32 + lane] : 0.0f};
      out[k] = warp_sum_df(x);
    }
  }
  __syncthreads();
}

// Fixed-order block sum of integer counts; thread 0 gets the result.  `red` >= 32 ints.
__device__ int block_sum_i(int v, int* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_i(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  int r = 0;
  if (warp == 0) r = warp_sum_i(lane < nw ? red[lane] : 0);
  __syncthreads();
  return r;
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

// Running sum: plain for double; Kahan-compensated for float (s - c is the sum).
template <typename T>
struct Acc {
  T s = 0, c = 0;
  __device__ __forceinline__ void add(T v) {
    if (sizeof(T) == 4) {
      const T y = v - c;
      const T t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += v;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
  __device__ __forceinline__ DF df() const { return DF{(float)s, -(float)c}; }
  __device__ __forceinline__ T rounded() const { return s - c; }
};

template <typename T>
struct PairStats {
  Acc<T> cost, sq;
  int nv = 0, ni = 0;
};

// State in the compute type: the FP64 buffers, or their FP32 mirrors on the mixed path.
template <typename T> __device__ __forceinline__ const T* st_pose(const Dev& d, int b);
template <> __device__ __forceinline__ const double* st_pose<double>(const Dev& d, int b) { return d.pose[b]; }
template <> __device__ __forceinline__ const float* st_pose<float>(const Dev& d, int b) { return d.pose_f[b]; }
template <typename T> __device__ __forceinline__ const T* st_lm(const Dev& d, int b);
template <> __device__ __forceinline__ const double* st_lm<double>(const Dev& d, int b) { return d.lm[b]; }
template <> __device__ __forceinline__ const float* st_lm<float>(const Dev& d, int b) { return d.lm_f[b]; }
template <typename T> __device__ __forceinline__ const T* st_rig(const Dev& d);
template <> __device__ __forceinline__ const double* st_rig<double>(const Dev& d) { return d.rig; }
template <> __device__ __forceinline__ const float* st_rig<float>(const Dev& d) { return d.rig_f; }
template <typename T> __device__ __forceinline__ const T* st_dc(const Dev& d);
template <> __device__ __forceinline__ const double* st_dc<double>(const Dev& d) { return d.dc; }
template <> __device__ __forceinline__ const float* st_dc<float>(const Dev& d) { return d.dc_f; }

// A camera's rig record (fx fy cx cy | R_cb | t_cb) and a pose (R | t) by 16-byte loads
// (records are 16-byte aligned in shared and global memory).
__device__ __forceinline__ void load_rig16(const float* rg, float r[16]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = reinterpret_cast<const float4*>(rg)[k];
    r[4 * k] = v.x; r[4 * k + 1] = v.y; r[4 * k + 2] = v.z; r[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void load_rig16(const double* rg, double r[16]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double2 v = reinterpret_cast<const double2*>(rg)[k];
    r[2 * k] = v.x; r[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void load_pose12(const float* P, float r[12]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 v = reinterpret_cast<const float4*>(P)[k];
    r[4 * k] = v.x; r[4 * k + 1] = v.y; r[4 * k + 2] = v.z; r[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void load_pose12(const double* P, double r[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 v = reinterpret_cast<const double2*>(P)[k];
    r[2 * k] = v.x; r[2 * k + 1] = v.y;
  }
}

// Residuals of the observations [o0, o1) of one (landmark, keyframe) pair at pose P
// and landmark pw; with JAC also the pair's camera-frame information M3 (sym 00 01 02 11
// 12 22) and a3 = sum w A^T r, A = d pi(X_c) / d X_b = J_pi R_cb.
template <typename T, bool JAC>
__device__ __forceinline__ void eval_pair(const T* __restrict__ P, const T* pw, int o0, int o1,
                                          const int32_t* __restrict__ obs_cam, const T* __restrict__ uv,
                                          const T* rig, T hub, T zmin, T X[3], T M3[6], T a3[3],
                                          PairStats<T>& st) {
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
    T rg[16];
    load_rig16(rig + obs_cam[n] * RIG_STRIDE, rg);
    const T fx = rg[0], fy = rg[1], cx = rg[2], cy = rg[3];
    const T* Rc = rg + 4;
    const T xc = fma(Rc[0], X[0], fma(Rc[1], X[1], fma(Rc[2], X[2], rg[13])));
    const T yc = fma(Rc[3], X[0], fma(Rc[4], X[1], fma(Rc[5], X[2], rg[14])));
    const T zc = fma(Rc[6], X[0], fma(Rc[7], X[1], fma(Rc[8], X[2], rg[15])));
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
    st.cost.add((T)0.5 * rho);
    st.sq.add(s);
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

// Candidate pose Exp(xi) T0 computed by a group of 16 lanes (lane gl of the group; both
// groups of the warp call it together; `act` false: shuffles only).  Lanes 0-8 produce the
// rotation entries, lanes 9-11 the translation, so each step is one warp instruction for
// all entries: on GB300 an FP64 instruction occupies its sub-partition's FP64 pipe for
// ~64 cycles whatever the number of active lanes.  For theta < 0.1 the coefficients
// A = sin t / t, B = (1 - cos t) / t^2, C = (t - sin t) / t^3 come from their Taylor
// series in t^2 up to t^10 (truncation < 2e-19), computed by lanes 0, 1, 2 in parallel;
// otherwise from sin and cos.  fixed: copy T0.
__constant__ double c_exp_series[3][6] = {
    {1.0, -1.0 / 6.0, 1.0 / 120.0, -1.0 / 5040.0, 1.0 / 362880.0, -1.0 / 39916800.0},
    {0.5, -1.0 / 24.0, 1.0 / 720.0, -1.0 / 40320.0, 1.0 / 3628800.0, -1.0 / 479001600.0},
    {1.0 / 6.0, -1.0 / 120.0, 1.0 / 5040.0, -1.0 / 362880.0, 1.0 / 39916800.0, -1.0 / 6227020800.0}};

__device__ __forceinline__ double sel3(const double v[3], int k) { return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]); }

__device__ __forceinline__ void pose_plus_group16(const double* T0, const double* xi, double* T1, float* F1,
                                                  bool act, bool fixed, int gl) {
  double ph[3] = {0.0, 0.0, 0.0}, rho[3] = {0.0, 0.0, 0.0};
  if (act && !fixed)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      rho[k] = xi[k];
      ph[k] = xi[3 + k];
    }
  const double th2 = fma(ph[2], ph[2], fma(ph[1], ph[1], ph[0] * ph[0]));
  // th2 >= 0: compare bit patterns as integers (no FP64 compare)
  const bool series = __double_as_longlong(th2) < __double_as_longlong(0.01);
  double v = 0.0;
  if (series) {
    const int w = gl % 3;
    v = c_exp_series[w][5];
#pragma unroll
    for (int k = 4; k >= 0; --k) v = fma(v, th2, c_exp_series[w][k]);
  }
  const double As = __shfl_sync(0xffffffffu, v, 0, 16);
  const double Bs = __shfl_sync(0xffffffffu, v, 1, 16);
  const double Cs = __shfl_sync(0xffffffffu, v, 2, 16);
  double A = As, B = Bs, C = Cs;
  if (!series) {
    const double th = sqrt(th2);
    double sn, cs;
    sincos(th, &sn, &cs);
    A = sn / th;
    B = (1.0 - cs) / th2;
    C = (th - sn) / (th2 * th);
  }
  // rotation part, lanes 0-8: entry (r, c) of Re = I + A [ph]x + B [ph]x^2
  const int r = gl < 9 ? gl / 3 : (gl < 12 ? gl - 9 : 0), c = gl < 9 ? gl % 3 : 0;
  double Kx = 0.0;                                 // [ph]x (r, c)
  if (r == 0 && c == 1) Kx = -ph[2];
  if (r == 0 && c == 2) Kx = ph[1];
  if (r == 1 && c == 0) Kx = ph[2];
  if (r == 1 && c == 2) Kx = -ph[0];
  if (r == 2 && c == 0) Kx = -ph[1];
  if (r == 2 && c == 1) Kx = ph[0];
  const double dg = (r == c) ? 1.0 : 0.0;
  const double K2 = fma(sel3(ph, r), sel3(ph, c), (r == c) ? -th2 : 0.0);   // [ph]x^2 = ph ph^T - th2 I
  const double Re = fma(A, Kx, fma(B, K2, dg));
  // R1 (r, c) = sum_m Re(r, m) T0(m, c), lanes 0-8
  const double e0 = __shfl_sync(0xffffffffu, Re, 3 * r, 16);
  const double e1 = __shfl_sync(0xffffffffu, Re, 3 * r + 1, 16);
  const double e2 = __shfl_sync(0xffffffffu, Re, 3 * r + 2, 16);
  double t00 = 0.0, t01 = 0.0, t02 = 0.0;
  if (act) {
    if (gl < 9) {
      t00 = T0[c];
      t01 = T0[3 + c];
      t02 = T0[6 + c];
    } else {
      t00 = T0[9];
      t01 = T0[10];
      t02 = T0[11];
    }
  }
  const double rt = fma(e2, t02, fma(e1, t01, e0 * t00));        // (Re T0)(r, c) or (Re t0)_r
  // translation, lanes 9-11: t1_r = (Re t0)_r + rho_r + B (ph x rho)_r + C (ph x (ph x rho))_r
  const int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
  const double p1 = sel3(ph, r1), p2 = sel3(ph, r2);
  const double u = fma(p1, sel3(rho, r2), -p2 * sel3(rho, r1));  // (ph x rho)_r on lanes 9-11
  const double u1 = __shfl_sync(0xffffffffu, u, 9 + r1, 16);
  const double u2 = __shfl_sync(0xffffffffu, u, 9 + r2, 16);
  const double w = fma(p1, u2, -p2 * u1);
  const double t1 = fma(C, w, fma(B, u, rt + sel3(rho, r)));
  if (act && gl < 12) {
    double o;
    if (fixed) o = T0[gl];
    else o = gl < 9 ? rt : t1;
    T1[gl] = o;
    if (F1) F1[gl] = (float)o;
  }
}

// Candidate poses of all keyframes: keyframe (CTA q of CS, 16-lane group g) = q + CS g,
// whole warps in step (every lane takes part in the group shuffles).
__device__ __forceinline__ void pose_candidates(const Dev& d, int q, int CS) {
  const int cur = d.ctrl->cur;
  const int groups = blockDim.x / 16;
  for (int base = 0; base < d.K; base += CS * groups) {
    const int a = base + (int)(threadIdx.x / 16) * CS + q;
    const bool act = a < d.K;
    const int ac = act ? a : 0;
    const int pb = d.kf_pb[ac];
    pose_plus_group16(d.pose[cur] + ac * POSE_STRIDE, d.dc + 6 * max(pb, 0), d.pose[cur ^ 1] + ac * POSE_STRIDE,
                      d.mixed ? d.pose_f[cur ^ 1] + ac * POSE_STRIDE : nullptr, act, pb < 0, threadIdx.x & 15);
  }
}

// Programmatic dependent launch: the iteration kernels are launched so that the next
// kernel's launch overlaps this one's tail; each waits for its predecessor's completion
// (and memory) before touching any memory, then lets its own successor launch.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// =================================================================== kernels

// Per-window device view for the batched kernels: the CTA copies its window's Dev into
// shared memory (CTA-uniform) and runs the same body as the single-window kernel.
__device__ __forceinline__ void load_dev(Dev& dst, const Dev* src) {
  static_assert(sizeof(Dev) % 4 == 0, "Dev size");
  for (int i = threadIdx.x; i < (int)(sizeof(Dev) / 4); i += blockDim.x)
    reinterpret_cast<int*>(&dst)[i] = reinterpret_cast<const int*>(src)[i];
  __syncthreads();
}

__device__ __forceinline__ void solve_init_body(const Dev& d, double lam0, double huber, double zmin, int iters, int reset,
                                                int refine) {
  Ctrl* c = d.ctrl;
  if (threadIdx.x == 0) {
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
    c->n_parts = 0;
    c->maxdiag_lm = 0ull;
    c->maxdiag_kf = 0ull;
    c->refine_max = refine;
    c->refined = 0;
    c->berr = CUDART_NAN;
  }
}

__global__ void k_solve_init(Dev d, double lam0, double huber, double zmin, int iters, int reset, int refine) { pdl_enter();
  solve_init_body(d, lam0, huber, zmin, iters, reset, refine);
}
__global__ void k_solve_init_b(const Dev* __restrict__ wins, double lam0, double huber, double zmin, int iters,
                               int reset, int refine) { pdl_enter();
  __shared__ Dev sd;
  load_dev(sd, wins + blockIdx.x);
  solve_init_body(sd, lam0, huber, zmin, iters, reset, refine);
}

// ------------------------------------------------------------ tile staging
// A linearisation tile's inputs are contiguous ranges (its pairs, their observations, its
// landmarks' pair offsets), so a CTA copies them into shared memory with asynchronous copies
// issued all at once: one memory latency per tile instead of a chain of dependent loads
// (pair -> observation -> camera) per thread.  Tiles with more than LIN_TILE_OBS
// observations read the observations in place.
__device__ __forceinline__ void cpa4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cpa_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
// one element of T (4 or 8 bytes)
template <typename T>
__device__ __forceinline__ void cpa_t(T* dst, const T* src) {
  if constexpr (sizeof(T) == 4) cpa4(dst, src); else cpa8(dst, src);
}

// Staged tile inputs, at the start of the dynamic shared memory after 128 doubles of
// reduction scratch: uv (2 LIN_TILE_OBS T), camera (LIN_TILE_OBS), pair keyframe and landmark
// (LIN_TILE_PAIRS each), pair observation offsets (LIN_TILE_PAIRS + 1, absolute) and the
// landmarks' pair offsets (LIN_TILE_LMS + 1, absolute).
template <typename T>
struct TileStage {
  T* uv;
  int *cam, *pkf, *plm, *pobs, *lmp;
  char* end;                                   // first byte after the staging area (16-aligned)
};
template <typename T>
__host__ __device__ constexpr size_t tile_stage_bytes() {
  return sizeof(T) * 2 * LIN_TILE_OBS + sizeof(int) * (LIN_TILE_OBS + 2 * LIN_TILE_PAIRS + (LIN_TILE_PAIRS + 4) +
                                                       (LIN_TILE_LMS + 4));
}
template <typename T>
__device__ __forceinline__ TileStage<T> tile_stage(double* smem) {
  TileStage<T> s;
  s.uv = reinterpret_cast<T*>(smem + 128);
  s.cam = reinterpret_cast<int*>(s.uv + 2 * LIN_TILE_OBS);
  s.pkf = s.cam + LIN_TILE_OBS;
  s.plm = s.pkf + LIN_TILE_PAIRS;
  s.pobs = s.plm + LIN_TILE_PAIRS;
  s.lmp = s.pobs + LIN_TILE_PAIRS + 4;
  s.end = reinterpret_cast<char*>(s.lmp + LIN_TILE_LMS + 4);
  return s;
}
// Issue the copies of the tile's pairs, landmark pair offsets and (if they fit) observations.
template <typename T>
__device__ __forceinline__ void stage_tile(const Dev& d, const LinTile& t, const TileStage<T>& s, bool obs) {
  const int np = t.p1 - t.p0, nl = t.l1 - t.l0, no = t.o1 - t.o0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    cpa4(s.pkf + i, d.pair_kf + t.p0 + i);
    cpa4(s.plm + i, d.pair_lm + t.p0 + i);
  }
  for (int i = threadIdx.x; i <= np; i += blockDim.x) cpa4(s.pobs + i, d.pair_obs + t.p0 + i);
  for (int i = threadIdx.x; i <= nl; i += blockDim.x) cpa4(s.lmp + i, d.lm_pair + t.l0 + i);
  if (obs) {
    const T* uv = reinterpret_cast<const T*>(d.obs_uv);
    for (int i = threadIdx.x; i < no; i += blockDim.x) {
      cpa4(s.cam + i, d.obs_cam + t.o0 + i);
      if constexpr (sizeof(T) == 4) cpa8(s.uv + 2 * i, uv + 2 * (size_t)(t.o0 + i));
      else cpa16(s.uv + 2 * i, uv + 2 * (size_t)(t.o0 + i));
    }
  }
}

// ----------------------------------------------------------------- k_lin
// Thread per (landmark, keyframe) pair; each pair writes its contributions to its own
// shared-memory slot, then owner threads sum them in pair order (per landmark: its
// contiguous pairs; per keyframe and component: the tile's pairs of that keyframe), so
// there are no atomics and the sums are reproducible.  The pair summaries leave through
// shared memory as one contiguous store.
template <typename T>
__host__ __device__ constexpr size_t lin_smem_bytes(int C) {
  return sizeof(double) * 128 + tile_stage_bytes<T>() +
         sizeof(T) * ((size_t)C * RIG_STRIDE + LIN_TILE_PAIRS * (21 + PAIR_LIN) + LIN_TILE_LMS * 3) +
         sizeof(int) * (2 * (K_MAX + 4) + LIN_TILE_PAIRS);
}
template <typename T>
__device__ __forceinline__ void k_lin_body(const Dev& d, int item) {
  Ctrl* ctrl = d.ctrl;
  if (!ctrl->need_lin) return;
  extern __shared__ __align__(16) double smem[];
  const LinTile tile = d.lin_tiles[item];
  const int nl = tile.l1 - tile.l0, np = tile.p1 - tile.p0;
  const bool obs_s = tile.o1 - tile.o0 <= LIN_TILE_OBS;
  double* s_red = smem;                                // 128
  const TileStage<T> sg = tile_stage<T>(smem);
  T* s_rig = reinterpret_cast<T*>(sg.end);             // C * 16
  T* s_pair = s_rig + d.C * RIG_STRIDE;                // LIN_TILE_PAIRS * 21
  T* s_plin = s_pair + LIN_TILE_PAIRS * 21;            // LIN_TILE_PAIRS * PAIR_LIN
  T* s_lm = s_plin + LIN_TILE_PAIRS * PAIR_LIN;        // LIN_TILE_LMS * 3
  int* s_kfo = reinterpret_cast<int*>(s_lm + LIN_TILE_LMS * 3);   // kf_n + 1 (absolute)
  int* s_kfs = s_kfo + K_MAX + 4;                      // kf_n: each keyframe's slot in kf_part
  int* s_kfi = s_kfs + K_MAX + 4;                      // kfi_n
  const int cur = ctrl->cur;
  const T* pose = st_pose<T>(d, cur);
  const T* lmp = st_lm<T>(d, cur);
  stage_tile<T>(d, tile, sg, obs_s);
  for (int i = threadIdx.x; i < 3 * nl; i += blockDim.x) cpa_t<T>(s_lm + i, lmp + 3 * (size_t)tile.l0 + i);
  for (int i = threadIdx.x; i <= tile.kf_n; i += blockDim.x) {
    cpa4(s_kfo + i, d.lin_kf_off + tile.kfl_off + i);
    cpa4(s_kfs + i, d.lin_kf_slot + tile.kfl_off + i);
  }
  for (int i = threadIdx.x; i < tile.kfi_n; i += blockDim.x) cpa4(s_kfi + i, d.lin_kf_idx + tile.kfi0 + i);
  const T* rig = st_rig<T>(d);
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = rig[i];
  cpa_wait_all();
  __syncthreads();

  const T hub = (T)ctrl->huber, zmin = (T)ctrl->zmin;
  PairStats<T> st;
  for (int qi = threadIdx.x; qi < np; qi += blockDim.x) {
    const int a = sg.pkf[qi], jl = sg.plm[qi] - tile.l0;
    T X[3], M3[6], a3[3], Pv[12];
    load_pose12(pose + a * POSE_STRIDE, Pv);
    if (obs_s)
      eval_pair<T, true>(Pv, s_lm + 3 * jl, sg.pobs[qi] - tile.o0, sg.pobs[qi + 1] - tile.o0,
                         sg.cam, sg.uv, s_rig, hub, zmin, X, M3, a3, st);
    else
      eval_pair<T, true>(Pv, s_lm + 3 * jl, sg.pobs[qi], sg.pobs[qi + 1], d.obs_cam,
                         reinterpret_cast<const T*>(d.obs_uv), s_rig, hub, zmin, X, M3, a3, st);
    T* pl = s_plin + qi * PAIR_LIN;
#pragma unroll
    for (int k = 0; k < 6; ++k) pl[k] = M3[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) pl[6 + k] = X[k];
    // landmark block: J_lm = A R  ->  Hll += R^T M3 R, g_l += R^T a3
    T M[9], G[9];
    const T* R = Pv;
    sym3_full(M3, M);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) G[r * 3 + c] = M[r * 3] * R[c] + M[r * 3 + 1] * R[3 + c] + M[r * 3 + 2] * R[6 + c];
    T* sl = s_pair + qi * 21;
    const int si[6] = {0, 0, 0, 1, 1, 2}, sj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int r = si[k], c = sj[k];
      sl[k] = R[r] * G[c] + R[3 + r] * G[3 + c] + R[6 + r] * G[6 + c];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) sl[6 + r] = R[r] * a3[0] + R[3 + r] * a3[1] + R[6 + r] * a3[2];
    // pose gradient B^T a3 = (a3, X x a3) and diag of B^T M3 B (fixed keyframe: unused)
    sl[9] = a3[0];
    sl[10] = a3[1];
    sl[11] = a3[2];
    sl[12] = X[1] * a3[2] - X[2] * a3[1];
    sl[13] = X[2] * a3[0] - X[0] * a3[2];
    sl[14] = X[0] * a3[1] - X[1] * a3[0];
    sl[15] = M3[0];
    sl[16] = M3[3];
    sl[17] = M3[5];
    sl[18] = M3[3] * X[2] * X[2] - 2 * M3[4] * X[1] * X[2] + M3[5] * X[1] * X[1];
    sl[19] = M3[0] * X[2] * X[2] - 2 * M3[2] * X[0] * X[2] + M3[5] * X[0] * X[0];
    sl[20] = M3[0] * X[1] * X[1] - 2 * M3[1] * X[0] * X[1] + M3[3] * X[0] * X[0];
  }
  if constexpr (sizeof(T) == 4) {                  // mixed: (hi, lo) float pairs, summed by k_decide
    DF v[2] = {st.cost.df(), st.sq.df()};
    DF o[2];
    block_sum_df_pair<2>(v, o, reinterpret_cast<float*>(s_red));   // contains barriers: slots complete
    const int nv = block_sum_i(st.nv, reinterpret_cast<int*>(s_red));
    const int ni = block_sum_i(st.ni, reinterpret_cast<int*>(s_red));
    if (threadIdx.x == 0) {
      float4* lp = reinterpret_cast<float4*>(d.lin_part + item * 4);
      lp[0] = make_float4(o[0].hi, o[0].lo, o[1].hi, o[1].lo);
      lp[1] = make_float4((float)nv, 0.0f, (float)ni, 0.0f);
    }
  } else {
    double v[4] = {st.cost.value(), st.sq.value(), (double)st.nv, (double)st.ni};
    block_sum4(v, s_red);                            // contains barriers: slots complete
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) d.lin_part[item * 4 + k] = v[k];
    }
  }
  {                                                  // pair summaries: one contiguous store
    T* out = reinterpret_cast<T*>(d.pair_lin) + (size_t)tile.p0 * PAIR_LIN;
    for (int e = threadIdx.x; e < np * PAIR_LIN; e += blockDim.x) out[e] = s_plin[e];
  }
  // per landmark and value (Hll 6, g_l 3): sum of its pairs (contiguous, in order); one
  // thread per (landmark, value), so the FP64 stores (and, on the mixed path, the FP32 -> FP64
  // conversions, each a full FP64-pipe slot) spread over the CTA's warps
  T mx = 0;
  for (int e = threadIdx.x; e < nl * 9; e += blockDim.x) {
    const int l = e / 9, k = e - 9 * l, j = tile.l0 + l;
    Acc<T> h;
    for (int q = sg.lmp[l]; q < sg.lmp[l + 1]; ++q) h.add(s_pair[(q - tile.p0) * 21 + k]);
    const bool dg = k == 0 || k == 3 || k == 5;
    if constexpr (sizeof(T) == 4) {                  // FP32 inputs of the landmark blocks
      const float r = h.rounded();
      if (k < 6) d.lm_H[j * 6 + k] = (double)r; else d.lm_g[j * 3 + k - 6] = (double)r;
      if (dg) mx = fmaxf(mx, r);
    } else {
      const double r = h.value();
      if (k < 6) d.lm_H[j * 6 + k] = r; else d.lm_g[j * 3 + k - 6] = r;
      if (dg) mx = fmax(mx, r);
    }
  }
  // per keyframe and component: sum over this tile's pairs of that keyframe, in pair
  // order (the tile's pairs of each keyframe are listed in lin_kf_idx)
  for (int e = threadIdx.x; e < tile.kf_n * 12; e += blockDim.x) {
    const int ka = e / 12, comp = e % 12;
    Acc<T> sum;
    for (int i = s_kfo[ka]; i < s_kfo[ka + 1]; ++i) sum.add(s_pair[s_kfi[i - tile.kfi0] * 21 + 9 + comp]);
    const size_t at = (size_t)s_kfs[ka] * 12 + comp;   // keyframe-major slot
    if constexpr (sizeof(T) == 4)
      reinterpret_cast<float2*>(d.kf_part)[at] = make_float2(sum.s, -sum.c);
    else
      d.kf_part[at] = sum.value();
  }
  double mxd;
  if constexpr (sizeof(T) == 4)
    mxd = (double)block_max_f(mx, reinterpret_cast<float*>(s_red));
  else
    mxd = block_max(mx, s_red);
  if (threadIdx.x == 0 && mxd > 0.0)
    atomicMax(&ctrl->maxdiag_lm, (unsigned long long)__double_as_longlong(mxd));
}

template <typename T>
// Mixed path: four CTAs per SM (the staged tile takes ~55 KB of shared memory at 32 cameras).
__global__ void __launch_bounds__(LIN_THREADS, sizeof(T) == 4 ? 4 : 2) k_lin(Dev d) { pdl_enter(); k_lin_body<T>(d, blockIdx.x); }
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_lin_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_lin_body<T>(sd, it.y);
}

// g_p and diag(Hpp) of keyframe `item`: fixed-order sum of the covering tiles' partials,
// which are contiguous (keyframe-major slots of 12 values).  Thread t reads the values t + 384 i
// (coalesced; its component is t mod 12, its slots t / 12 + 32 i) in eight interleaved sums
// (i mod 8, combined pairwise); warp c then adds component c's 32 thread sums by a butterfly.
__device__ __forceinline__ void k_kf_reduce_body(const Dev& d, int item) {
  __shared__ double s_v[384];
  __shared__ DF s_vf[384];
  const int a = item, tid = threadIdx.x;
  const int n = (d.kf_tiles_off[a + 1] - d.kf_tiles_off[a]) * 12;
  const size_t base = (size_t)d.kf_tiles_off[a] * 12;
  const bool mixed = d.mixed != 0;
  if (mixed) {                                       // tile partials are (hi, lo) floats
    const float2* kp = reinterpret_cast<const float2*>(d.kf_part) + base;
    DF s8[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] = DF{0.0f, 0.0f};
    int t = tid;
    for (; t + 7 * 384 < n; t += 8 * 384) {
      float2 x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = kp[t + 384 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) s8[u] = df_add(s8[u], DF{x[u].x, x[u].y});
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (t + 384 * u < n) {
        const float2 x = kp[t + 384 * u];
        s8[u] = df_add(s8[u], DF{x.x, x.y});
      }
    s_vf[(tid % 12) * 32 + tid / 12] = df_add(df_add(df_add(s8[0], s8[1]), df_add(s8[2], s8[3])),
                                              df_add(df_add(s8[4], s8[5]), df_add(s8[6], s8[7])));
  } else {
    const double* kp = d.kf_part + base;
    double s8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int t = tid;
    for (; t + 7 * 384 < n; t += 8 * 384) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = kp[t + 384 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) s8[u] += x[u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (t + 384 * u < n) s8[u] += kp[t + 384 * u];
    s_v[(tid % 12) * 32 + tid / 12] = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;        // warp = component (12)
  double v;
  if (mixed) {
    const DF x = warp_sum_df(s_vf[warp * 32 + lane]);
    v = (double)x.hi + (double)x.lo;
  } else {
    v = warp_sum(s_v[warp * 32 + lane]);
  }
  if (lane == 0) {
    if (warp < 6) {
      d.kf_gp[a * 6 + warp] = v;
    } else {
      d.kf_dp[a * 6 + warp - 6] = v;
      if (v > 0.0) atomicMax(&d.ctrl->maxdiag_kf, (unsigned long long)__double_as_longlong(v));
    }
  }
}

__global__ void __launch_bounds__(384) k_kf_reduce(Dev d) { pdl_enter(); k_kf_reduce_body(d, blockIdx.x); }
__global__ void __launch_bounds__(384) k_kf_reduce_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_kf_reduce_body(sd, it.y);
}

// Closed-form inverse of V_j = Hll_j + lam D_l,j (adjugate / determinant), stored with tau
// in lm_Vinv.  Mixed path only: Hll_j is summed from FP32 products, so information below
// ~2^-23 of its trace is rounding noise (a landmark drifting to infinity along its ray has
// an eigenvalue ~1e-15 of the others).  If V_j then fails the positive-definite test, the
// block is retried with tau = 2^-20 tr(Hll_j) added to its diagonal; tau enters the
// predicted reduction in k_backsub.  The FP64 path never adds tau.
template <typename T>
__device__ void landmark_vinv(const Dev& d, int j, double lam, double floor_, double inv[6]) {
  const double* H = d.lm_H + 6 * j;
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
    d.ctrl->nonpd = 1;
  }
  if (sizeof(T) == 4) {                              // the mixed path reads V^-1 in FP32
    float* o = reinterpret_cast<float*>(d.lm_Vinv) + j * VINV_STRIDE;
    for (int k = 0; k < 6; ++k) o[k] = (float)inv[k];
    o[6] = (float)tau;
  } else {
    for (int k = 0; k < 6; ++k) d.lm_Vinv[j * VINV_STRIDE + k] = inv[k];
    d.lm_Vinv[j * VINV_STRIDE + 6] = tau;
  }
}

// Per pair: W = J_pose^T W J_lm = [G; [X]x G] with G = M3 R (6 x 3), Y = W V^-1, the pair's
// diagonal-block term U - Y W^T (U = B^T M3 B, lower 21) and Y g_l.
template <typename T>
__device__ __forceinline__ void pair_schur_terms(const T* pl, const T* R_pose, const T* vinv6,
                                                 const T* gl3, T W[18], T Y[18], T Dg[21], T bY[6]) {
  T M3[6], X[3], M[9], R[9], G[9];
#pragma unroll
  for (int k = 0; k < 6; ++k) M3[k] = pl[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) X[k] = pl[6 + k];
  sym3_full(M3, M);
#pragma unroll
  for (int k = 0; k < 9; ++k) R[k] = R_pose[k];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) G[r * 3 + c] = M[r * 3] * R[c] + M[r * 3 + 1] * R[3 + c] + M[r * 3 + 2] * R[6 + c];
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
    for (int k = 0; k < 6; ++k) s6[k] = vinv6[k];
    sym3_full(s6, Vi);
  }
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Y[r * 3 + c] = W[r * 3] * Vi[c] + W[r * 3 + 1] * Vi[3 + c] + W[r * 3 + 2] * Vi[6 + c];
  T U[36];
  pose_info(M, X, U);
  int k = 0;
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c <= r; ++c, ++k)
      Dg[k] = U[r * 6 + c] - (Y[r * 3] * W[c * 3] + Y[r * 3 + 1] * W[c * 3 + 1] + Y[r * 3 + 2] * W[c * 3 + 2]);
  const T g0 = gl3[0], g1 = gl3[1], g2 = gl3[2];
#pragma unroll
  for (int r = 0; r < 6; ++r) bY[r] = Y[r * 3] * g0 + Y[r * 3 + 1] * g1 + Y[r * 3 + 2] * g2;
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

// Tiles whose landmarks span more than SPAN_MAX free keyframes: every block product is
// added straight into the global reduced camera system with atomics (rare in sliding
// windows; not bit-reproducible).
template <typename T>
__device__ __forceinline__ void k_schur_direct_body(const Dev& d, int item) {
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
  const SchurTile tile = d.direct_tiles[item];
  const int nl = tile.l1 - tile.l0;
  const int n_c = d.n_c;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);
  const int rows = 6 * tile.span;
  if (!tile.direct) {
    for (int i = threadIdx.x; i < rows * (rows + 1) / 2; i += blockDim.x) s_win[i] = 0.0;
    for (int i = threadIdx.x; i < rows; i += blockDim.x) s_b[i] = 0.0;
  }
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int j = tile.l0 + l;
    double inv[6];
    landmark_vinv<T>(d, j, lam, floor_, inv);
    for (int k = 0; k < 6; ++k) s_vinv[l * 6 + k] = inv[k];
    for (int k = 0; k < 3; ++k) s_gl[l * 3 + k] = d.lm_g[j * 3 + k];
  }
  for (int l = threadIdx.x; l <= nl; l += blockDim.x) s_blk[l] = d.lm_blk[tile.l0 + l] - tile.b0;
  __syncthreads();

  auto acc_S = [&](int pr, int pc, int r, int c, double v) {
    if (tile.direct) {
      const int gr = 6 * pr + r, gc = 6 * pc + c;  // a lower entry; S is kept symmetric
      atomicAdd(d.S + (size_t)gr * n_c + gc, v);
      if (gr != gc) atomicAdd(d.S + (size_t)gc * n_c + gr, v);
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

  // phase 4: the window (and its part of b) as this tile's partial, summed per RCS block
  // in a fixed order by k_rcs_reduce
  if (!tile.direct) {
    const int nw_ = rows * (rows + 1) / 2;
    double* out = d.schur_part + tile.part_off;
    for (int i = threadIdx.x; i < nw_; i += blockDim.x) out[i] = s_win[i];
    for (int i = threadIdx.x; i < rows; i += blockDim.x) out[nw_ + i] = s_b[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(SCHUR_THREADS) k_schur_direct(Dev d) { pdl_enter(); k_schur_direct_body<T>(d, blockIdx.x); }
template <typename T>
__global__ void __launch_bounds__(SCHUR_THREADS) k_schur_direct_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_schur_direct_body<T>(sd, it.y);
}

// ------------------------------------------------------------ k_schur_group
// Reduced camera system from a tile of landmarks that share the same window of free
// keyframes [k_lo, k_lo + span): their contributions to that window of S,
//   S_ab += sum_j (U_ja - Y_ja W_ja^T) (a = b),   S_ab -= sum_j Y_ja W_jb^T (a > b),
//   b_a  += sum_j Y_ja g_l,j,
// (a keyframe of the window that does not observe a landmark contributes zero blocks).
// Register-blocked: a work item is half of a 6x6 block (a, b), a >= b (rows 3h..3h+2),
// accumulated over a share of the tile's landmarks (G groups split the landmarks when the
// window has few blocks; windows with more than 128 blocks take several passes over the
// landmarks).  Per landmark an off-diagonal item reads three rows of Y_a and all of W_b
// (9 short vectors) and does 54 FMAs.  Sums run per staged chunk in T, then into a
// compensated (Kahan) accumulator on the mixed path or a plain FP64 one; groups are
// combined in a fixed order and the window is written as the tile's partial, summed over
// tiles by k_rcs_reduce.  About 100 registers on the mixed path: two CTAs per SM.
constexpr int kStage = 76;         // per (landmark, block): Y[6][4] W[6][4] Dg[21] bY[6] pad
// Threads of a group Schur CTA.  512 threads on the mixed path (the 2 x 253 half-block items of
// the widest window in one pass) capped the registers at 128 and ran slower at 100 keyframes
// x 32 cameras (0.45 against 0.38 ms) than two 256-thread CTAs per SM with two passes.
template <typename T>
__host__ __device__ constexpr int group_threads() { return 256; }
template <typename T>
struct GroupChunk {
  static constexpr int value = sizeof(T) == 4 ? 16 : 8;
};

// Per-tile tables in front of the staging area: the landmarks' pair offsets, the window's
// rotations and each keyframe's window slot (16-byte multiples).
constexpr size_t kGroupLpBytes = ((SCHUR_TILE_LMS + 1) * sizeof(int) + 15) / 16 * 16;
__host__ __device__ constexpr size_t group_rot_bytes(size_t t) { return (SPAN_MAX * 9 * t + 15) / 16 * 16; }
constexpr size_t kGroupSlotBytes = K_MAX;

size_t group_smem_bytes(int max_span, bool mixed) {
  const size_t t = mixed ? 4 : 8;
  const int ch = mixed ? 16 : 8;
  // the staging area also holds the groups' partials for the combine: <= 256 items x 18 x 8 B
  const size_t stage = std::max((size_t)ch * max_span * kStage * t,
                                (size_t)(mixed ? group_threads<float>() : group_threads<double>()) * 18 * 8);
  return sizeof(double) * 64 + t * (size_t)SCHUR_TILE_LMS * 9 + kGroupLpBytes + group_rot_bytes(t) +
         kGroupSlotBytes + stage;
}

template <typename T>
__device__ __forceinline__ void load_row3(const T* p, T& x, T& y, T& z);
template <>
__device__ __forceinline__ void load_row3<float>(const float* p, float& x, float& y, float& z) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  x = v.x;
  y = v.y;
  z = v.z;
}
template <>
__device__ __forceinline__ void load_row3<double>(const double* p, double& x, double& y, double& z) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  x = v.x;
  y = v.y;
  z = p[2];
}

// Half-block work items: off-diagonal (a > b): rows 3h..3h+2 x 6 columns, index
// (r - 3h) * 6 + c.  Diagonal, h = 0: lower entries of rows 0-2 (6) then b rows 0-2 (3);
// h = 1: lower entries of rows 3-5 (15) then b rows 3-5 (3).  In the staged Dg[21] the
// lower entry (r, c) is r(r+1)/2 + c, so both halves are contiguous runs followed by bY.
// The tile's partial is written in this layout, [half block][18].

template <typename T>
__device__ __forceinline__ void k_schur_group_body(const Dev& d, int item) {
  constexpr int CH = GroupChunk<T>::value;
  constexpr bool kKahan = sizeof(T) == 4;
  using Out = typename std::conditional<sizeof(T) == 4, DF, double>::type;
  extern __shared__ __align__(16) double smem[];
  double* s_red = smem;                               // 64
  T* s_vinv = reinterpret_cast<T*>(s_red + 64);       // SCHUR_TILE_LMS * 6
  T* s_gl = s_vinv + SCHUR_TILE_LMS * 6;              // SCHUR_TILE_LMS * 3
  int* s_lp = reinterpret_cast<int*>(s_gl + SCHUR_TILE_LMS * 3);   // pair offsets of the tile's landmarks
  T* s_rot = reinterpret_cast<T*>(reinterpret_cast<char*>(s_lp) + kGroupLpBytes);   // window rotations
  signed char* s_slot = reinterpret_cast<signed char*>(s_rot) + group_rot_bytes(sizeof(T));   // per keyframe
  T* s_stg = reinterpret_cast<T*>(s_slot + kGroupSlotBytes);   // CH * max_span * kStage
  __shared__ unsigned s_mask[16];                     // per staged landmark: keyframes present
  const SchurTile tile = d.schur_tiles[item];
  const int nl = tile.l1 - tile.l0;
  const int span = tile.span;
  const double lam = d.ctrl->lam;
  const double floor_ = diag_floor(d, s_red);
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const int j = tile.l0 + l;
    double inv[6];
    landmark_vinv<T>(d, j, lam, floor_, inv);
    for (int k = 0; k < 6; ++k) s_vinv[l * 6 + k] = (T)inv[k];
    for (int k = 0; k < 3; ++k) s_gl[l * 3 + k] = (T)d.lm_g[j * 3 + k];
  }
  if (span == 0) return;                             // landmarks seen only by the fixed keyframe
  const T* pose = st_pose<T>(d, d.ctrl->cur);
  // per tile, once: pair offsets, window slot of each keyframe (-1: fixed or outside) and
  // the window's rotations, so that a chunk's pairs need only independent loads
  for (int i = threadIdx.x; i <= nl; i += blockDim.x) s_lp[i] = d.lm_pair[tile.l0 + i];
  for (int a = threadIdx.x; a < d.K; a += blockDim.x) {
    const int pb = d.kf_pb[a];
    s_slot[a] = (signed char)(pb >= tile.k_lo && pb < tile.k_lo + span ? pb - tile.k_lo : -1);
  }
  for (int e = threadIdx.x; e < span * 9; e += blockDim.x) {
    const int pbk = tile.k_lo + e / 9, a = pbk < d.fixed_kf ? pbk : pbk + 1;
    s_rot[e] = pose[a * POSE_STRIDE + e % 9];
  }
  const int nblk = span * (span + 1) / 2;            // <= 253 (span <= SPAN_MAX)
  const int n_half = 2 * nblk;
  constexpr int NT = group_threads<T>();
  const int G = max(1, min(CH, NT / n_half));
  const int n_items = n_half * G;                    // > NT only when G == 1
  Out* out = reinterpret_cast<Out*>(d.schur_part) + tile.part_off;
  // this thread's first pair of the next chunk, loaded while the current chunk's products run
  int pf_a = 0, pf_l = 0;
  T pf_v[PAIR_LIN];
  auto prefetch = [&](int c0n) {
    const int q = s_lp[c0n] + threadIdx.x;
    if (q < s_lp[min(c0n + CH, nl)]) {
      pf_a = d.pair_kf[q];
      pf_l = d.pair_lm[q] - tile.l0;
      const T* plq = reinterpret_cast<const T*>(d.pair_lin) + (size_t)q * PAIR_LIN;
#pragma unroll
      for (int k = 0; k < PAIR_LIN; ++k) pf_v[k] = plq[k];
    }
  };
  __syncthreads();                                   // s_lp complete
  prefetch(0);
  for (int it0 = 0; it0 < n_items; it0 += NT) {     // passes
    const int t = it0 + threadIdx.x;
    const bool working = t < n_items;
    const int hb = t % n_half, g = t / n_half;
    const int blk = hb >> 1, h = hb & 1;
    int ba = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
    while (ba * (ba + 1) / 2 > blk) --ba;
    while ((ba + 1) * (ba + 2) / 2 <= blk) ++ba;
    const int bb = blk - ba * (ba + 1) / 2;
    const bool diag = ba == bb;
    T acc[18], cmp[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      acc[k] = 0;
      cmp[k] = 0;
    }
    for (int c0 = 0; c0 < nl; c0 += CH) {
      const int nc = min(CH, nl - c0);
      __syncthreads();                               // previous chunk consumed
      if (threadIdx.x < CH) s_mask[threadIdx.x] = 0u;
      __syncthreads();
      // stage each pair's terms as one 76-value record (16-byte stores) and mark it present
      const int q0 = s_lp[c0], q1 = s_lp[c0 + nc];
      for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
        int a, l;                                    // keyframe, index of the landmark in the tile
        T pv[PAIR_LIN];
        if (q == q0 + (int)threadIdx.x) {            // prefetched
          a = pf_a;
          l = pf_l;
#pragma unroll
          for (int k = 0; k < PAIR_LIN; ++k) pv[k] = pf_v[k];
        } else {                                     // loaded before the slot test: no load chain
          a = d.pair_kf[q];
          l = d.pair_lm[q] - tile.l0;
          const T* plq = reinterpret_cast<const T*>(d.pair_lin) + (size_t)q * PAIR_LIN;
#pragma unroll
          for (int k = 0; k < PAIR_LIN; ++k) pv[k] = plq[k];
        }
        const int w = s_slot[a];
        if (w < 0) continue;
        T W[18], Y[18], Dg[21], bY[6];
        pair_schur_terms<T>(pv, s_rot + w * 9, s_vinv + l * 6, s_gl + l * 3, W, Y, Dg, bY);
        T* st = s_stg + ((l - c0) * span + w) * kStage;
        if constexpr (sizeof(T) == 4) {              // 19 16-byte stores per record
          float4* s4 = reinterpret_cast<float4*>(st);
#pragma unroll
          for (int r = 0; r < 6; ++r) {
            s4[r] = make_float4(Y[r * 3], Y[r * 3 + 1], Y[r * 3 + 2], 0.f);
            s4[6 + r] = make_float4(W[r * 3], W[r * 3 + 1], W[r * 3 + 2], 0.f);
          }
#pragma unroll
          for (int k = 0; k < 5; ++k) s4[12 + k] = make_float4(Dg[4 * k], Dg[4 * k + 1], Dg[4 * k + 2], Dg[4 * k + 3]);
          s4[17] = make_float4(Dg[20], bY[0], bY[1], bY[2]);
          s4[18] = make_float4(bY[3], bY[4], bY[5], 0.f);
        } else {
#pragma unroll
          for (int r = 0; r < 6; ++r) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              st[r * 4 + k] = Y[r * 3 + k];
              st[24 + r * 4 + k] = W[r * 3 + k];
            }
          }
#pragma unroll
          for (int k = 0; k < 21; ++k) st[48 + k] = Dg[k];
#pragma unroll
          for (int r = 0; r < 6; ++r) st[69 + r] = bY[r];
        }
        atomicOr(&s_mask[l - c0], 1u << w);
      }
      {                                              // the next chunk (or the next pass's first)
        const int cn = c0 + CH < nl ? c0 + CH : (it0 + NT < n_items ? 0 : -1);
        if (cn >= 0) prefetch(cn);
      }
      __syncthreads();
      if (working) {
        T part[18];
#pragma unroll
        for (int k = 0; k < 18; ++k) part[k] = 0;
        for (int lr = g; lr < nc; lr += G) {
          // a block takes a landmark's term only if it observes both keyframes (records of
          // the others are never read, so they need no zeroing); a track covers consecutive
          // keyframes, so a warp's items, which share ba, mostly skip together
          if (!((s_mask[lr] >> ba) & (s_mask[lr] >> bb) & 1u)) continue;
          const T* base = s_stg + lr * span * kStage;
          if (diag) {
            const T* st = base + ba * kStage;
            if (h == 0) {
#pragma unroll
              for (int k = 0; k < 6; ++k) part[k] += st[48 + k];
#pragma unroll
              for (int k = 0; k < 3; ++k) part[6 + k] += st[69 + k];
            } else {
#pragma unroll
              for (int k = 0; k < 15; ++k) part[k] += st[48 + 6 + k];
#pragma unroll
              for (int k = 0; k < 3; ++k) part[15 + k] += st[72 + k];
            }
          } else {
            const T* Ya = base + ba * kStage + 12 * h;
            const T* Wb = base + bb * kStage + 24;
            T w[18];
#pragma unroll
            for (int c = 0; c < 6; ++c) load_row3<T>(Wb + 4 * c, w[3 * c], w[3 * c + 1], w[3 * c + 2]);
#pragma unroll
            for (int r = 0; r < 3; ++r) {
              T y0, y1, y2;
              load_row3<T>(Ya + 4 * r, y0, y1, y2);
#pragma unroll
              for (int c = 0; c < 6; ++c)
                part[r * 6 + c] = fma(-y0, w[3 * c], fma(-y1, w[3 * c + 1], fma(-y2, w[3 * c + 2], part[r * 6 + c])));
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 18; ++k) {
          if (kKahan) {                              // acc - cmp is the running sum
            const T yk = part[k] - cmp[k];
            const T sm = acc[k] + yk;
            cmp[k] = (sm - acc[k]) - yk;
            acc[k] = sm;
          } else {
            acc[k] += part[k];
          }
        }
      }
    }
    if (G == 1) {
      // one group: each item writes its 18 values, contiguous ([half block][18])
      if (working) {
#pragma unroll
        for (int k = 0; k < 18; ++k) {
          if constexpr (sizeof(T) == 4)
            out[hb * 18 + k] = DF{(float)acc[k], -(float)cmp[k]};
          else
            out[hb * 18 + k] = (double)acc[k];
        }
      }
    } else {
      // several groups (single pass): every group's values in the staging area
      // [group][half block][18], combined by a fixed pairwise tree (group g takes g + step),
      // then group 0's written as it is
      Out* s_out = reinterpret_cast<Out*>(s_stg);
      __syncthreads();
      if (working) {
#pragma unroll
        for (int k = 0; k < 18; ++k) {
          if constexpr (sizeof(T) == 4)
            s_out[(g * n_half + hb) * 18 + k] = DF{(float)acc[k], -(float)cmp[k]};
          else
            s_out[(g * n_half + hb) * 18 + k] = (double)acc[k];
        }
      }
      for (int step = 1; step < G; step *= 2) {
        __syncthreads();
        if (working && g % (2 * step) == 0 && g + step < G) {
          Out* dst = s_out + (g * n_half + hb) * 18;
          const Out* src = s_out + ((g + step) * n_half + hb) * 18;
#pragma unroll
          for (int k = 0; k < 18; ++k) {
            if constexpr (sizeof(T) == 4)
              dst[k] = df_add(dst[k], src[k]);
            else
              dst[k] += src[k];
          }
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n_half * 18; e += blockDim.x) out[e] = s_out[e];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(group_threads<T>(), sizeof(T) == 4 ? 2 : 1) k_schur_group(Dev d) { pdl_enter();
  k_schur_group_body<T>(d, blockIdx.x);
}
template <typename T>
__global__ void __launch_bounds__(group_threads<T>(), sizeof(T) == 4 ? 2 : 1)
    k_schur_group_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_schur_group_body<T>(sd, it.y);
}

// Block (a, b), a >= b, of the reduced camera system (and b_a when a == b): fixed-order sum
// of the window partials of the Schur tiles covering it, assigned (zero when no tile covers
// it); the direct tiles' atomics are added after this kernel.
__device__ __forceinline__ void k_rcs_reduce_body(const Dev& d, int item) {
  // A covering tile's partial of block (a, b) is 36 consecutive values (two half blocks of
  // 18, k_schur_group's layout) starting at blk_part_at[i].  Thread (g, e), g < 7, e < 36,
  // sums value e over the covering tiles g, g + 7, ... (four interleaved sums, combined
  // pairwise); the seven group sums are then added in order g = 0..6.
  __shared__ double s_sum[7 * 36];
  __shared__ DF s_sumf[7 * 36];
  const int blk = item;
  const int t0 = d.blk_tiles_off[blk], t1 = d.blk_tiles_off[blk + 1];
  int a = (int)((sqrtf(8.0f * (float)blk + 1.0f) - 1.0f) * 0.5f);
  while (a * (a + 1) / 2 > blk) --a;
  while ((a + 1) * (a + 2) / 2 <= blk) ++a;
  const int b = blk - a * (a + 1) / 2;
  const bool mixed = d.mixed != 0;
  const int g = threadIdx.x / 36, e = threadIdx.x % 36;
  const int* at = d.blk_part_at;
  if (g < 7) {
    if (mixed) {
      const DF* sp = reinterpret_cast<const DF*>(d.schur_part);
      DF s4[4] = {DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}, DF{0.0f, 0.0f}};
      int t = t0 + g;
      for (; t + 3 * 7 < t1; t += 4 * 7) {
        DF x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = sp[at[t + 7 * u] + e];
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] = df_add(s4[u], x[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (t + 7 * u < t1) s4[u] = df_add(s4[u], sp[at[t + 7 * u] + e]);
      s_sumf[g * 36 + e] = df_add(df_add(s4[0], s4[1]), df_add(s4[2], s4[3]));
    } else {
      double s4[4] = {0.0, 0.0, 0.0, 0.0};
      int t = t0 + g;
      for (; t + 3 * 7 < t1; t += 4 * 7) {
        double x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = d.schur_part[at[t + 7 * u] + e];
#pragma unroll
        for (int u = 0; u < 4; ++u) s4[u] += x[u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (t + 7 * u < t1) s4[u] += d.schur_part[at[t + 7 * u] + e];
      s_sum[g * 36 + e] = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    }
  }
  __syncthreads();
  if (threadIdx.x >= 36) return;
  double sum;
  if (mixed) {
    DF x = s_sumf[e];
#pragma unroll
    for (int k = 1; k < 7; ++k) x = df_add(x, s_sumf[k * 36 + e]);
    sum = (double)x.hi + (double)x.lo;
  } else {
    sum = s_sum[e];
#pragma unroll
    for (int k = 1; k < 7; ++k) sum += s_sum[k * 36 + e];
  }
  // value e -> entry: off-diagonal blocks row-major (r = e / 6, c = e % 6); diagonal blocks
  // [lower entries of rows 0-2 (6), b rows 0-2 (3), unused (9) | lower entries of rows 3-5
  // (15), b rows 3-5 (3)], lower entry il = r (r + 1) / 2 + c
  int r, c;
  if (a != b) {
    r = e / 6;
    c = e % 6;
  } else {
    int il;
    if (e < 6) {
      il = e;
    } else if (e < 9) {
      d.bS[6 * a + (e - 6)] = sum;
      return;
    } else if (e < 18) {
      return;
    } else if (e < 33) {
      il = 6 + (e - 18);
    } else {
      d.bS[6 * a + 3 + (e - 33)] = sum;
      return;
    }
    r = 0;
    while ((r + 1) * (r + 2) / 2 <= il) ++r;
    c = il - r * (r + 1) / 2;
  }
  const int gr = 6 * a + r, gc = 6 * b + c;          // both triangles: rows read contiguously
  d.S[(size_t)gr * d.n_c + gc] = sum;
  if (gr != gc) d.S[(size_t)gc * d.n_c + gr] = sum;
}

__global__ void __launch_bounds__(256) k_rcs_reduce(Dev d) { pdl_enter(); k_rcs_reduce_body(d, d.act_blk[blockIdx.x]); }
__global__ void __launch_bounds__(256) k_rcs_reduce_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_rcs_reduce_body(sd, it.y);
}

// ----------------------------------------------------------------- k_chol
// Dense FP64 Cholesky of the damped reduced camera system, then the two triangular
// solves.  One CTA; the matrix lives in shared memory when it fits (SMEM) else in global.
template <bool SMEM>
__device__ __forceinline__ void k_chol_body(const Dev& d, int item) {
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
    ctrl->pred_part[0] = v[0];
    ctrl->step2_part[0] = v[1];
    ctrl->n_parts = 1;
  }
  __syncthreads();
  pose_candidates(d, 0, 1);
  if (d.mixed)
    for (int i = threadIdx.x; i < d.n_c; i += blockDim.x) d.dc_f[i] = (float)d.dc[i];
}

template <bool SMEM>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol(Dev d) { pdl_enter(); k_chol_body<SMEM>(d, blockIdx.x); }
template <bool SMEM>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_chol_body<SMEM>(sd, it.y);
}

// ---------------------------------------------------------- k_chol_cluster
// The damped reduced camera system A = S + lam D_p (n_c x n_c, FP64) factored A = L L^T
// by a thread-block cluster of CS CTAs, then dc = A^-1 (b - g_p).
//
// Layout: A is padded to NP = 8 * NB rows (identity in the padding) and split into 8-row
// block rows; block row r lives in the shared memory of CTA r % CS.  Right-looking by
// 8-column panels.  Step k (the diagonal block L_kk already factored and pushed, with the
// reciprocals of its diagonal, to every CTA):
//   1. every CTA solves its block rows r > k against L_kk (L_rk = A_rk L_kk^-T); CTA 0
//      does the same for the right-hand side, carried as an extra row, which fuses the
//      forward substitution L y = rhs into the factorisation; each CTA pushes its new
//      panel blocks L_rk to every CTA;                                   cluster barrier
//   2. look-ahead: the owner of block k+1 first updates and factors its diagonal block and
//      pushes it; then every CTA applies A_rc -= L_rk L_ck^T to its block rows (c in
//      (k, r]) and CTA 0 updates the right-hand side;                    cluster barrier
// On GB300 a dependent FP64 FMA takes ~64 cycles, a divide ~430 and a square root ~680,
// so the pivot chain uses rsqrt and multiplications, and the diagonal blocks' inverses
// are formed once, in parallel, after the factorisation.
// Backward substitution L^T x = y runs from the last block: the owner of block k sums the
// contributions other CTAs pushed into its slots (fixed order), multiplies by L_kk^-T,
// writes x_k, and pushes the running contributions of block row k to the owners of blocks
// < k.  All pushes are plain DSMEM stores made visible by the next cluster barrier.
constexpr int kCB = 8;
constexpr size_t kClusterSmemMaxBytes = 220 * 1024;   // dynamic shared memory of one Cholesky CTA

struct CholSmem {
  int NP, NB, nlb, CS;
  size_t rows_len;                                 // packed lower block rows, max over CTAs
  __host__ __device__ size_t rows_off() const { return 0; }
  __host__ __device__ size_t panel_off() const { return rows_off() + rows_len; }
  __host__ __device__ size_t lkk_off() const { return panel_off() + (size_t)2 * NB * kCB * kCB; }   // two panels
  __host__ __device__ size_t y_off() const { return lkk_off() + 2 * (kCB * kCB + kCB); }   // two L_kk buffers
  __host__ __device__ size_t acc_off() const { return y_off() + NP; }
  __host__ __device__ size_t contrib_off() const { return acc_off() + NP; }
  __host__ __device__ size_t linv_off() const { return contrib_off() + (size_t)nlb * CS * kCB; }
  __host__ __device__ size_t rdiag_off() const { return linv_off() + (size_t)nlb * kCB * kCB; }
  __host__ __device__ size_t nrm_off() const { return rdiag_off() + (size_t)nlb * kCB; }
  __host__ __device__ size_t red_off() const { return nrm_off() + (size_t)CS * 4; }
  __host__ __device__ size_t flag_off() const { return red_off() + 128; }
  // gathered factor on CTA 0 (small systems): packed lower block rows of all of L, then
  // the inverses of all diagonal blocks
  __host__ __device__ size_t gl_len() const { return (size_t)32 * NB * (NB + 1); }
  __host__ __device__ size_t gl_off() const { return flag_off() + 8; }
  __host__ __device__ size_t glinv_off() const { return gl_off() + gl_len(); }
  __host__ __device__ size_t base_doubles() const { return flag_off() + 8; }
  __host__ __device__ size_t doubles() const {
    return gather ? glinv_off() + (size_t)NB * kCB * kCB : base_doubles();
  }
  bool gather;                                     // backward substitution on CTA 0
  // CTA q's lb-th block row is block row r = q + lb CS; only its columns [0, 8(r+1)) are
  // stored (the lower triangle), row-major with width 8(r+1), one block row after another.
  __host__ __device__ size_t row_off(int q, int lb) const {
    return (size_t)kCB * kCB * ((size_t)lb * (q + 1) + (size_t)CS * lb * (lb - 1) / 2);
  }
  __host__ __device__ int row_width(int q, int lb) const { return kCB * (q + lb * CS + 1); }
};

__host__ __device__ inline CholSmem chol_layout(int n_c, int CS) {
  CholSmem L;
  L.NB = (n_c + kCB - 1) / kCB;
  L.NP = L.NB * kCB;
  L.nlb = (L.NB + CS - 1) / CS;
  L.CS = CS;
  L.rows_len = 0;
  for (int q = 0; q < CS; ++q) {
    int nb = 0;
    while (nb < L.nlb && q + nb * CS < L.NB) ++nb;
    const size_t len = L.row_off(q, nb);
    if (len > L.rows_len) L.rows_len = len;
  }
  L.gather = false;
  L.gather = (L.base_doubles() + L.gl_len() + (size_t)L.NB * kCB * kCB) * sizeof(double) <= kClusterSmemMaxBytes;
  return L;
}

// Reciprocal square root of a positive FP64 pivot by Halley's iteration for x^(-1/2):
// with y0 an approximation and e = 1 - x y0^2, y = y0 (1 + e/2 + 3e^2/8) has relative
// error O(e^3).  The seed is the FP32 hardware approximation (relative error ~2^-22), so
// one step is below FP64 rounding.  The FP64 -> FP32 -> FP64 moves of the seed are done
// on the bit patterns with integer operations: on GB300 every FP64-pipe instruction,
// conversions included, costs ~64 cycles of a sub-partition's FP64 pipe whatever the
// number of active lanes, and this leaves five on the pivot chain.  `ok` is false
// unless x is positive and its exponent within 2^+-120 (then the result is meaningless
// and the caller reports a non-positive-definite system).
__device__ __forceinline__ double rsqrt_halley(double x, bool& ok) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  ok = hi >= 0 && ex >= 1023 - 120 && ex <= 1023 + 120;
  const int fe = min(max(ex - 1023 + 127, 1), 254);
  const float xf = __int_as_float((fe << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29));
  const int rb = __float_as_int(rsqrtf(xf));
  const int rexp = ((rb >> 23) & 0xff) - 127 + 1023;
  const double y0 = __hiloint2double((rexp << 20) | ((rb & 0x7fffff) >> 3), (rb & 7) << 29);
  const double t = x * y0;
  const double e = fma(-t, y0, 1.0);
  const double q = e * fma(0.375, e, 0.5);
  return fma(y0, q, y0);
}

// Entry-parallel layout of an 8x8 lower-triangular block in one warp: lanes 0-27 hold
// the entries (i, j) with 1 <= j <= i (lane (i-1)i/2 + j-1); lanes 28-31 hold column 0,
// rows 0-3 in slot 0 and rows 4-7 in slot 1.  A pivot then costs one scaling and one
// update instruction instead of one update per remaining column.
__device__ __forceinline__ int ep_lane(int i, int j) { return j >= 1 ? (i - 1) * i / 2 + (j - 1) : 28 + (i & 3); }
__device__ __forceinline__ bool ep_slot1(int i, int j) { return j == 0 && i >= 4; }

// u 2^de for a normal u by adding de to the exponent bits (zero is kept as it is).
__device__ __forceinline__ double scale_exp_bits(double u, int de) {
  const int hi = __double2hiint(u);
  return __hiloint2double((hi & 0x7ff00000) ? hi + de : hi, __double2loint(u));
}

// Packed index of the strictly lower entry (i, m), m < i, of an 8x8 diagonal block.
__device__ __forceinline__ int pk_lower(int i, int m) { return (i - 1) * i / 2 + m; }

// Factor the 8x8 block D (row stride NP) in place with warp 0 (other threads return at
// once): L overwrites D, blk receives M_im = L_im / L_mm at pk_lower(i, m) (m < i) and the
// reciprocals 1/L_ii at blk[28 + i]; a pivot that is not a positive normal number sets *flag.
//
// The pivot chain avoids square roots and divisions: column c is eliminated as
//   a_ij <- (a_ij p_c - a_ic a_jc) 2^-e_c,   p_c = a_cc = m 2^e_c (1 <= m < 2),
// so an entry after pivot c is s_{c+1} times the Schur complement entry of ordinary
// elimination, with s_0 = 1 and s_{c+1} = s_c p_c 2^-e_c in [1, 2^(c+1)).  The power-of-two
// scaling is exact and is applied to the exponent bits on the integer pipe, which leaves one
// multiplication and one FMA on the FP64 chain per pivot.  Afterwards, with
// R_j = (p_j s_j)^-1/2: L_ij = a_ij R_j (i >= j, a_ij the value when column j was the pivot
// column), 1/L_jj = s_j R_j and M_ij = a_ij / p_j.
__device__ __forceinline__ void factor8_warp(double* D, int NP, double* blk, int* flag) {
  const int tid = threadIdx.x;
  if (tid >= 32) return;
  const unsigned full = 0xffffffffu;
  const int lane = tid;
  int i0, j0;                                      // slot-0 entry of this lane
  if (lane < 28) {
    i0 = 1;
    while (i0 * (i0 + 1) / 2 <= lane) ++i0;
    j0 = lane - (i0 - 1) * i0 / 2 + 1;
  } else {
    i0 = lane - 28;
    j0 = 0;
  }
  double v0 = D[i0 * NP + j0];
  double v1 = lane >= 28 ? D[(lane - 24) * NP] : 0.0;
  bool bad = false;
  double pk = 1.0, ph = 1.0;                       // lane c < 8: p_c and its mantissa p_c 2^-e_c
#pragma unroll
  for (int c = 0; c < kCB; ++c) {
    const double p = __shfl_sync(full, v0, ep_lane(c, c));
    const int phi = __double2hiint(p);
    const int ex = (phi >> 20) & 0x7ff;
    bad |= phi < 0x00100000 || ex == 0x7ff;        // not a positive normal number
    if (lane == c) {
      pk = p;
      ph = __hiloint2double((phi & 0x800fffff) | 0x3ff00000, __double2loint(p));
    }
    const int la = ep_lane(i0, c), lb = ep_lane(j0, c);
    const double xa0 = __shfl_sync(full, v0, la), xa1 = __shfl_sync(full, v1, la);
    const double xb0 = __shfl_sync(full, v0, lb), xb1 = __shfl_sync(full, v1, lb);
    const double aic = ep_slot1(i0, c) ? xa1 : xa0;
    const double ajc = ep_slot1(j0, c) ? xb1 : xb0;
    if (lane < 28 && j0 > c) v0 = scale_exp_bits(fma(v0, p, -(aic * ajc)), (1023 - ex) * 0x100000);
  }
  // s_c = prod_{m < c} mantissa(p_m): inclusive scan over lanes 0-7, then shifted by one
  double sc = ph;
#pragma unroll
  for (int o = 1; o < kCB; o <<= 1) {
    const double y = __shfl_up_sync(full, sc, o);
    if (lane >= o) sc *= y;
  }
  sc = __shfl_up_sync(full, sc, 1);
  if (lane == 0) sc = 1.0;
  bool ok;
  const double R = rsqrt_halley(pk * sc, ok);
  if (lane < kCB) bad |= !ok;
  const double dinv = sc * R;                      // 1/L_cc
  const double qinv = dinv * R;                    // 1/p_c
  const double Rj = __shfl_sync(full, R, j0), Qj = __shfl_sync(full, qinv, j0);
  D[i0 * NP + j0] = v0 * Rj;
  if (lane >= 28) D[(lane - 24) * NP] = v1 * Rj;
  if (lane < 28) {
    if (j0 < i0) blk[pk_lower(i0, j0)] = v0 * Qj;
  } else {
    if (i0 > 0) blk[pk_lower(i0, 0)] = v0 * Qj;
    blk[pk_lower(lane - 24, 0)] = v1 * Qj;
  }
  if (lane < kCB) blk[kCB * (kCB - 1) / 2 + lane] = dinv;
  bad = __any_sync(full, bad);
  if (lane == 0 && bad) *flag = 1;
}

// Factor the 8x8 block D (row stride NP) in place and push, to every CTA of the cluster, the
// strictly lower block M (28 entries packed row by row) and the reciprocals 1/L_mm of its
// diagonal: the form the panel solve uses, 36 doubles sent as 16-byte stores (the number of
// remote stores, not their size, sets the cost of the push).  A non-PD flag goes to every
// CTA.  rdiag (may be null) keeps the reciprocals for the owner.
__device__ __forceinline__ void chol_factor_push(double* D, int NP, double* lkk, int* flag, double* rdiag,
                                                 cooperative_groups::cluster_group& cluster, int CS) {
  const int tid = threadIdx.x;
  __shared__ __align__(16) double s_blk[kCB * (kCB - 1) / 2 + kCB];   // packed M, then 1/L_mm
  factor8_warp(D, NP, s_blk, flag);
  __syncthreads();
  if (rdiag && tid < kCB) rdiag[tid] = s_blk[kCB * (kCB - 1) / 2 + tid];
  constexpr int NV2 = (kCB * (kCB - 1) / 2 + kCB) / 2;   // 16-byte stores per CTA
  for (int e = tid; e < CS * NV2; e += blockDim.x) {
    const int dst = e / NV2, t = e % NV2;
    reinterpret_cast<double2*>(cluster.map_shared_rank(lkk, dst))[t] = reinterpret_cast<const double2*>(s_blk)[t];
  }
  if (*flag && tid < CS) *cluster.map_shared_rank(flag, tid) = 1;
}

// Backward substitution L^T x = y (y in ybuf on every CTA, acc and contrib zero).  The
// owner of block k writes x_k to d.dc (adds it when `accumulate`).  Ends with a cluster
// barrier.
__device__ __forceinline__ void chol_backward(const Dev& d, const CholSmem& Ls, int q, const double* rows,
                                              const double* ybuf, double* acc, double* contrib, const double* linv,
                                              double* red, bool accumulate,
                                              cooperative_groups::cluster_group& cluster) {
  const int CS = Ls.CS, NB = Ls.NB, n = d.n_c;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = NB - 1; k >= 0; --k) {
    if (q == k % CS) {
      const int lb = k / CS;
      const double* R = rows + Ls.row_off(q, lb);
      const int W = Ls.row_width(q, lb);
      double* xk = red;                            // 8 values, CTA-local
      double* tk = red + 16;
      if (tid < kCB * 16) {                        // t_i = y_i - acc_i - sum over CTAs (fixed order)
        const int i = tid / 16, src = tid % 16;
        double v = src < CS ? contrib[(lb * CS + src) * kCB + i] : 0.0;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
        if (src == 0) tk[i] = ybuf[kCB * k + i] - acc[kCB * k + i] - v;
      }
      __syncthreads();
      if (tid < kCB * kCB) {                       // x = L_kk^-T t
        const int i = tid / kCB, c = tid % kCB;
        double v = linv[(lb * kCB + c) * kCB + i] * tk[c];
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 8);
        if (c == 0) {
          xk[i] = v;
          if (kCB * k + i < n) d.dc[kCB * k + i] = accumulate ? d.dc[kCB * k + i] + v : v;
        }
      }
      __syncthreads();
      for (int g = tid; g < kCB * k; g += nt) {    // acc[k'] += L_kk'^T x_k, pushed to owners
        double s = 0.0;
#pragma unroll
        for (int i = 0; i < kCB; ++i) s = fma(R[i * W + g], xk[i], s);
        const double a = acc[g] + s;
        acc[g] = a;
        const int kp = g / kCB, dst = kp % CS;
        if (dst != q) cluster.map_shared_rank(contrib, dst)[((kp / CS) * CS + q) * kCB + (g % kCB)] = a;
      }
    }
    cluster.sync();
  }
}

constexpr int kPW = 32;                            // panel width of the blocked factorisation
constexpr int kPD = kPW + 1;                       // shared-memory row stride (no bank conflicts)

// |x| to FP32 with a relative error below 2^-20 using integer operations only (no FP64
// pipe instruction): exponent rebiased, mantissa truncated; below the FP32 normal range
// gives 0, above it +inf (NaN in gives +inf or NaN).
__device__ __forceinline__ float abs_f32_approx(double x) {
  const int hi = __double2hiint(x) & 0x7fffffff;
  const int fe = ((hi >> 20) & 0x7ff) - 1023 + 127;
  if (fe <= 0) return 0.f;
  if (fe >= 255) return __int_as_float(0x7f800000);
  return __int_as_float((fe << 23) | ((hi & 0xfffff) << 3));
}

// Backward substitution L^T x = t by one CTA from the gathered factor G (packed lower
// block rows) and the diagonal-block inverses GI: per block, from the last, x_k =
// L_kk^-T t_k, then t_j -= (L_kj)^T x_k for the entries above.  t is overwritten; x goes
// to d.dc; xs holds 8 doubles of CTA-local scratch.
__device__ __forceinline__ void chol_backward_single(const Dev& d, const CholSmem& Ls, const double* G,
                                                     const double* GI, double* t, double* xs) {
  const int NB = Ls.NB, n = d.n_c, tid = threadIdx.x, nt = blockDim.x;
  for (int k = NB - 1; k >= 0; --k) {
    if (tid < kCB * kCB) {
      const int i = tid / kCB, c = tid % kCB;
      double v = GI[k * kCB * kCB + c * kCB + i] * t[kCB * k + c];
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 8);
      if (c == 0) {
        xs[i] = v;
        if (kCB * k + i < n) d.dc[kCB * k + i] = v;
      }
    }
    __syncthreads();
    const double* Rk = G + (size_t)32 * k * (k + 1);
    const int W = kCB * (k + 1);
    for (int j = tid; j < kCB * k; j += nt) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < kCB; ++i) acc = fma(Rk[i * W + j], xs[i], acc);
      t[j] -= acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double rcs_rhs(const Dev& d, int i) {
  const int pb = i / 6, comp = i % 6;
  const int kf = pb < d.fixed_kf ? pb : pb + 1;
  return d.bS[i] - d.kf_gp[kf * 6 + comp];
}

__device__ __forceinline__ double rcs_damp(const Dev& d, int i, double lam, double floor_) {
  const int pb = i / 6, comp = i % 6;
  const int kf = pb < d.fixed_kf ? pb : pb + 1;
  return lam * fmax(d.kf_dp[kf * 6 + comp], floor_);
}

// Split-phase cluster barrier: arrive (release: this thread's earlier shared and DSMEM
// writes become visible) and wait (acquire).  Every thread of every CTA calls both, in
// alternation.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// ------------------------------------------------- blocked Cholesky (large systems)
// When the reduced camera system is large, its trailing updates exceed what the 8-row block
// steps of the cluster form can hide, so the cluster factors A = L L^T right-looking by
// 32-column panels held in global memory (Lw, L2-resident), only inside the factor's envelope
// (rows [32 (p + 1), panel_end[p]) below panel p are the only ones with nonzeros in its
// columns).  Per panel p, between cluster barriers:
//   A  every warp of the cluster solves rows below the panel: L_ip = A_ip L_pp^-T and
//      y_i -= L_ip y_p;
//   B  16 x 16 tiles of the next panel's columns take A_ij -= L_ip L_jp^T (all CTAs);
//   C  CTA 0 factors the next panel's diagonal block while the other CTAs update the rest of
//      the trailing tiles (columns of the panels after the next).
// k_blk_load first copies the damped system (padding rows: identity) and the right-hand side
// to Lw and yw.  The right-hand side is carried as in the cluster form (y = L^-1 (b - g_p)
// formed during the factorisation); CTA 0 then runs the backward substitution.  Data written
// by other CTAs of the cluster is read through L2 (__ldcg) after the barrier that orders it.

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared-memory scratch of the blocked factorisation (doubles): the diagonal block with the
// right-hand side as a 33rd row, the packed 8x8 factor, 1/L_ii, the M-form of the panel's
// diagonal block, y_p, and two 16-row tile operands.
constexpr int kBlkD = (kPW + 1) * kPD, kBlkB8 = 40, kBlkMs = kPW * kPD, kBlkTile = 16 * kPD;
constexpr int kBlkScratch = kBlkD + kBlkB8 + kPW + kBlkMs + kPW + 2 * kBlkTile;

// One CTA (>= 256 threads) factors the 32 x 32 diagonal block of panel p by 8-column
// sub-blocks, the right-hand side rows riding along so that the sub-block solves also form
// y_p = L_pp^-1 y_p.  Look-ahead: after the solve of sub-block k, warp 0 updates the diagonal
// 8 x 8 block of sub-block k+1 and factors it while the other warps update the rest.  Writes
// L_pp, 1/L_ii and y_p; a pivot that is not a positive normal number sets *flag.
__device__ void blk_panel_factor(const Dev& d, int p, double* scr, int* flag) {
  constexpr int kRows = kPW + 1;
  double* D = scr;
  double* s_b8 = scr + kBlkD;
  double* s_dinv = s_b8 + kBlkB8;
  const int npw = d.npw, o = p * kPW, tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < kPW * kPW; e += nt) {
    const int i = e / kPW, j = e % kPW;
    D[i * kPD + j] = j <= i ? __ldcg(d.Lw + (size_t)(o + i) * npw + o + j) : 0.0;
  }
  if (tid < kPW) D[kPW * kPD + tid] = __ldcg(d.yw + o + tid);
  __syncthreads();
  factor8_warp(D, kPD, s_b8, flag);
  __syncthreads();
  for (int kb = 0; kb < kPW / kCB; ++kb) {
    const int c0 = kb * kCB;
    if (tid < kCB) s_dinv[c0 + tid] = s_b8[kCB * (kCB - 1) / 2 + tid];
    // rows below the sub-block (and the right-hand side row): t L_kk^T = a, 8 lanes per row
    {
      const int row = c0 + kCB + tid / kCB, c = tid % kCB, base = (tid & 31) & ~(kCB - 1);
      double t = row < kRows ? D[row * kPD + c0 + c] : 0.0;
#pragma unroll
      for (int m = 0; m < kCB - 1; ++m) {
        const double x = __shfl_sync(0xffffffffu, t, base + m);
        if (c > m) t = fma(-x, s_b8[pk_lower(c, m)], t);
      }
      if (row < kRows) D[row * kPD + c0 + c] = t * s_b8[kCB * (kCB - 1) / 2 + c];
    }
    __syncthreads();
    if (kb + 1 == kPW / kCB) break;
    // trailing entries: D_rc -= sum_m L_r,m L_c,m over this sub-block's columns, c <= r
    // (c < 32 for the right-hand side row)
    const int r0 = c0 + kCB, c1 = r0 + kCB;
    if (tid < 32) {
      for (int e = tid; e < kCB * (kCB + 1) / 2; e += 32) {   // the next diagonal block
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int r = r0 + i, c = r0 + e - i * (i + 1) / 2;
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int m = 0; m < kCB; m += 2) {
          a0 = fma(D[r * kPD + c0 + m], D[c * kPD + c0 + m], a0);
          a1 = fma(D[r * kPD + c0 + m + 1], D[c * kPD + c0 + m + 1], a1);
        }
        D[r * kPD + c] -= a0 + a1;
      }
      __syncwarp();
      factor8_warp(D + r0 * kPD + r0, kPD, s_b8, flag);
    } else {
      const int R = kRows - r0;
      for (int e = tid - 32; e < R * kPW; e += nt - 32) {
        const int r = r0 + e / kPW, c = e % kPW;
        if (c < r0 || c > r || (r < c1 && c < c1)) continue;   // outside, or the next diagonal block
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int m = 0; m < kCB; m += 2) {
          a0 = fma(D[r * kPD + c0 + m], D[c * kPD + c0 + m], a0);
          a1 = fma(D[r * kPD + c0 + m + 1], D[c * kPD + c0 + m + 1], a1);
        }
        D[r * kPD + c] -= a0 + a1;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < kPW * kPW; e += nt) {
    const int i = e / kPW, j = e % kPW;
    if (j <= i) d.Lw[(size_t)(o + i) * npw + o + j] = D[i * kPD + j];
  }
  if (tid < kPW) {
    d.Ldinv[o + tid] = s_dinv[tid];
    d.yw[o + tid] = D[kPW * kPD + tid];
  }
  __syncthreads();                                 // scratch free for the next use
}

// Phase A of panel p: warp gw of the cluster (CTA q, warp w: gw = 8 q + w) takes the rows
// o + 32 + gw, + 8 CS, ... below the panel inside its envelope: L_ip = A_ip L_pp^-T by the
// column recursion u_c = a_c - sum_{m<c} u_m M_cm (M_cm = L_cm / L_mm), t_c = u_c / L_cc, then
// y_i -= L_ip y_p.
__device__ void blk_trsm_rows(const Dev& d, int p, int q, int CS, double* scr) {
  double* Ms = scr + kBlkD + kBlkB8 + kPW;         // Ms[m * kPD + c] = M_cm (c > m)
  double* s_dv = Ms - kPW;
  double* s_yp = Ms + kBlkMs;
  const int npw = d.npw, o = p * kPW, end = d.panel_end[p], tid = threadIdx.x;
  for (int e = tid; e < kPW * kPW; e += blockDim.x) {   // row-major reads of L_pp
    const int c = e / kPW, m = e % kPW;
    Ms[m * kPD + c] = c > m ? __ldcg(d.Lw + (size_t)(o + c) * npw + o + m) * __ldcg(d.Ldinv + o + m) : 0.0;
  }
  if (tid < kPW) {
    s_dv[tid] = __ldcg(d.Ldinv + o + tid);
    s_yp[tid] = __ldcg(d.yw + o + tid);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  for (int row = o + kPW + q * nw + warp; row < end; row += CS * nw) {
    double* a = d.Lw + (size_t)row * npw + o;
    double u = __ldcg(a + lane);
#pragma unroll 4
    for (int m = 0; m < kPW - 1; ++m) {
      const double x = __shfl_sync(0xffffffffu, u, m);
      if (lane > m) u = fma(-x, Ms[m * kPD + lane], u);
    }
    const double t = u * s_dv[lane];
    a[lane] = t;
    const double sy = warp_sum(t * s_yp[lane]);
    if (lane == 0) d.yw[row] = __ldcg(d.yw + row) - sy;
  }
  __syncthreads();                                 // scratch free for the next use
}

// Tile (ti, tj), ti >= tj, of the trailing lower triangle after panel p (16 x 16, rows and
// columns counted from the first row below the panel): A_ij -= sum over the panel's 32
// columns of L_i,m L_j,m.  One entry per thread (256 threads).
__device__ void blk_syrk_tile(const Dev& d, int p, int ti, int tj, double* scr) {
  double* sa = scr + kBlkD + kBlkB8 + kPW + kBlkMs + kPW;
  double* sb = sa + kBlkTile;
  const int npw = d.npw, o = p * kPW, o2 = o + kPW, tid = threadIdx.x;
  const int ra = o2 + 16 * ti, rb = o2 + 16 * tj;
  for (int e = tid; e < 16 * kPW; e += blockDim.x) {
    const int r = e / kPW, m = e % kPW;
    sa[r * kPD + m] = __ldcg(d.Lw + (size_t)(ra + r) * npw + o + m);
    sb[r * kPD + m] = __ldcg(d.Lw + (size_t)(rb + r) * npw + o + m);
  }
  __syncthreads();
  if (tid < 256) {
    const int r = tid / 16, c = tid % 16, gi = ra + r, gj = rb + c;
    if (gj <= gi) {
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int m = 0; m < kPW; m += 2) {
        a0 = fma(sa[r * kPD + m], sb[c * kPD + m], a0);
        a1 = fma(sa[r * kPD + m + 1], sb[c * kPD + m + 1], a1);
      }
      double* x = d.Lw + (size_t)gi * npw + gj;
      *x = __ldcg(x) - (a0 + a1);
    }
  }
  __syncthreads();
}

// The blocked factorisation over the cluster (every CTA calls it; ends with a cluster
// barrier).  A failed pivot sets *flag on every CTA and stops the loop uniformly.
__device__ void blk_factor_cluster(const Dev& d, int q, int CS, double* scr, int* flag,
                                   cooperative_groups::cluster_group& cluster) {
  const int npan = d.npw / kPW, tid = threadIdx.x;
  auto factor = [&](int p) {
    blk_panel_factor(d, p, scr, flag);
    if (*flag)
      for (int r = tid; r < CS; r += blockDim.x) *cluster.map_shared_rank(flag, r) = 1;
  };
  auto rest_tile = [&](int p, int t) {             // triangle of the tiles ti >= tj >= 2
    int k = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (k * (k + 1) / 2 > t) --k;
    while ((k + 1) * (k + 2) / 2 <= t) ++k;
    blk_syrk_tile(d, p, k + 2, t - k * (k + 1) / 2 + 2, scr);
  };
  if (q == 0) factor(0);
  cluster.sync();
  for (int p = 0; p < npan && !*flag; ++p) {       // *flag is uniform after each barrier
    const int below = d.panel_end[p] - kPW * (p + 1);
    const int nt16 = below > 0 ? below / 16 : 0;
    if (below > 0) {
      blk_trsm_rows(d, p, q, CS, scr);             // A
      cluster.sync();
      for (int t = q; t < 2 * nt16 - 1; t += CS)   // B: tiles (ti, 0) then (ti >= 1, 1)
        blk_syrk_tile(d, p, t < nt16 ? t : t - nt16 + 1, t < nt16 ? 0 : 1, scr);
      cluster.sync();
    }
    if (p + 1 < npan) {                            // C
      const int n_rest = nt16 >= 2 ? (nt16 - 2) * (nt16 - 1) / 2 : 0;
      if (q == 0) {
        if (CS == 1)
          for (int t = 0; t < n_rest; ++t) rest_tile(p, t);
        factor(p + 1);
      } else {
        for (int t = q - 1; t < n_rest; t += CS - 1) rest_tile(p, t);
      }
      cluster.sync();
    }
  }
}

// Backward substitution L^T x = y of the blocked form by one CTA (generic thread count, a
// multiple of 32), by 32-column panels from the last; `smem` holds `avail` doubles.  Panel q's
// rows are needed only over the columns [c_lo, o + 32) of its envelope (c_lo: the first panel
// whose envelope holds the rows); that segment is copied to shared memory asynchronously while
// the previous panel is solved (read from global memory when it is wider than the staging
// buffer).  Per panel: x_q solves L_qq^T x_q = w_q (one warp, column recursion v_c = w_c -
// sum_{m>c} (L_mc / L_mm) v_m, x = v / L_cc), then w_c -= sum_m L_{o+m, c} x_m for the columns
// c in [c_lo, o) (two threads per column, the halves added in a fixed order).  Writes d.dc.
__device__ void blk_backward_cta(const Dev& d, double* smem, size_t avail) {
  const int n = d.n_c, npw = d.npw, npan = npw / kPW, tid = threadIdx.x, nt = blockDim.x;
  double* s_w = smem;                              // npw: y, then the running right-hand side
  double* s_dv = s_w + npw;                        // npw: 1 / L_ii
  double* s_part = s_dv + npw;                     // 2 x npw: the halves of a column's update
  double* s_m = s_part + 2 * npw;                  // kPW x kPD: L_{o+m, o+c} / L_{o+m, o+m}, m > c
  double* s_x = s_m + kPW * kPD;                   // kPW
  double* s_buf = s_x + kPW;                       // 2 x kPW x wmax: staged row segments
  const size_t fixed = 4 * (size_t)npw + kPW * kPD + kPW;
  const size_t room = avail > fixed ? (avail - fixed) / (2 * kPW) : 0;
  const int wmax = (room < 256 ? (int)room : 256) & ~1;
  auto c_lo_of = [&](int q) {
    int p = q;
    while (p > 0 && d.panel_end[p - 1] > q * kPW) --p;
    return p * kPW;
  };
  auto stage = [&](int q) {
    const int o = q * kPW, c0 = c_lo_of(q), W = o + kPW - c0;
    if (W > wmax) return;
    double* buf = s_buf + (q & 1) * kPW * wmax;
    const int nv = W / 2;                          // 16-byte pieces per row
    for (int e = tid; e < kPW * nv; e += nt) {
      const int r = e / nv, k = e % nv;
      cp_async16(buf + r * wmax + 2 * k, d.Lw + (size_t)(o + r) * npw + c0 + 2 * k);
    }
  };
  for (int i = tid; i < npw; i += nt) {
    s_w[i] = __ldcg(d.yw + i);
    s_dv[i] = __ldcg(d.Ldinv + i);
  }
  stage(npan - 1);
  cp_async_commit();
  for (int q = npan - 1; q >= 0; --q) {
    const int o = q * kPW, c0 = c_lo_of(q), W = o + kPW - c0;
    const bool staged = W <= wmax;
    const double* buf = s_buf + (q & 1) * kPW * wmax;
    cp_async_wait_all();
    __syncthreads();                               // panel q staged; the other buffer free
    if (q > 0) stage(q - 1);
    cp_async_commit();
    auto Lat = [&](int m, int c) {                 // L_{o+m, c}, c in [c0, o + 32)
      return staged ? buf[m * wmax + (c - c0)] : __ldcg(d.Lw + (size_t)(o + m) * npw + c);
    };
    for (int e = tid; e < kPW * kPW; e += nt) {
      const int m = e / kPW, c = e % kPW;
      s_m[m * kPD + c] = m > c ? Lat(m, o + c) * s_dv[o + m] : 0.0;
    }
    __syncthreads();
    if (tid < kPW) {
      double v = o + tid < n ? s_w[o + tid] : 0.0;
#pragma unroll 4
      for (int m = kPW - 1; m > 0; --m) {
        const double x = __shfl_sync(0xffffffffu, v, m);
        if (tid < m) v = fma(-s_m[m * kPD + tid], x, v);
      }
      const double xv = v * s_dv[o + tid];
      s_x[tid] = xv;
      if (o + tid < n) d.dc[o + tid] = xv;
    }
    __syncthreads();                               // x_q visible
    const int ncol = o - c0;                       // a multiple of 32
    for (int e = tid; e < 2 * ncol; e += nt) {     // lanes l and l + 16 of a warp: one column's halves
      const int l = e & 31, c = c0 + (e >> 5) * 16 + (l & 15), h = l >> 4;
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int m = 16 * h; m < 16 * h + 16; m += 2) {
        a0 = fma(Lat(m, c), s_x[m], a0);
        a1 = fma(Lat(m + 1, c), s_x[m + 1], a1);
      }
      s_part[h * npw + c] = a0 + a1;
    }
    __syncthreads();
    for (int c = c0 + tid; c < o; c += nt) s_w[c] -= s_part[c] + s_part[npw + c];
  }
  __syncthreads();
}

// Dynamic shared memory of the cluster kernel in the blocked form, besides its layout: the
// factorisation scratch and the backward substitution's arrays with 256-column staging.
size_t blk_cluster_smem(int npw) {
  const size_t back = 4 * (size_t)npw + kPW * kPD + kPW + 2 * (size_t)kPW * 256;
  return (std::max<size_t>(kBlkScratch, back) + 8) * sizeof(double);
}

__device__ __forceinline__ void chol_cluster_body(const Dev& d) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) double smem[];
  Ctrl* ctrl = d.ctrl;
  if (ctrl->nonpd) return;                         // uniform: a landmark block failed
  const int CS = (int)cluster.num_blocks();
  const int q = (int)cluster.block_rank();
  const int n = d.n_c;
  const CholSmem Ls = chol_layout(n, CS);
  const int NB = Ls.NB, NP = Ls.NP;
  double* rows = smem + Ls.rows_off();             // packed lower block rows of this CTA
  double* panel0 = smem + Ls.panel_off();          // two buffers [c][i][m] = L[8c+i][8k+m]
  double* lkk0 = smem + Ls.lkk_off();              // two buffers: packed M of L_kk, then 8 reciprocals of the diagonal
  double* ybuf = smem + Ls.y_off();                // right-hand side row / y
  double* acc = smem + Ls.acc_off();               // backward contributions of own rows
  double* contrib = smem + Ls.contrib_off();       // [lb][from CTA][8]
  double* linv = smem + Ls.linv_off();             // [lb][i][m] inverse of own diagonal blocks
  double* rdiag = smem + Ls.rdiag_off();           // [lb][i] reciprocals of own diagonal entries
  double* nrm = smem + Ls.nrm_off();               // [CTA][4] refinement norms
  double* red = smem + Ls.red_off();
  // the blocked form uses all of shared memory below its last 8 doubles as scratch, with the
  // flag there (its launch may ask for more than the layout)
  unsigned dyn_bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  const size_t dyn_doubles = dyn_bytes / sizeof(double);
  int* flag = reinterpret_cast<int*>(smem + (d.chol_blocked ? dyn_doubles - 8 : Ls.flag_off()));
  const int tid = threadIdx.x, nt = blockDim.x;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, red);        // block-level, contains barriers
  auto rowp = [&](int lb) { return rows + Ls.row_off(q, lb); };

  // inverses of own diagonal blocks (thread per (block, column))
  auto own_block_inverses = [&]() {
    for (int e = tid; e < Ls.nlb * kCB; e += nt) {
      const int lb = e / kCB, j = e % kCB, r = q + lb * CS;
      if (r >= NB) continue;
      const int W = Ls.row_width(q, lb);
      const double* D = rowp(lb) + kCB * r;
      double z[kCB];
#pragma unroll
      for (int i = 0; i < kCB; ++i) {
        double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
        for (int m = 0; m < i; ++m) s = fma(-D[i * W + m], z[m], s);
        z[i] = i < j ? 0.0 : s * rdiag[lb * kCB + i];
      }
#pragma unroll
      for (int i = 0; i < kCB; ++i) linv[(lb * kCB + i) * kCB + j] = z[i];
    }
  };

  if (d.chol_blocked) {
    // ---- blocked factorisation over the cluster (Lw, yw loaded by k_blk_load), then the
    // backward substitution on CTA 0; shared memory is scratch until then.  The factor's rows
    // are loaded into their block rows only if the refinement below applies a correction.
    if (tid == 0) *flag = 0;
    cluster.sync();
    blk_factor_cluster(d, q, CS, smem, flag, cluster);
    if (!*flag && q == 0) blk_backward_cta(d, smem, dyn_doubles - 8);
    for (int c = tid; c < NP; c += nt) acc[c] = 0.0;
    for (int e = tid; e < Ls.nlb * CS * kCB; e += nt) contrib[e] = 0.0;
    cluster.sync();                                // dc visible everywhere
  } else {
    // ---- load own block rows (damped, padded), rhs on CTA 0
    for (int lb = 0; lb < Ls.nlb; ++lb) {
      const int r = q + lb * CS;
      if (r >= NB) break;
      const int W = Ls.row_width(q, lb);
      double* R = rowp(lb);
      for (int e = tid; e < kCB * W; e += nt) {
        const int i = e / W, c = e % W, gi = kCB * r + i;
        double v = 0.0;
        if (gi < n && c < n) {
          if (c <= gi) v = d.S[(size_t)gi * n + c];
          if (c == gi) v += rcs_damp(d, gi, lam, floor_);
        } else if (gi >= n && c == gi) {
          v = 1.0;
        }
        R[e] = v;
      }
    }
    for (int c = tid; c < NP; c += nt) {
      ybuf[c] = (q == 0 && c < n) ? rcs_rhs(d, c) : 0.0;
      acc[c] = 0.0;
    }
    for (int e = tid; e < Ls.nlb * CS * kCB; e += nt) contrib[e] = 0.0;
    if (tid == 0) *flag = 0;
    cluster.sync();
    if (q == 0) chol_factor_push(rows, kCB, lkk0, flag, rdiag, cluster, CS);   // block 0: CTA 0's first row block
    cluster_arrive();                                // A_0

    // ---- factorisation with the forward substitution fused.  Per step k two split
    // barriers: A_k (L_kk pushed) and B_k (panel k pushed).  The owner of block k+1 factors
    // it between its arrival at B_k and its wait there, so the factorisation does not wait
    // for the whole cluster's panel exchange, and every CTA arrives at A_{k+1} before its
    // trailing update.  L_kk and the panels alternate between two buffers.
    bool broke = false;
    for (int k = 0; k < NB; ++k) {
      cluster_wait();                                // A_k: L_kk (and flag) visible everywhere
      if (*flag) {                                   // uniform: pushed before A_k
        broke = true;
        break;
      }
      const double* lkk = lkk0 + (k & 1) * (kCB * kCB + kCB);
      double* panel = panel0 + (size_t)(k & 1) * NB * kCB * kCB;
      // 1. TRSM of own block rows below k, and of the right-hand side on CTA 0: solve
      //    t L_kk^T = a for each row, entry-parallel (8 lanes per row, one column each).
      //    With u_c = t_c L_cc: u_c = a_c - sum_{m<c} u_m M_cm (M_cm = L_cm / L_mm, pushed
      //    with L_kk), one update instruction per column, and t_c = u_c / L_cc at the end.
      const double* linvd = lkk + kCB * (kCB - 1) / 2;
      const int n_trsm = (Ls.nlb * kCB + 1) * kCB;
      for (int e0 = 0; e0 < n_trsm; e0 += nt) {       // warp-uniform trip count
        const int e = e0 + tid, row = e / kCB, c = e % kCB;
        double* a = nullptr;
        if (e < n_trsm) {
          if (row < Ls.nlb * kCB) {
            const int lb = row / kCB, i = row % kCB, r = q + lb * CS;
            if (r > k && r < NB) a = rowp(lb) + i * Ls.row_width(q, lb) + kCB * k;
          } else if (q == 0) {
            a = ybuf + kCB * k;
          }
        }
        double t = a ? a[c] : 0.0;
        const int base = (tid & 31) & ~(kCB - 1);
  #pragma unroll
        for (int m = 0; m < kCB - 1; ++m) {
          const double x = __shfl_sync(0xffffffffu, t, base + m);
          if (c > m) t = fma(-x, lkk[(c - 1) * c / 2 + m], t);
        }
        if (a) a[c] = t * linvd[c];
      }
      __syncthreads();
      for (int lb = 0; lb < Ls.nlb; ++lb) {          // push panel blocks L_rk to every CTA
        const int r = q + lb * CS;
        if (r <= k || r >= NB) continue;
        const double* R = rowp(lb);
        const int W = Ls.row_width(q, lb);
        for (int e = tid; e < CS * kCB * kCB / 2; e += nt) {
          const int dst = e / (kCB * kCB / 2), t = e % (kCB * kCB / 2), i = t / (kCB / 2), m = 2 * (t % (kCB / 2));
          reinterpret_cast<double2*>(cluster.map_shared_rank(panel, dst) + (size_t)r * kCB * kCB)[t] =
              *reinterpret_cast<const double2*>(R + i * W + kCB * k + m);
        }
      }
      cluster_arrive();                              // B_k
      // 2a. look-ahead: owner of block k+1 updates its diagonal block with its own L_{k+1,k}
      //     and factors it
      if (k + 1 < NB && q == (k + 1) % CS) {
        const int lb = (k + 1) / CS;
        double* R = rowp(lb);
        const int W = Ls.row_width(q, lb);
        for (int e = tid; e < kCB * kCB; e += nt) {
          const int i = e / kCB, j = e % kCB;
          if (j > i) continue;
          double s = 0.0;
  #pragma unroll
          for (int m = 0; m < kCB; ++m) s = fma(R[i * W + kCB * k + m], R[j * W + kCB * k + m], s);
          R[i * W + kCB * (k + 1) + j] -= s;
        }
        __syncthreads();
        chol_factor_push(R + kCB * (k + 1), W, lkk0 + ((k + 1) & 1) * (kCB * kCB + kCB), flag, rdiag + lb * kCB,
                         cluster, CS);
      }
      cluster_wait();                                // B_k: panel k visible everywhere
      // L_{k+1,k+1} is pushed: signal A_{k+1} before this CTA's trailing update, which then
      // overlaps the next step's chain.  Panels alternate between two buffers, and a CTA
      // cannot reach the next write of this buffer (step k+2) before every CTA has arrived
      // at A_{k+2}, after its own trailing update of step k.
      cluster_arrive();                              // A_{k+1}
      // 2b. trailing update of own block rows: A_rc -= L_rk L_ck^T, c in (k, r]
      for (int lb = 0; lb < Ls.nlb; ++lb) {
        const int r = q + lb * CS;
        if (r <= k + 1 || r >= NB) continue;
        double* R = rowp(lb);
        const int W = Ls.row_width(q, lb);
        const double* Lr = panel + (size_t)r * kCB * kCB;
        const int cnt = (r - k) * kCB * kCB;
        for (int e = tid; e < cnt; e += nt) {
          const int c = k + 1 + e / (kCB * kCB), t = e % (kCB * kCB), i = t / kCB, j = t % kCB;
          const double* Lc = panel + (size_t)c * kCB * kCB + j * kCB;
          double s = 0.0;
  #pragma unroll
          for (int m = 0; m < kCB; ++m) s = fma(Lr[i * kCB + m], Lc[m], s);
          R[i * W + kCB * c + j] -= s;
        }
      }
      if (q == 0) {
        const double* y = ybuf + kCB * k;
        for (int e = tid; e < NP - kCB * (k + 1); e += nt) {
          const int g = kCB * (k + 1) + e, c = g / kCB, j = g % kCB;
          const double* Lc = panel + (size_t)c * kCB * kCB + j * kCB;
          double s = 0.0;
  #pragma unroll
          for (int m = 0; m < kCB; ++m) s = fma(y[m], Lc[m], s);
          ybuf[g] -= s;
        }
      }
      __syncthreads();                               // own rows updated before the next TRSM
    }
    if (!broke) cluster_wait();                      // A_NB: the factor complete everywhere
  }
  if (*flag) {
    if (q == 0 && tid == 0) ctrl->nonpd = 1;
    return;
  }
  if (!d.chol_blocked) {                           // (blocked form: k_blk_back solved)
    own_block_inverses();
    if (Ls.gather) {
      // small system: own block rows and their diagonal inverses to CTA 0, which runs the
      // backward substitution alone (no cluster barrier per block)
      __syncthreads();
      double* gl = smem + Ls.gl_off();
      double* glinv = smem + Ls.glinv_off();
      for (int lb = 0; lb < Ls.nlb; ++lb) {
        const int r = q + lb * CS;
        if (r >= NB) break;
        const double* R = rowp(lb);
        double* dst = cluster.map_shared_rank(gl, 0) + (size_t)32 * r * (r + 1);
        for (int e = tid; e < kCB * kCB * (r + 1); e += nt) dst[e] = R[e];
        double* dli = cluster.map_shared_rank(glinv, 0) + (size_t)r * kCB * kCB;
        for (int e = tid; e < kCB * kCB; e += nt) dli[e] = linv[lb * kCB * kCB + e];
      }
      cluster.sync();
      if (q == 0) chol_backward_single(d, Ls, gl, glinv, ybuf, red);
      cluster.sync();                              // dc visible everywhere
    } else {
      if (q == 0) {
        for (int e = tid; e < CS * NP; e += nt) {
          const int dst = e / NP, c = e % NP;
          if (dst != 0) cluster.map_shared_rank(ybuf, dst)[c] = ybuf[c];
        }
      }
      cluster.sync();
      chol_backward(d, Ls, q, rows, ybuf, acc, contrib, linv, red, false, cluster);
    }
  }

  // ---- iterative refinement in FP64: r = rhs - A dc from the assembled S (global, lower
  // triangle), stopped by the backward-error test |r| <= |A| |dc| eps sqrt(n) (infinity
  // norms, eps = 2^-53) or after refine_max corrections dc += A^-1 r.
  const int refine_max = ctrl->refine_max;
  for (int it_r = 0; it_r < refine_max; ++it_r) {
    // residual of own rows, one warp per row; the rows' entries of ybuf hold r.  The
    // norms only feed the stopping test and the reported backward error: kept in FP32.
    {
      const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
      float m_r = 0.f, m_a = 0.f, m_x = 0.f, m_b = 0.f;
      for (int e = warp; e < Ls.nlb * kCB; e += nw) {
        const int lb = e / kCB, i = e % kCB, gi = kCB * (q + lb * CS) + i;
        if (gi >= NP) continue;
        if (gi >= n) {                             // padding rows: zero residual
          if (lane == 0) ybuf[gi] = 0.0;
          continue;
        }
        double s = 0.0;
        float sa = 0.f;
#pragma unroll 4
        for (int j = lane; j < n; j += 32) {
          double a = d.S[(size_t)gi * n + j];       // S holds both triangles
          if (j == gi) a += rcs_damp(d, gi, lam, floor_);
          s = fma(a, d.dc[j], s);
          sa += abs_f32_approx(a);
        }
        s = warp_sum(s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sa += __shfl_xor_sync(0xffffffffu, sa, o);
        const double b = rcs_rhs(d, gi), r = b - s;
        if (lane == 0) ybuf[gi] = r;
        m_r = fmaxf(m_r, abs_f32_approx(r));
        m_a = fmaxf(m_a, sa);
        m_x = fmaxf(m_x, abs_f32_approx(d.dc[gi]));
        m_b = fmaxf(m_b, abs_f32_approx(b));
      }
      float* redf = reinterpret_cast<float*>(red + 32);
      if (lane == 0) {
        redf[warp] = m_r;
        redf[32 + warp] = m_a;
        redf[64 + warp] = m_x;
        redf[96 + warp] = m_b;
      }
      __syncthreads();
      if (tid < CS * 4) {                          // push this CTA's maxima to every CTA
        const int dst = tid / 4, k = tid % 4;
        float v = 0.f;
        for (int w = 0; w < nw; ++w) v = fmaxf(v, redf[32 * k + w]);
        reinterpret_cast<float*>(cluster.map_shared_rank(nrm, dst))[q * 4 + k] = v;
      }
    }
    for (int e = tid; e < NP; e += nt) acc[e] = 0.0;
    for (int e = tid; e < Ls.nlb * CS * kCB; e += nt) contrib[e] = 0.0;
    cluster.sync();                                // norms and residual rows visible
    const float* nrmf = reinterpret_cast<const float*>(nrm);
    float rn = 0.f, an = 0.f, xn = 0.f, bn = 0.f;
    for (int c = 0; c < CS; ++c) {
      rn = fmaxf(rn, nrmf[c * 4]);
      an = fmaxf(an, nrmf[c * 4 + 1]);
      xn = fmaxf(xn, nrmf[c * 4 + 2]);
      bn = fmaxf(bn, nrmf[c * 4 + 3]);
    }
    if (it_r == 0 && q == 0 && tid == 0) ctrl->berr = (double)(rn / fmaxf(an * xn + bn, 1e-30f));
    if (rn <= an * xn * 0x1p-53f * sqrtf((float)n)) break;   // uniform over the cluster
    if (d.chol_blocked && it_r == 0) {
      // a correction: own block rows of the blocked form's factor and their inverses
      for (int lb = 0; lb < Ls.nlb; ++lb) {
        const int r = q + lb * CS;
        if (r >= NB) break;
        const int W = Ls.row_width(q, lb);
        double* R = rowp(lb);
        for (int e = tid; e < kCB * W; e += nt) {
          const int i = e / W, c = e % W, gi = kCB * r + i;
          R[e] = c <= gi ? d.Lw[(size_t)gi * d.npw + c] : 0.0;
        }
        if (tid < kCB) rdiag[lb * kCB + tid] = d.Ldinv[kCB * r + tid];
      }
      __syncthreads();
      own_block_inverses();
      __syncthreads();
    }
    // forward sweep L y = r, right-looking: the owner of block k forms y_k = L_kk^-1 r_k
    // and pushes it to every CTA, which then updates its own rows below k
    for (int k = 0; k < NB; ++k) {
      if (q == k % CS) {                           // uniform over the CTA
        const int lb = k / CS, i = (tid / kCB) & (kCB - 1), c = tid % kCB;
        double v = 0.0;
        if (tid < kCB * kCB) {
          v = linv[(lb * kCB + i) * kCB + c] * ybuf[kCB * k + c];
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 8);
        }
        __syncthreads();                           // r_k read before y_k overwrites it
        if (tid < kCB * kCB)
          for (int dst = c; dst < CS; dst += kCB) cluster.map_shared_rank(ybuf, dst)[kCB * k + i] = v;
      }
      cluster.sync();
      for (int e = tid; e < Ls.nlb * kCB; e += nt) {
        const int lb = e / kCB, i = e % kCB, r = q + lb * CS;
        if (r <= k || r >= NB) continue;
        const double* Rk = rowp(lb) + i * Ls.row_width(q, lb) + kCB * k;
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < kCB; ++m) s = fma(Rk[m], ybuf[kCB * k + m], s);
        ybuf[kCB * r + i] -= s;
      }
      __syncthreads();
    }
    chol_backward(d, Ls, q, rows, ybuf, acc, contrib, linv, red, true, cluster);
    if (q == 0 && tid == 0) ctrl->refined = it_r + 1;
  }

  // ---- epilogue: predicted-reduction part and step norm of own rows (one partial per
  // CTA, summed in order by k_decide), candidate poses
  {
    double v0 = 0.0, v1 = 0.0;
    const int n_own = Ls.nlb * kCB;
    for (int e = tid; e < n_own; e += nt) {
      const int lb = e / kCB, i = kCB * (q + lb * CS) + e % kCB;
      if (i < n) {
        const int pb = i / 6, comp = i % 6;
        const int kf = pb < d.fixed_kf ? pb : pb + 1;
        const double D = fmax(d.kf_dp[kf * 6 + comp], floor_);
        const double xi = d.dc[i];
        v0 += xi * (lam * D * xi - d.kf_gp[kf * 6 + comp]);
        v1 += xi * xi;
      }
    }
    const int nw_own = min((n_own + 31) / 32, nt / 32);   // warps holding own rows
    if ((tid >> 5) < nw_own) {
      v0 = warp_sum(v0);
      v1 = warp_sum(v1);
      if ((tid & 31) == 0) {
        red[2 * (tid >> 5)] = v0;
        red[2 * (tid >> 5) + 1] = v1;
      }
    }
    __syncthreads();
    if (tid == 0) {
      double p0 = 0.0, p1 = 0.0;
      for (int w = 0; w < nw_own; ++w) {             // fixed order
        p0 += red[2 * w];
        p1 += red[2 * w + 1];
      }
      ctrl->pred_part[q] = p0;
      ctrl->step2_part[q] = p1;
      if (q == 0) ctrl->n_parts = CS;
    }
  }
  pose_candidates(d, q, CS);
  if (d.mixed)
    for (int i = q * nt + tid; i < d.n_c; i += CS * nt) d.dc_f[i] = (float)d.dc[i];
}

__global__ void __launch_bounds__(256) k_chol_cluster(Dev d) { pdl_enter(); chol_cluster_body(d); }
// Batched: one cluster per window (cluster index = window).
__global__ void __launch_bounds__(256) k_chol_cluster_b(const Dev* __restrict__ wins) { pdl_enter();
  __shared__ Dev sd;
  load_dev(sd, wins + blockIdx.x / cooperative_groups::this_cluster().dim_blocks().x);
  if (sd.chol_fallback) return;                    // uniform over the cluster
  chol_cluster_body(sd);
}

// Copy of the damped reduced camera system (padding rows: identity) and of its right-hand
// side to the blocked form's working arrays Lw and yw.
__global__ void __launch_bounds__(256) k_blk_load(Dev d) { pdl_enter();
  __shared__ double s_red[64];
  Ctrl* ctrl = d.ctrl;
  if (ctrl->nonpd) return;
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);      // block-level, contains barriers
  const int n = d.n_c, npw = d.npw;
  const size_t total = (size_t)npw * npw;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / npw), j = (int)(e % npw);
    double v = 0.0;
    if (j <= i) {
      if (i < n) {
        v = d.S[(size_t)i * n + j];
        if (i == j) v += rcs_damp(d, i, lam, floor_);
      } else if (i == j) {
        v = 1.0;
      }
    }
    d.Lw[e] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npw; i += gridDim.x * blockDim.x)
    d.yw[i] = i < n ? rcs_rhs(d, i) : 0.0;
}

// --------------------------------------------------------------- k_backsub
template <typename T>
__host__ __device__ constexpr size_t backsub_smem_bytes(int C) {
  return sizeof(double) * 128 + tile_stage_bytes<T>() +
         sizeof(T) * ((size_t)C * RIG_STRIDE + LIN_TILE_PAIRS * (3 + PAIR_LIN) + LIN_TILE_LMS * 3);
}
template <typename T>
__device__ __forceinline__ void k_backsub_body(const Dev& d, int item) {
  extern __shared__ __align__(16) double smem[];
  Ctrl* ctrl = d.ctrl;
  const LinTile tile = d.lin_tiles[item];
  if (ctrl->nonpd) {
    if (threadIdx.x < 4) d.bs_part[item * 4 + threadIdx.x] = 0.0;
    return;
  }
  const int nl = tile.l1 - tile.l0, np = tile.p1 - tile.p0;
  const bool obs_s = tile.o1 - tile.o0 <= LIN_TILE_OBS;
  double* s_red = smem;                              // 128
  const TileStage<T> sg = tile_stage<T>(smem);
  T* s_rig = reinterpret_cast<T*>(sg.end);           // C * 16
  T* s_acc = s_rig + d.C * RIG_STRIDE;               // LIN_TILE_PAIRS * 3 (per pair slots)
  T* s_plin = s_acc + LIN_TILE_PAIRS * 3;            // LIN_TILE_PAIRS * PAIR_LIN
  T* s_new = s_plin + LIN_TILE_PAIRS * PAIR_LIN;     // LIN_TILE_LMS * 3
  stage_tile<T>(d, tile, sg, obs_s);
  {
    const T* pl = reinterpret_cast<const T*>(d.pair_lin) + (size_t)tile.p0 * PAIR_LIN;
    for (int e = threadIdx.x; e < np * PAIR_LIN; e += blockDim.x) cpa_t<T>(s_plin + e, pl + e);
  }
  const T* rig = st_rig<T>(d);
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = rig[i];
  cpa_wait_all();
  const double lam = ctrl->lam;
  const double floor_ = diag_floor(d, s_red);   // contains __syncthreads
  const int cur = ctrl->cur;
  const T* pose = st_pose<T>(d, cur);
  const T* dcT = st_dc<T>(d);
  // phase 1: W_ja^T dc_a = R_a^T M3 (rho + phi x X) accumulated per landmark
  for (int qi = threadIdx.x; qi < np; qi += blockDim.x) {
    const int a = sg.pkf[qi];
    const int pb = d.kf_pb[a];
    T* acc = s_acc + qi * 3;
    if (pb < 0) {
      acc[0] = acc[1] = acc[2] = 0;
      continue;
    }
    const T* pl = s_plin + qi * PAIR_LIN;
    const T* xi = dcT + 6 * pb;
    T X[3] = {pl[6], pl[7], pl[8]};
    T u[3];
    u[0] = xi[0] + (xi[4] * X[2] - xi[5] * X[1]);
    u[1] = xi[1] + (xi[5] * X[0] - xi[3] * X[2]);
    u[2] = xi[2] + (xi[3] * X[1] - xi[4] * X[0]);
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
    T R[12];
    load_pose12(pose + a * POSE_STRIDE, R);
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = R[c] * w3[0] + R[3 + c] * w3[1] + R[6 + c] * w3[2];
  }
  __syncthreads();
  // phase 2: dp_j = -V_j^-1 (g_l + acc); candidate landmark; predicted-reduction part
  // (FP64 path: in FP64; mixed path: in FP32 with compensated sums, the new landmark
  // position in FP64).  Thread per (landmark, component c): each forms the three sums
  // g_l + acc, then its row of V_j^-1 and its components of dp_j, the candidate and the
  // predicted reduction (spreading the FP64 work over the CTA's warps).
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  Acc<float> lp_f, st2_f;
  for (int e = threadIdx.x; e < nl * 3; e += blockDim.x) {
    const int l = e / 3, c = e - 3 * l, j = tile.l0 + l;
    Acc<T> w0, w1, w2;
    for (int q = sg.lmp[l]; q < sg.lmp[l + 1]; ++q) {
      const T* acc = s_acc + (q - tile.p0) * 3;
      w0.add(acc[0]);
      w1.add(acc[1]);
      w2.add(acc[2]);
    }
    // row c of the symmetric V^-1 (00 01 02 11 12 22)
    const int i0 = c == 0 ? 0 : (c == 1 ? 1 : 2), i1 = c == 0 ? 1 : (c == 1 ? 3 : 4), i2 = c == 0 ? 2 : (c == 1 ? 4 : 5);
    const int hd = c == 0 ? 0 : (c == 1 ? 3 : 5);
    double ec;
    if constexpr (sizeof(T) == 4) {
      const float* Vi = reinterpret_cast<const float*>(d.lm_Vinv) + VINV_STRIDE * j;
      const float tau = Vi[6];
      const float g0 = (float)d.lm_g[3 * j], g1 = (float)d.lm_g[3 * j + 1], g2 = (float)d.lm_g[3 * j + 2];
      const float t0 = g0 + w0.rounded(), t1 = g1 + w1.rounded(), t2 = g2 + w2.rounded();
      const float dpc = -(Vi[i0] * t0 + Vi[i1] * t1 + Vi[i2] * t2);
      const float gc = c == 0 ? g0 : (c == 1 ? g1 : g2);
      const float lamf = (float)lam, fl = (float)floor_;
      const float Dc = fmaxf((float)d.lm_H[6 * j + hd], fl);
      lp_f.add(dpc * ((lamf * Dc + tau) * dpc - gc));
      st2_f.add(dpc * dpc);
      ec = dpc;
    } else {
      const double* Vi = d.lm_Vinv + VINV_STRIDE * j;
      const double tau = Vi[6];
      const double* g = d.lm_g + 3 * j;
      const double t0 = g[0] + w0.value(), t1 = g[1] + w1.value(), t2 = g[2] + w2.value();
      const double dpc = -(Vi[i0] * t0 + Vi[i1] * t1 + Vi[i2] * t2);
      const double Dc = fmax(d.lm_H[6 * j + hd], floor_);
      v[1] += dpc * ((lam * Dc + tau) * dpc - g[c]);
      v[2] += dpc * dpc;
      ec = dpc;
    }
    d.dp[j * 3 + c] = ec;
    const double nc = d.lm[cur][3 * j + c] + ec;
    d.lm[cur ^ 1][3 * j + c] = nc;
    const T mc = (T)nc;
    s_new[l * 3 + c] = mc;
    if constexpr (sizeof(T) == 4) d.lm_f[cur ^ 1][3 * j + c] = mc;
  }
  __syncthreads();
  // phase 3: candidate cost, same arithmetic and order as k_lin's cost
  const T* pnew = st_pose<T>(d, cur ^ 1);
  const T hub = (T)ctrl->huber, zmin = (T)ctrl->zmin;
  PairStats<T> st;
  for (int qi = threadIdx.x; qi < np; qi += blockDim.x) {
    const int a = sg.pkf[qi], jl = sg.plm[qi] - tile.l0;
    T X[3], Pv[12];
    load_pose12(pnew + a * POSE_STRIDE, Pv);
    if (obs_s)
      eval_pair<T, false>(Pv, s_new + 3 * jl, sg.pobs[qi] - tile.o0, sg.pobs[qi + 1] - tile.o0,
                          sg.cam, sg.uv, s_rig, hub, zmin, X, nullptr, nullptr, st);
    else
      eval_pair<T, false>(Pv, s_new + 3 * jl, sg.pobs[qi], sg.pobs[qi + 1], d.obs_cam,
                          reinterpret_cast<const T*>(d.obs_uv), s_rig, hub, zmin, X, nullptr, nullptr, st);
  }
  if constexpr (sizeof(T) == 4) {                  // mixed: (hi, lo) float pairs, summed by k_decide
    DF f[3] = {st.cost.df(), lp_f.df(), st2_f.df()};
    DF o[3];
    block_sum_df_pair<3>(f, o, reinterpret_cast<float*>(s_red));
    if (threadIdx.x == 0) {
      float4* bp = reinterpret_cast<float4*>(d.bs_part + item * 4);
      bp[0] = make_float4(o[0].hi, o[0].lo, o[1].hi, o[1].lo);
      bp[1] = make_float4(o[2].hi, o[2].lo, 0.0f, 0.0f);
    }
  } else {
    v[0] = st.cost.value();
    block_sum4(v, s_red);
    if (threadIdx.x == 0) {
      d.bs_part[item * 4 + 0] = v[0];
      d.bs_part[item * 4 + 1] = v[1];
      d.bs_part[item * 4 + 2] = v[2];
      d.bs_part[item * 4 + 3] = 0.0;
    }
  }
}

template <typename T>
// Mixed path: six CTAs per SM (the staged tile takes ~34 KB of shared memory at 32 cameras).
__global__ void __launch_bounds__(LIN_THREADS, sizeof(T) == 4 ? 6 : 1) k_backsub(Dev d) { pdl_enter(); k_backsub_body<T>(d, blockIdx.x); }
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_backsub_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_backsub_body<T>(sd, it.y);
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

__device__ __forceinline__ void k_decide_body(const Dev& d, int item) {
  __shared__ double s_red[128];
  __shared__ double s_sum[8 * 256];
  __shared__ DF s_sumf[8 * 256];
  Ctrl* ctrl = d.ctrl;
  // fixed-order sums of the tile partials.  A tile's four partials are two 16-byte halves
  // (lin: (cost, sum r^2), (n_valid, n_inlier); candidate: (cost, L part), (|dp|^2, 0)).
  // Thread t (1024) takes array t / 512 and half t % 2 of the tiles (t % 512) / 2 + 256 i,
  // loading them coalesced, eight at a time, into four interleaved sums per value (combined
  // pairwise); warp w < 8 then adds the 256 thread sums of value w in a fixed order.  The
  // mixed path's partials are (hi, lo) float pairs summed as such: on GB300 an FP64 add holds
  // a sub-partition's FP64 pipe for ~64 cycles per warp instruction.
  {
    const int tid = threadIdx.x, arr = tid >> 9, u = tid & 511, half = u & 1, r0 = u >> 1;
    const int n = d.n_lin_tiles;
    const int slot = (arr * 2 + half) * 2;           // values slot, slot + 1 of s_sum*
    if (d.mixed) {
      const float4* part = reinterpret_cast<const float4*>(arr == 0 ? d.lin_part : d.bs_part);
      DF a0[4], a1[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) a0[k] = a1[k] = DF{0.0f, 0.0f};
      int r = r0;
      for (; r + 7 * 256 < n; r += 8 * 256) {
        float4 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = part[(r + 256 * k) * 2 + half];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          a0[k & 3] = df_add(a0[k & 3], DF{x[k].x, x[k].y});
          a1[k & 3] = df_add(a1[k & 3], DF{x[k].z, x[k].w});
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (r + 256 * k < n) {
          const float4 x = part[(r + 256 * k) * 2 + half];
          a0[k & 3] = df_add(a0[k & 3], DF{x.x, x.y});
          a1[k & 3] = df_add(a1[k & 3], DF{x.z, x.w});
        }
      s_sumf[slot * 256 + r0] = df_add(df_add(a0[0], a0[1]), df_add(a0[2], a0[3]));
      s_sumf[(slot + 1) * 256 + r0] = df_add(df_add(a1[0], a1[1]), df_add(a1[2], a1[3]));
    } else {
      const double2* part = reinterpret_cast<const double2*>(arr == 0 ? d.lin_part : d.bs_part);
      double a0[4] = {0.0, 0.0, 0.0, 0.0}, a1[4] = {0.0, 0.0, 0.0, 0.0};
      int r = r0;
      for (; r + 7 * 256 < n; r += 8 * 256) {
        double2 x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = part[(r + 256 * k) * 2 + half];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          a0[k & 3] += x[k].x;
          a1[k & 3] += x[k].y;
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (r + 256 * k < n) {
          const double2 x = part[(r + 256 * k) * 2 + half];
          a0[k & 3] += x.x;
          a1[k & 3] += x.y;
        }
      s_sum[slot * 256 + r0] = (a0[0] + a0[1]) + (a0[2] + a0[3]);
      s_sum[(slot + 1) * 256 + r0] = (a1[0] + a1[1]) + (a1[2] + a1[3]);
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    if (warp < 8) {                                  // value warp: lin 0-3, candidate 4-7
      double v;
      if (d.mixed) {
        DF x = s_sumf[warp * 256 + lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) x = df_add(x, s_sumf[warp * 256 + lane + 32 * k]);
        x = warp_sum_df(x);
        v = (double)x.hi + (double)x.lo;
      } else {
        double x = s_sum[warp * 256 + lane];
#pragma unroll
        for (int k = 1; k < 8; ++k) x += s_sum[warp * 256 + lane + 32 * k];
        v = warp_sum(x);
      }
      if (lane == 0) s_red[warp] = v;
    }
  }
  __syncthreads();
  double lin[4], bs[4];
  for (int k = 0; k < 4; ++k) lin[k] = s_red[k];
  for (int k = 0; k < 3; ++k) bs[k] = s_red[4 + k];
  bs[3] = 0.0;
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
    rec.berr = ctrl->berr;
    rec.refined = ctrl->refined;
    rec.reserved = 0;
    ctrl->berr = CUDART_NAN;
    ctrl->refined = 0;
    bool acc = false;
    if (nonpd) {
      rec.cost1 = rec.gain = rec.pred = rec.step_norm = CUDART_NAN;
    } else {
      const double F1 = bs[0];
      double pp = 0.0, sp = 0.0;
      for (int k = 0; k < ctrl->n_parts; ++k) {    // fixed order
        pp += ctrl->pred_part[k];
        sp += ctrl->step2_part[k];
      }
      const double L = 0.5 * (pp + bs[1]);
      rec.cost1 = F1;
      rec.pred = L;
      rec.step_norm = sqrt(sp + bs[2]);
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
    ctrl->maxdiag_kf = 0ull;                         // recomputed by k_kf_reduce every iteration
  }
}

__global__ void __launch_bounds__(KDECIDE_THREADS) k_decide(Dev d) { pdl_enter(); k_decide_body(d, blockIdx.x); }
__global__ void __launch_bounds__(KDECIDE_THREADS) k_decide_b(const Dev* __restrict__ wins, const int2* __restrict__ items) { pdl_enter();
  __shared__ Dev sd;
  const int2 it = items[blockIdx.x];
  load_dev(sd, wins + it.x);
  k_decide_body(sd, it.y);
}

// ------------------------------------------------------------- evaluation
template <typename T>
__global__ void __launch_bounds__(LIN_THREADS) k_eval(Dev d, double huber, double zmin, double* part) {
  extern __shared__ __align__(16) double smem[];
  const LinTile tile = d.lin_tiles[blockIdx.x];
  double* s_red = smem;
  T* s_rig = reinterpret_cast<T*>(s_red + 128);
  const T* rig = st_rig<T>(d);
  for (int i = threadIdx.x; i < d.C * RIG_STRIDE; i += blockDim.x) s_rig[i] = rig[i];
  __syncthreads();
  const int cur = d.ctrl->cur;
  const T* pose = st_pose<T>(d, cur);
  const T* lmp = st_lm<T>(d, cur);
  PairStats<T> st;
  for (int q = tile.p0 + threadIdx.x; q < tile.p1; q += blockDim.x) {
    const int a = d.pair_kf[q], j = d.pair_lm[q];
    T X[3];
    eval_pair<T, false>(pose + a * POSE_STRIDE, lmp + 3 * j, d.pair_obs[q], d.pair_obs[q + 1], d.obs_cam,
                        reinterpret_cast<const T*>(d.obs_uv), s_rig, (T)huber, (T)zmin, X, nullptr, nullptr, st);
  }
  double v[4] = {st.cost.value(), st.sq.value(), (double)st.nv, (double)st.ni};
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
    if (mode == 0 && d.mixed)
      for (int k = 0; k < POSE_STRIDE; ++k) d.pose_f[cur][i * POSE_STRIDE + k] = (float)P[k];
  } else {
    if (i >= d.M) return;
    double* L = d.lm[cur] + 3 * i;
    double* U = user + 3 * (size_t)lm_order[i];
    for (int k = 0; k < 3; ++k) {
      if (mode == 1) L[k] = U[k]; else U[k] = L[k];
    }
    if (mode == 1 && d.mixed)
      for (int k = 0; k < 3; ++k) d.lm_f[cur][3 * i + k] = (float)L[k];
  }
}

size_t tsize(const Dev& d) { return d.mixed ? sizeof(float) : sizeof(double); }
size_t lin_smem(const Dev& d) { return d.mixed ? lin_smem_bytes<float>(d.C) : lin_smem_bytes<double>(d.C); }
size_t backsub_smem(const Dev& d) { return d.mixed ? backsub_smem_bytes<float>(d.C) : backsub_smem_bytes<double>(d.C); }
size_t eval_smem(const Dev& d) { return sizeof(double) * 128 + tsize(d) * d.C * RIG_STRIDE; }
constexpr int kCholSmemMaxN = 160;
size_t chol_smem(int n) { return sizeof(double) * ((size_t)n * n + n); }
constexpr size_t kClusterSmemMax = kClusterSmemMaxBytes;
int g_cluster_max = 16;                         // largest cluster size the device launches

// Cluster size for the distributed Cholesky, or 0 when the system is too large for the
// cluster's shared memory (then the single-CTA global-memory kernel runs).
int chol_cluster_size(int n_c) {
  for (int cs : {16, 8}) {
    if (cs > g_cluster_max) continue;
    if (chol_layout(n_c, cs).doubles() * sizeof(double) <= kClusterSmemMax) return cs;
  }
  return 0;
}

}  // namespace

// ================================================================ launchers

// Programmatic dependent launch for the iteration kernels (captured into the solve graph as
// programmatic edges).  cluster > 0 adds a cluster dimension.
bool g_pdl = true;
template <typename... P, typename... A>
cudaError_t launch_ex(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int cluster, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (cluster > 0) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = cluster;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  if (g_pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Opt a kernel into `want` bytes of dynamic shared memory, clamped to what is left of the
// 227 KB per-CTA limit after its static shared memory (the batched kernels stage their
// window's Dev there).  Launches request far less than the clamp except the Cholesky ones,
// whose plans are checked against the same limit.
template <typename F>
cudaError_t set_dyn_smem(F* f, size_t want) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  const size_t limit = 227 * 1024 - fa.sharedSizeBytes;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::min(want, limit));
}

cudaError_t set_kernel_attributes() {
  cudaError_t e;
  const size_t big = 227 * 1024;
  if ((e = set_dyn_smem(k_lin<double>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_lin<float>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_direct<double>, SchurSmem<double>::bytes())) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_direct<float>, SchurSmem<float>::bytes())) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_group<double>, group_smem_bytes(SPAN_MAX, false))) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_group<float>, group_smem_bytes(SPAN_MAX, true))) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_chol<true>, chol_smem(kCholSmemMaxN))) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_chol_cluster, kClusterSmemMax)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chol_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
    return e;
  if ((e = set_dyn_smem(k_chol_cluster_b, kClusterSmemMax)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_chol_cluster_b, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
    return e;
  if ((e = set_dyn_smem(k_lin_b<float>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_lin_b<double>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_backsub_b<float>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_backsub_b<double>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_backsub<float>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_backsub<double>, big)) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_group_b<float>, group_smem_bytes(SPAN_MAX, true))) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_group_b<double>, group_smem_bytes(SPAN_MAX, false))) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_direct_b<float>, SchurSmem<float>::bytes())) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_schur_direct_b<double>, SchurSmem<double>::bytes())) != cudaSuccess) return e;
  if ((e = set_dyn_smem(k_chol_b<true>, chol_smem(kCholSmemMaxN))) != cudaSuccess) return e;
  {
    // largest cluster of 256-thread CTAs with the maximum shared memory that fits
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = kClusterSmemMax;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n_clusters = 0;
    g_cluster_max = (cudaOccupancyMaxActiveClusters(&n_clusters, k_chol_cluster, &cfg) == cudaSuccess &&
                     n_clusters > 0) ? 16 : 8;
    cudaGetLastError();
  }
  return cudaSuccess;
}

int kernels_per_iteration() { return 7; }
int kernels_per_solve_init() { return 1; }

cudaError_t enqueue_solve_init(const Dev& d, double lam0, double huber, double zmin, int iters, int reset,
                               int refine, cudaStream_t s) {
  k_solve_init<<<1, 256, 0, s>>>(d, lam0, huber, zmin, iters, reset, refine);
  return cudaGetLastError();
}

// One part per kernel of the iteration (a part whose kernel is not launched for this
// window's plan reads as zero).
// chol: the reduced-system solve (the cluster kernel, after k_blk_load in the blocked form).
int profile_parts() { return 8; }
const char* profile_names() { return "lin,kf_reduce,schur_group,rcs_reduce,schur_direct,chol,backsub,decide"; }

cudaError_t enqueue_iteration(const Dev& d, cudaStream_t s, cudaEvent_t* ev, const SideStream* side) {
  cudaError_t e;
  auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
  if ((e = mark(0)) != cudaSuccess) return e;
  if (d.mixed)
    { if ((e = launch_ex(k_lin<float>, dim3(d.n_lin_tiles), dim3(LIN_THREADS), lin_smem(d), s, 0, d)) != cudaSuccess) return e; }
  else
    { if ((e = launch_ex(k_lin<double>, dim3(d.n_lin_tiles), dim3(LIN_THREADS), lin_smem(d), s, 0, d)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(1)) != cudaSuccess) return e;
  { if ((e = launch_ex(k_kf_reduce, dim3(d.K), dim3(384), 0, s, 0, d)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(2)) != cudaSuccess) return e;
  if (d.n_schur_tiles > 0) {
    const size_t sm = group_smem_bytes(d.max_span, d.mixed != 0);
    if (d.mixed)
      { if ((e = launch_ex(k_schur_group<float>, dim3(d.n_schur_tiles), dim3(group_threads<float>()), sm, s, 0, d)) != cudaSuccess) return e; }
    else
      { if ((e = launch_ex(k_schur_group<double>, dim3(d.n_schur_tiles), dim3(group_threads<double>()), sm, s, 0, d)) != cudaSuccess) return e; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = mark(3)) != cudaSuccess) return e;
  { if ((e = launch_ex(k_rcs_reduce, dim3(d.n_act), dim3(256), 0, s, 0, d)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(4)) != cudaSuccess) return e;
  if (d.n_direct_tiles > 0) {
    if (d.mixed)
      { if ((e = launch_ex(k_schur_direct<float>, dim3(d.n_direct_tiles), dim3(SCHUR_THREADS), SchurSmem<float>::bytes(), s, 0, d)) != cudaSuccess) return e; }
    else
      { if ((e = launch_ex(k_schur_direct<double>, dim3(d.n_direct_tiles), dim3(SCHUR_THREADS), SchurSmem<double>::bytes(), s, 0, d)) != cudaSuccess) return e; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }

  if ((e = mark(5)) != cudaSuccess) return e;
  if (chol_cluster_size(d.n_c) > 0) {
    const int CS = chol_cluster_size(d.n_c);
    size_t smem = chol_layout(d.n_c, CS).doubles() * sizeof(double);
    if (d.chol_blocked) {
      // the cluster kernel factors by panels from the working copy, then solves
      const size_t n_load = std::min(((size_t)d.npw * d.npw + 255) / 256, (size_t)152 * 8);
      if ((e = launch_ex(k_blk_load, dim3((unsigned)n_load), dim3(256), 0, s, 0, d)) != cudaSuccess) return e;
      smem = std::max(smem, blk_cluster_smem(d.npw));
    }
    if ((e = launch_ex(k_chol_cluster, dim3(CS), dim3(256), smem, s, CS, d)) != cudaSuccess) return e;
  } else if (d.n_c <= kCholSmemMaxN) {
    { if ((e = launch_ex(k_chol<true>, dim3(1), dim3(CHOL_THREADS), chol_smem(d.n_c), s, 0, d)) != cudaSuccess) return e; }
  } else {
    { if ((e = launch_ex(k_chol<false>, dim3(1), dim3(CHOL_THREADS), 0, s, 0, d)) != cudaSuccess) return e; }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(6)) != cudaSuccess) return e;
  if (d.mixed)
    { if ((e = launch_ex(k_backsub<float>, dim3(d.n_lin_tiles), dim3(LIN_THREADS), backsub_smem(d), s, 0, d)) != cudaSuccess) return e; }
  else
    { if ((e = launch_ex(k_backsub<double>, dim3(d.n_lin_tiles), dim3(LIN_THREADS), backsub_smem(d), s, 0, d)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = mark(7)) != cudaSuccess) return e;
  { if ((e = launch_ex(k_decide, dim3(1), dim3(KDECIDE_THREADS), 0, s, 0, d)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return mark(8);
}

int solve_kernels_per_iteration(const Dev& d) {
  int blocked = 0;
  if (chol_cluster_size(d.n_c) > 0 && d.chol_blocked) blocked = 1;   // k_blk_load
  return 6 + (d.n_schur_tiles > 0 ? 1 : 0) + (d.n_direct_tiles > 0 ? 1 : 0) + blocked;
}

void batch_plan_sizes(Dev* hd, int n_win, BatchLaunch& b) {
  b.lin_smem = b.backsub_smem = b.group_smem = b.chol_smem = 0;
  b.direct_smem = hd[0].mixed ? SchurSmem<float>::bytes() : SchurSmem<double>::bytes();
  b.n_fallback = 0;
  int max_span = 1;
  for (int w = 0; w < n_win; ++w) {
    const Dev& d = hd[w];
    b.lin_smem = std::max(b.lin_smem, lin_smem(d));
    b.backsub_smem = std::max(b.backsub_smem, backsub_smem(d));
    max_span = std::max(max_span, d.max_span);
    const size_t cs = chol_layout(d.n_c, b.chol_cs).doubles() * sizeof(double);
    hd[w].chol_fallback = cs > kClusterSmemMax ? 1 : 0;
    hd[w].chol_blocked = 0;                        // batched windows factor in their cluster
    if (hd[w].chol_fallback) b.n_fallback++;
    else b.chol_smem = std::max(b.chol_smem, cs);
  }
  b.group_smem = group_smem_bytes(max_span, hd[0].mixed != 0);
}

int batch_kernels_per_iteration(const BatchLaunch& b) {
  return 6 + (b.n_schur > 0 ? 1 : 0) + (b.n_direct > 0 ? 1 : 0) + b.n_fallback;
}

cudaError_t enqueue_batch_init(const BatchLaunch& b, double lam0, double huber, double zmin, int iters, int reset,
                               int refine, cudaStream_t s) {
  k_solve_init_b<<<b.n_win, 256, 0, s>>>(b.wins, lam0, huber, zmin, iters, reset, refine);
  return cudaGetLastError();
}

cudaError_t enqueue_batch_iteration(const BatchLaunch& b, cudaStream_t s) {
  cudaError_t e;
  if (b.mixed)
    { if ((e = launch_ex(k_lin_b<float>, dim3(b.n_lin), dim3(LIN_THREADS), b.lin_smem, s, 0, b.wins, b.lin_items)) != cudaSuccess) return e; }
  else
    { if ((e = launch_ex(k_lin_b<double>, dim3(b.n_lin), dim3(LIN_THREADS), b.lin_smem, s, 0, b.wins, b.lin_items)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  { if ((e = launch_ex(k_kf_reduce_b, dim3(b.n_kf), dim3(384), 0, s, 0, b.wins, b.kf_items)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (b.n_schur > 0) {
    if (b.mixed)
      { if ((e = launch_ex(k_schur_group_b<float>, dim3(b.n_schur), dim3(group_threads<float>()), b.group_smem, s, 0, b.wins, b.schur_items)) != cudaSuccess) return e; }
    else
      { if ((e = launch_ex(k_schur_group_b<double>, dim3(b.n_schur), dim3(group_threads<double>()), b.group_smem, s, 0, b.wins, b.schur_items)) != cudaSuccess) return e; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  { if ((e = launch_ex(k_rcs_reduce_b, dim3(b.n_blkit), dim3(256), 0, s, 0, b.wins, b.blk_items)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (b.n_direct > 0) {
    if (b.mixed)
      { if ((e = launch_ex(k_schur_direct_b<float>, dim3(b.n_direct), dim3(SCHUR_THREADS), b.direct_smem, s, 0, b.wins, b.direct_items)) != cudaSuccess) return e; }
    else
      { if ((e = launch_ex(k_schur_direct_b<double>, dim3(b.n_direct), dim3(SCHUR_THREADS), b.direct_smem, s, 0, b.wins, b.direct_items)) != cudaSuccess) return e; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (b.n_fallback < b.n_win) {
    if ((e = launch_ex(k_chol_cluster_b, dim3(b.n_win * b.chol_cs), dim3(256), b.chol_smem, s, b.chol_cs, b.wins)) !=
        cudaSuccess)
      return e;
  }
  for (int f = 0; f < b.n_fallback; ++f) {
    const Dev& d = b.fallback_host[f];
    if (d.n_c <= kCholSmemMaxN)
      { if ((e = launch_ex(k_chol<true>, dim3(1), dim3(CHOL_THREADS), chol_smem(d.n_c), s, 0, d)) != cudaSuccess) return e; }
    else
      { if ((e = launch_ex(k_chol<false>, dim3(1), dim3(CHOL_THREADS), 0, s, 0, d)) != cudaSuccess) return e; }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (b.mixed)
    { if ((e = launch_ex(k_backsub_b<float>, dim3(b.n_lin), dim3(LIN_THREADS), b.backsub_smem, s, 0, b.wins, b.lin_items)) != cudaSuccess) return e; }
  else
    { if ((e = launch_ex(k_backsub_b<double>, dim3(b.n_lin), dim3(LIN_THREADS), b.backsub_smem, s, 0, b.wins, b.lin_items)) != cudaSuccess) return e; }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  { if ((e = launch_ex(k_decide_b, dim3(b.n_win), dim3(KDECIDE_THREADS), 0, s, 0, b.wins, b.win_items)) != cudaSuccess) return e; }
  return cudaGetLastError();
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
