// Motion-only bundle adjustment (multi-camera PnP), batched over independent frames, and the
// loop-closure relative pose that is the same problem with the landmarks shifted into a map
// frame.
//
// cuVSLAM (arXiv 2506.04359) estimates the pose of every tracked frame from the 2D
// observations of map landmarks (Sec. 2.2.1 stereo, Eq. PnP over the two cameras; Sec. 2.2.2
// multi-stereo, the same sum over every camera of the rig):
//     T^bw = argmin  sum_j sum_k rho(|pi(T^cb_k T^bw p^w_j) - o_{j,k}|^2),
// the landmarks held fixed.  The residual, Jacobian, Huber weights, Marquardt diagonal,
// Nielsen damping update and accept rule are those of the bundle-adjustment solve, with a
// single 6-DoF pose: the normal equations are one 6 x 6 system.  The loop-closure step
// (Sec. 2.3, relative pose estimation) solves T^bm = argmin sum rho(|pi(T^cb_k T^bm T^mw p^w_j)
// - o_{j,k}|^2) for a fixed map pose T^mw per query frame: the landmarks are staged as
// T^mw p^w_j (in FP64) and the rest is the PnP solve.
//
// Design: one CTA per frame runs all LM iterations of its frame (frames are independent,
// so a batch is one launch with no grid-wide waits).  The frame's observations, with their
// landmark positions gathered, are staged in shared memory once when they fit, so every
// iteration's two passes (linearisation and candidate cost) read shared memory only.  Each
// thread accumulates its observations' 21 + 6 normal-equation terms, cost and counts; the
// block sums them in a fixed order with a reduce-scatter butterfly (31 adds per warp for
// 32 values instead of 5 per value).  One thread then factors the damped 6 x 6 system in
// FP64, forms the candidate pose and, after the candidate-cost pass, takes the accept
// decision.  T = double is the FP64 path; T = float runs the per-observation arithmetic in
// FP32 with two-float (TwoSum) warp sums, converted to FP64 once per warp, and keeps the
// solve, the pose and the decision in FP64.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/cvba.h"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kNV = 32;               // H (21, upper triangle row-major), g (6), F, sum r^2, n_valid, n_inlier, pad
constexpr int kCMax = 64;
constexpr size_t kSmemCap = 200 * 1024;

template <typename T>
struct ObsS {        // one staged observation
  T u, v, x, y, z;
  int cam;
};

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Reduce-scatter over the warp: on return v[0] of lane l is the warp's sum of value l.
// The pairing order is fixed, so the result is reproducible.
__device__ __forceinline__ void warp_reduce_scatter(double v[kNV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = lane & s;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const double send = up ? v[i] : v[i + s];
      const double keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

// Two-float version: (hi, lo) pairs summed with TwoSum.
__device__ __forceinline__ void warp_reduce_scatter_df(float h[kNV], float l[kNV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = lane & s;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float sh = up ? h[i] : h[i + s], sl = up ? l[i] : l[i + s];
      const float kh = up ? h[i + s] : h[i], kl = up ? l[i + s] : l[i];
      const float oh = __shfl_xor_sync(0xffffffffu, sh, s), ol = __shfl_xor_sync(0xffffffffu, sl, s);
      float s1, e1;
      two_sum(kh, oh, s1, e1);
      e1 += kl + ol;
      two_sum(s1, e1, h[i], l[i]);
    }
  }
}

// Block sum of the per-thread values into out[kNV] (FP64), fixed order.
template <typename T>
__device__ __forceinline__ void block_sum(T v[kNV], double* red, double* out);

template <>
__device__ __forceinline__ void block_sum<double>(double v[kNV], double* red, double* out) {
  warp_reduce_scatter(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  red[warp * kNV + lane] = v[0];
  __syncthreads();
  if (warp == 0) {
    double s = red[lane];
    for (int w = 1; w < kWarps; ++w) s += red[w * kNV + lane];
    out[lane] = s;
  }
  __syncthreads();
}

template <>
__device__ __forceinline__ void block_sum<float>(float v[kNV], double* red, double* out) {
  float lo[kNV];
#pragma unroll
  for (int i = 0; i < kNV; ++i) lo[i] = 0.f;
  warp_reduce_scatter_df(v, lo);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  red[warp * kNV + lane] = (double)v[0] + (double)lo[0];
  __syncthreads();
  if (warp == 0) {
    double s = red[lane];
    for (int w = 1; w < kWarps; ++w) s += red[w * kNV + lane];
    out[lane] = s;
  }
  __syncthreads();
}

// Single-value block sum (candidate cost), fixed order.
template <typename T>
__device__ __forceinline__ double block_sum1(T v, double* red) {
  double d = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = d;
  __syncthreads();
  double s = red[0];
  for (int w = 1; w < kWarps; ++w) s += red[w];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------- observation model

// Residual and (if JAC) the 2 x 6 Jacobian with respect to the left twist of the pose.
// P: pose [R (row-major) | t] as R0..R8, t0..t2; Q: camera fx fy cx cy, R_cb (9), t_cb (3).
template <typename T, bool JAC>
__device__ __forceinline__ bool obs_eval(const T* P, const T* Q, T px, T py, T pz, T ou, T ov, T zmin, T r[2],
                                         T J[2][6]) {
  const T xb = P[0] * px + P[1] * py + P[2] * pz + P[9];
  const T yb = P[3] * px + P[4] * py + P[5] * pz + P[10];
  const T zb = P[6] * px + P[7] * py + P[8] * pz + P[11];
  const T xc = Q[4] * xb + Q[5] * yb + Q[6] * zb + Q[13];
  const T yc = Q[7] * xb + Q[8] * yb + Q[9] * zb + Q[14];
  const T zc = Q[10] * xb + Q[11] * yb + Q[12] * zb + Q[15];
  if (!(zc > zmin)) return false;
  const T iz = T(1) / zc;
  const T xn = xc * iz, yn = yc * iz;
  r[0] = Q[0] * xn + Q[2] - ou;
  r[1] = Q[1] * yn + Q[3] - ov;
  if (JAC) {
    // A = dpi/dX_c R_cb, rows a0, a1
    const T f0 = Q[0] * iz, f1 = Q[1] * iz;
    T a0[3], a1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      a0[b] = f0 * (Q[4 + b] - xn * Q[10 + b]);
      a1[b] = f1 * (Q[7 + b] - yn * Q[10 + b]);
    }
    // J = [A | A (-[X_b]x)]; -[X_b]x = [[0, zb, -yb], [-zb, 0, xb], [yb, -xb, 0]]
    J[0][0] = a0[0], J[0][1] = a0[1], J[0][2] = a0[2];
    J[1][0] = a1[0], J[1][1] = a1[1], J[1][2] = a1[2];
    J[0][3] = a0[2] * yb - a0[1] * zb;
    J[0][4] = a0[0] * zb - a0[2] * xb;
    J[0][5] = a0[1] * xb - a0[0] * yb;
    J[1][3] = a1[2] * yb - a1[1] * zb;
    J[1][4] = a1[0] * zb - a1[2] * xb;
    J[1][5] = a1[1] * xb - a1[0] * yb;
  }
  return true;
}

// -------------------------------------------------------------- SE(3) and 6 x 6 solve

// Left update T1 = Exp(xi) T0 (xi = (rho, phi)); Rodrigues coefficients A = sin t / t,
// B = (1 - cos t) / t^2, C = (t - sin t) / t^3 from their Taylor series in t^2 below
// t = 0.1 (truncation below 1e-21) and from sin / cos above.
__device__ void pose_plus(const double* T0, const double* xi, double* T1) {
  const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
  const double t2 = w0 * w0 + w1 * w1 + w2 * w2;
  double A, B, C;
  if (t2 < 0.01) {
    A = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880 + t2 * (-1.0 / 39916800)))));
    B = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800 + t2 * (-1.0 / 479001600)))));
    C = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800 +
                                                                              t2 * (-1.0 / 6227020800.0)))));
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    A = s / t;
    B = (1.0 - c) / t2;
    C = (t - s) / (t2 * t);
  }
  // W = [phi]x, W^2 = phi phi^T - t2 I
  const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
  double Re[9], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double w2ij = xi[3 + i] * xi[3 + j] - (i == j ? t2 : 0.0);
      Re[3 * i + j] = (i == j ? 1.0 : 0.0) + A * W[3 * i + j] + B * w2ij;
      V[3 * i + j] = (i == j ? 1.0 : 0.0) + B * W[3 * i + j] + C * w2ij;
    }
  double te[3];
  for (int i = 0; i < 3; ++i) te[i] = V[3 * i] * xi[0] + V[3 * i + 1] * xi[1] + V[3 * i + 2] * xi[2];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      T1[3 * i + j] = Re[3 * i] * T0[j] + Re[3 * i + 1] * T0[3 + j] + Re[3 * i + 2] * T0[6 + j];
    T1[9 + i] = Re[3 * i] * T0[9] + Re[3 * i + 1] * T0[10] + Re[3 * i + 2] * T0[11] + te[i];
  }
}

__device__ __forceinline__ int hidx(int i, int j) {   // upper-triangle row-major index, i <= j
  return i * 6 - i * (i - 1) / 2 + (j - i);
}

// delta solving (H + lam D) delta = -g by Cholesky; false if not positive definite.
__device__ bool solve6(const double* Hs, const double* g, const double* D, double lam, double* delta) {
  double L[36];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j <= i; ++j) L[6 * i + j] = Hs[hidx(j, i)] + (i == j ? lam * D[i] : 0.0);
  for (int j = 0; j < 6; ++j) {
    double d = L[6 * j + j];
    for (int k = 0; k < j; ++k) d -= L[6 * j + k] * L[6 * j + k];
    if (!(d > 0.0) || !isfinite(d)) return false;
    const double l = sqrt(d);
    L[6 * j + j] = l;
    for (int i = j + 1; i < 6; ++i) {
      double s = L[6 * i + j];
      for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
      L[6 * i + j] = s / l;
    }
  }
  double y[6];
  for (int i = 0; i < 6; ++i) {
    double s = -g[i];
    for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
    y[i] = s / L[6 * i + i];
  }
  for (int i = 5; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * delta[k];
    delta[i] = s / L[6 * i + i];
  }
  for (int i = 0; i < 6; ++i)
    if (!isfinite(delta[i])) return false;
  return true;
}

// ----------------------------------------------------------------------- kernel

struct PnpArgs {
  int n_frames, n_cams, n_lm, iters;
  double lam0, huber, zmin;
  const void* intr;
  const void* T_cb;
  const void* p_w;
  const int32_t* frame_off;
  const int32_t* cam;
  const int32_t* lm;
  const void* uv;
  double* T_bw;
  cvba_lm_record* trace;
  const double* T_mw;       // per-frame fixed transform applied to the landmarks, or null
};

struct PnpShared {
  double pose[12], cand[12];
  double lin[kNV];          // sums at the linearisation point
  double red[kWarps * kNV];
  double lam, nu, F1;
  int need_lin, nonpd, accept;
};

// The landmark position the frame's residuals use: p itself, or T^mw p (FP64) when the frame
// has a fixed transform (the loop-closure query: landmarks shifted into the map frame).
template <typename T>
__device__ __forceinline__ void landmark_in_frame(const PnpArgs& a, int f, const T* p, T q[3]) {
  if (!a.T_mw) {
    q[0] = p[0], q[1] = p[1], q[2] = p[2];
    return;
  }
  const double* M = a.T_mw + 12 * (size_t)f;
  const double x = (double)p[0], y = (double)p[1], z = (double)p[2];
  for (int r = 0; r < 3; ++r) q[r] = (T)(M[4 * r] * x + M[4 * r + 1] * y + M[4 * r + 2] * z + M[4 * r + 3]);
}

template <typename T, bool STAGED>
__global__ void __launch_bounds__(kThreads) k_pnp(PnpArgs a) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ PnpShared sh;
  __shared__ T rig[kCMax * 16];
  __shared__ T pose_t[12], cand_t[12];
  const int f = blockIdx.x, tid = threadIdx.x;
  const int o0 = a.frame_off[f], o1 = a.frame_off[f + 1], n = o1 - o0;
  const T* intr = static_cast<const T*>(a.intr);
  const T* tcb = static_cast<const T*>(a.T_cb);
  const T* pw = static_cast<const T*>(a.p_w);
  const T* uv = static_cast<const T*>(a.uv);
  for (int c = tid; c < a.n_cams; c += kThreads) {
    T* q = rig + 16 * c;
    for (int k = 0; k < 4; ++k) q[k] = intr[4 * c + k];
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) q[4 + 3 * r + k] = tcb[12 * c + 4 * r + k];
      q[13 + r] = tcb[12 * c + 4 * r + 3];
    }
  }
  if (tid < 3) {
    for (int k = 0; k < 3; ++k) sh.pose[3 * tid + k] = a.T_bw[12 * (size_t)f + 4 * tid + k];
    sh.pose[9 + tid] = a.T_bw[12 * (size_t)f + 4 * tid + 3];
  }
  if (tid == 0) {
    sh.lam = a.lam0;
    sh.nu = 2.0;
    sh.need_lin = 1;
  }
  // stage observations (landmark positions gathered); out-of-range indices are marked
  // with cam = -1 and skipped
  ObsS<T>* so = reinterpret_cast<ObsS<T>*>(dyn);
  int bad = 0;
  if (STAGED) {
    for (int i = tid; i < n; i += kThreads) {
      const int c = a.cam[o0 + i], j = a.lm[o0 + i];
      ObsS<T> o;
      const bool ok = c >= 0 && c < a.n_cams && j >= 0 && j < a.n_lm;
      o.cam = ok ? c : -1;
      o.u = uv[2 * (size_t)(o0 + i)];
      o.v = uv[2 * (size_t)(o0 + i) + 1];
      T q[3] = {T(0), T(0), T(0)};
      if (ok) landmark_in_frame(a, f, pw + 3 * (size_t)j, q);
      o.x = q[0];
      o.y = q[1];
      o.z = q[2];
      so[i] = o;
      bad += ok ? 0 : 1;
    }
  } else {
    for (int i = tid; i < n; i += kThreads) {
      const int c = a.cam[o0 + i], j = a.lm[o0 + i];
      bad += (c >= 0 && c < a.n_cams && j >= 0 && j < a.n_lm) ? 0 : 1;
    }
  }
  __syncthreads();
  const int n_bad = (int)block_sum1<double>((double)bad, sh.red);
  const T zmin = (T)a.zmin, hub = (T)a.huber;

  auto fetch = [&](int i, T& u, T& v, T& x, T& y, T& z) -> int {
    if (STAGED) {
      const ObsS<T> o = so[i];
      u = o.u, v = o.v, x = o.x, y = o.y, z = o.z;
      return o.cam;
    }
    const int c = a.cam[o0 + i], j = a.lm[o0 + i];
    if (c < 0 || c >= a.n_cams || j < 0 || j >= a.n_lm) return -1;
    u = uv[2 * (size_t)(o0 + i)], v = uv[2 * (size_t)(o0 + i) + 1];
    T q[3];
    landmark_in_frame(a, f, pw + 3 * (size_t)j, q);
    x = q[0], y = q[1], z = q[2];
    return c;
  };

  for (int it = 0; it < a.iters; ++it) {
    if (sh.need_lin) {
      if (tid < 12) pose_t[tid] = (T)sh.pose[tid];
      __syncthreads();
      T acc[kNV];
#pragma unroll
      for (int k = 0; k < kNV; ++k) acc[k] = T(0);
      for (int i = tid; i < n; i += kThreads) {
        T u, v, x, y, z;
        const int c = fetch(i, u, v, x, y, z);
        if (c < 0) continue;
        T r[2], J[2][6];
        if (!obs_eval<T, true>(pose_t, rig + 16 * c, x, y, z, u, v, zmin, r, J)) continue;
        const T s = r[0] * r[0] + r[1] * r[1];
        const T e = sqrt(s);
        const bool inl = e <= hub;
        const T w = inl ? T(1) : hub / e;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const T wj0 = w * J[0][p], wj1 = w * J[1][p];
#pragma unroll
          for (int q = p; q < 6; ++q) acc[hidx(p, q)] += wj0 * J[0][q] + wj1 * J[1][q];
          acc[21 + p] += wj0 * r[0] + wj1 * r[1];
        }
        acc[27] += T(0.5) * (inl ? s : T(2) * hub * e - hub * hub);
        acc[28] += s;
        acc[29] += T(1);
        acc[30] += inl ? T(1) : T(0);
      }
      block_sum<T>(acc, sh.red, sh.lin);
    }
    // damped 6 x 6 solve and candidate pose (FP64, one thread)
    double delta[6] = {0, 0, 0, 0, 0, 0}, D[6], L = 0.0;
    if (tid == 0) {
      const double* H = sh.lin;
      double dmax = 0.0;
      for (int i = 0; i < 6; ++i) dmax = fmax(dmax, H[hidx(i, i)]);
      for (int i = 0; i < 6; ++i) D[i] = fmax(H[hidx(i, i)], 1e-12 * dmax);
      const bool ok = solve6(H, H + 21, D, sh.lam, delta);
      sh.nonpd = ok ? 0 : 1;
      if (ok) {
        for (int i = 0; i < 6; ++i) L += delta[i] * (sh.lam * D[i] * delta[i] - H[21 + i]);
        L *= 0.5;
        pose_plus(sh.pose, delta, sh.cand);
      }
    }
    __syncthreads();
    double F1 = CUDART_NAN;
    if (!sh.nonpd) {
      if (tid < 12) cand_t[tid] = (T)sh.cand[tid];
      __syncthreads();
      T fc = T(0);
      for (int i = tid; i < n; i += kThreads) {
        T u, v, x, y, z;
        const int c = fetch(i, u, v, x, y, z);
        if (c < 0) continue;
        T r[2], J[2][6];
        if (!obs_eval<T, false>(cand_t, rig + 16 * c, x, y, z, u, v, zmin, r, J)) continue;
        const T s = r[0] * r[0] + r[1] * r[1];
        const T e = sqrt(s);
        fc += T(0.5) * (e <= hub ? s : T(2) * hub * e - hub * hub);
      }
      F1 = block_sum1<T>(fc, sh.red);
    }
    if (tid == 0) {
      const double F0 = sh.lin[27];
      const double gain = sh.nonpd ? CUDART_NAN : (L != 0.0 ? (F0 - F1) / L : CUDART_NAN);
      const bool acc = !sh.nonpd && L > 0.0 && isfinite(F1) && gain > 0.0;
      cvba_lm_record* rec = a.trace ? a.trace + (size_t)f * a.iters + it : nullptr;
      if (rec) {
        double sn = 0.0;
        for (int i = 0; i < 6; ++i) sn += delta[i] * delta[i];
        rec->cost0 = F0;
        rec->cost1 = F1;
        rec->lambda = sh.lam;
        rec->gain = gain;
        rec->pred = sh.nonpd ? CUDART_NAN : L;
        rec->step_norm = sh.nonpd ? CUDART_NAN : sqrt(sn);
        rec->rms_px = sh.lin[29] > 0.0 ? sqrt(sh.lin[28] / sh.lin[29]) : 0.0;
        rec->accepted = acc ? 1 : 0;
        rec->nonpd = sh.nonpd;
        rec->n_valid = (int)sh.lin[29];
        rec->n_inlier = (int)sh.lin[30];
        rec->n_bad_index = n_bad;
        rec->reserved = 0;
      }
      if (acc) {
        sh.lam *= fmax(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) * (2.0 * gain - 1.0) * (2.0 * gain - 1.0));
        sh.nu = 2.0;
        for (int k = 0; k < 12; ++k) sh.pose[k] = sh.cand[k];
      } else {
        sh.lam *= sh.nu;
        sh.nu *= 2.0;
      }
      sh.need_lin = acc ? 1 : 0;
    }
    __syncthreads();
  }
  if (tid < 3) {
    for (int k = 0; k < 3; ++k) a.T_bw[12 * (size_t)f + 4 * tid + k] = sh.pose[3 * tid + k];
    a.T_bw[12 * (size_t)f + 4 * tid + 3] = sh.pose[9 + tid];
  }
}

template <typename T, bool STAGED>
cudaError_t launch(const PnpArgs& a, size_t smem, cudaStream_t s) {
  // the attribute is per device and function: set it on every call (cheap)
  cudaError_t e = cudaFuncSetAttribute(k_pnp<T, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
  if (e != cudaSuccess) return e;
  k_pnp<T, STAGED><<<a.n_frames, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

namespace {
cvba_status pnp_solve(int dtype, int n_frames, int n_cams, int n_lm, int n_obs, const void* intr, const void* T_cb,
                      const void* p_w, const int32_t* frame_off, const int32_t* cam, const int32_t* lm,
                      const void* uv, const double* T_mw, double* T_bw, const cvba_opts* opts,
                      cvba_lm_record* trace, void* stream) {
  if ((dtype != 0 && dtype != 1) || n_frames < 1 || n_cams < 1 || n_cams > kCMax || n_lm < 1 || n_obs < 0 || !opts)
    return CVBA_ERR_INVALID_ARG;
  if (!intr || !T_cb || !p_w || !frame_off || !T_bw || (n_obs > 0 && (!cam || !lm || !uv)))
    return CVBA_ERR_INVALID_ARG;
  if (opts->iters < 0 || !(opts->huber_delta > 0.0) || !std::isfinite(opts->huber_delta) ||
      !std::isfinite(opts->z_min) || !(opts->lambda0 > 0.0) || !std::isfinite(opts->lambda0))
    return CVBA_ERR_INVALID_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the frames' observation segments: validated on the host (sizes the staging too)
  std::vector<int32_t> off((size_t)n_frames + 1);
  if (cudaMemcpyAsync(off.data(), frame_off, off.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  if (off[0] != 0 || off[n_frames] != n_obs) return CVBA_ERR_INVALID_ARG;
  int max_n = 0;
  for (int f = 0; f < n_frames; ++f) {
    if (off[f + 1] < off[f]) return CVBA_ERR_INVALID_ARG;
    max_n = std::max(max_n, off[f + 1] - off[f]);
  }
  if (opts->iters == 0) return CVBA_OK;
  PnpArgs a{n_frames, n_cams, n_lm, opts->iters, opts->lambda0, opts->huber_delta, opts->z_min,
            intr, T_cb, p_w, frame_off, cam, lm, uv, T_bw, trace, T_mw};
  const size_t per = dtype == 0 ? sizeof(ObsS<double>) : sizeof(ObsS<float>);
  const size_t smem = per * (size_t)max_n;
  cudaError_t e;
  if (smem <= kSmemCap)
    e = dtype == 0 ? launch<double, true>(a, smem, s) : launch<float, true>(a, smem, s);
  else
    e = dtype == 0 ? launch<double, false>(a, 0, s) : launch<float, false>(a, 0, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CVBA_ERR_OOM : CVBA_ERR_CUDA;
  }
  return CVBA_OK;
}

}  // namespace

extern "C" cvba_status cvba_pnp_solve(int dtype, int n_frames, int n_cams, int n_lm, int n_obs, const void* intr,
                                      const void* T_cb, const void* p_w, const int32_t* frame_off,
                                      const int32_t* cam, const int32_t* lm, const void* uv, double* T_bw,
                                      const cvba_opts* opts, cvba_lm_record* trace, void* stream) {
  return pnp_solve(dtype, n_frames, n_cams, n_lm, n_obs, intr, T_cb, p_w, frame_off, cam, lm, uv, nullptr, T_bw, opts,
                   trace, stream);
}

extern "C" cvba_status cvba_relpose_solve(int dtype, int n_frames, int n_cams, int n_lm, int n_obs, const void* intr,
                                          const void* T_cb, const void* p_w, const int32_t* frame_off,
                                          const int32_t* cam, const int32_t* lm, const void* uv, const double* T_mw,
                                          double* T_bm, const cvba_opts* opts, cvba_lm_record* trace, void* stream) {
  if (!T_mw) return CVBA_ERR_INVALID_ARG;
  return pnp_solve(dtype, n_frames, n_cams, n_lm, n_obs, intr, T_cb, p_w, frame_off, cam, lm, uv, T_mw, T_bm, opts,
                   trace, stream);
}

extern "C" int cvba_pnp_kernels_per_solve(void) { return 1; }
