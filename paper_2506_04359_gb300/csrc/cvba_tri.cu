// Multi-view landmark triangulation, batched over landmarks.
//
// cuVSLAM (arXiv 2506.04359, Sec. 2.2 "3D module") triangulates the new landmarks of a
// keyframe from their multi-view observations; the results are the landmarks the bundle
// adjustment refines.  For each landmark j with observations (keyframe i, camera k, pixel o),
// with the keyframe poses T^bw_i and the rig held fixed:
//   1. linear triangulation: with x = ((u - cx)/fx, (v - cy)/fy) and [R | t] = T^cb_k T^bw_i,
//      each observation gives x (R_3 p + t_3) = R_1 p + t_1 and y (R_3 p + t_3) = R_2 p + t_2;
//      p0 solves these in the least-squares sense (inhomogeneous DLT), through the 3 x 3
//      normal equations factored by Cholesky in FP64 with one step of iterative refinement
//      (corrected semi-normal equations, Bjorck, "Numerical Methods for Least Squares
//      Problems", 1996, Sec. 2.2.3), which restores the accuracy of an orthogonal solve;
//   2. opts->iters Levenberg-Marquardt iterations on p alone: the bundle-adjustment step
//      restricted to one landmark (Huber IRLS weights, Marquardt diagonal, Nielsen's update,
//      accept iff the predicted reduction and the gain are positive), a 3 x 3 system.
//
// Design: one thread per landmark (landmarks are independent and small: a few to a few tens
// of observations), the block's keyframe poses and rig in shared memory, the observations
// read from the landmark's segment on every pass (L1 resident after the first).  A whole
// batch is one launch.  T = double is the FP64 path; T = float runs the refinement's
// per-observation arithmetic in FP32 (the linear step, the 3 x 3 solves, the landmark state
// and the decisions stay FP64).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/cvba.h"

namespace {

constexpr int kThreads = 128;
constexpr int kKMax = 256;
constexpr int kCMax = 64;

struct TriArgs {
  int n_lm, n_kf, n_cams, iters;
  double lam0, huber, zmin;
  const void* intr;
  const void* T_cb;
  const double* T_bw;
  const int32_t* lm_off;
  const int32_t* kf;
  const int32_t* cam;
  const void* uv;
  double* p_lin;
  double* p_w;
  int32_t* status;
  cvba_lm_record* trace;
};

// Cholesky solve of the 3 x 3 SPD system (a00 a01 a02 a11 a12 a22) x = b; false if a pivot
// is not above tol (relative to the largest diagonal entry) or not finite.
__device__ bool solve3(const double a[6], const double b[3], double x[3], double rel_tol) {
  const double dmax = fmax(a[0], fmax(a[3], a[5]));
  const double tol = rel_tol * dmax;
  const double l00 = a[0];
  if (!(l00 > tol) || !isfinite(l00)) return false;
  const double s0 = sqrt(l00);
  const double l10 = a[1] / s0, l20 = a[2] / s0;
  const double d1 = a[3] - l10 * l10;
  if (!(d1 > tol) || !isfinite(d1)) return false;
  const double s1 = sqrt(d1);
  const double l21 = (a[4] - l20 * l10) / s1;
  const double d2 = a[5] - l20 * l20 - l21 * l21;
  if (!(d2 > tol) || !isfinite(d2)) return false;
  const double s2 = sqrt(d2);
  const double y0 = b[0] / s0, y1 = (b[1] - l10 * y0) / s1, y2 = (b[2] - l20 * y0 - l21 * y1) / s2;
  x[2] = y2 / s2;
  x[1] = (y1 - l21 * x[2]) / s1;
  x[0] = (y0 - l10 * x[1] - l20 * x[2]) / s0;
  return isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
}

// Residual of one observation at point (px, py, pz) and, if JAC, its 2 x 3 Jacobian.
// P: keyframe pose R (row-major), t; Q: camera fx fy cx cy, R_cb (9), t_cb (3).
template <typename T, bool JAC>
__device__ __forceinline__ bool obs_eval(const T* P, const T* Q, T px, T py, T pz, T ou, T ov, T zmin, T r[2],
                                         T J[2][3]) {
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
    // J = dpi/dX_c R_cb R_i
    const T f0 = Q[0] * iz, f1 = Q[1] * iz;
    T a0[3], a1[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      a0[b] = f0 * (Q[4 + b] - xn * Q[10 + b]);
      a1[b] = f1 * (Q[7 + b] - yn * Q[10 + b]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      J[0][b] = a0[0] * P[b] + a0[1] * P[3 + b] + a0[2] * P[6 + b];
      J[1][b] = a1[0] * P[b] + a1[1] * P[3 + b] + a1[2] * P[6 + b];
    }
  }
  return true;
}

// Dynamic shared memory: FP64 poses (K x 12) and rig (C x 16), then their T copies for the
// FP32 path (the FP64 path reads the FP64 arrays).
size_t tri_smem(int dtype, int K, int C) {
  const size_t n = (size_t)K * 12 + (size_t)C * 16;
  return sizeof(double) * n + (dtype == 1 ? sizeof(float) * n : 0);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_triangulate(TriArgs a) {
  extern __shared__ __align__(16) double smem_d[];
  double* pose_d = smem_d;
  double* rig_d = pose_d + 12 * a.n_kf;
  T* pose_t;
  T* rig_t;
  if (sizeof(T) == sizeof(double)) {
    pose_t = reinterpret_cast<T*>(pose_d);
    rig_t = reinterpret_cast<T*>(rig_d);
  } else {
    pose_t = reinterpret_cast<T*>(rig_d + 16 * a.n_cams);
    rig_t = pose_t + 12 * a.n_kf;
  }
  const T* intr = static_cast<const T*>(a.intr);
  const T* tcb = static_cast<const T*>(a.T_cb);
  const T* uv = static_cast<const T*>(a.uv);
  for (int i = threadIdx.x; i < a.n_kf * 12; i += kThreads) {
    const int k = i / 12, e = i % 12;   // R row-major then t, from [R | t] rows
    const double v = e < 9 ? a.T_bw[12 * k + 4 * (e / 3) + e % 3] : a.T_bw[12 * k + 4 * (e - 9) + 3];
    pose_d[i] = v;
    if (sizeof(T) != sizeof(double)) pose_t[i] = (T)v;
  }
  for (int c = threadIdx.x; c < a.n_cams; c += kThreads) {
    double q[16];
    for (int k = 0; k < 4; ++k) q[k] = (double)intr[4 * c + k];
    for (int r = 0; r < 3; ++r) {
      for (int k = 0; k < 3; ++k) q[4 + 3 * r + k] = (double)tcb[12 * c + 4 * r + k];
      q[13 + r] = (double)tcb[12 * c + 4 * r + 3];
    }
    for (int k = 0; k < 16; ++k) {
      rig_d[16 * c + k] = q[k];
      if (sizeof(T) != sizeof(double)) rig_t[16 * c + k] = (T)q[k];
    }
  }
  __syncthreads();
  const int j = blockIdx.x * kThreads + threadIdx.x;
  if (j >= a.n_lm) return;
  const int o0 = a.lm_off[j], o1 = a.lm_off[j + 1];
  auto valid_idx = [&](int n) {
    const int i = a.kf[n], c = a.cam[n];
    return i >= 0 && i < a.n_kf && c >= 0 && c < a.n_cams;
  };
  int n_bad = 0, n_ok = 0;
  for (int n = o0; n < o1; ++n) {
    const bool v = valid_idx(n);
    n_bad += v ? 0 : 1;
    n_ok += v ? 1 : 0;
  }
  double p[3] = {CUDART_NAN, CUDART_NAN, CUDART_NAN};
  int st = 0;
  if (n_ok < 2) {
    st = 1;
  } else {
    // linear step: normal equations of the stacked DLT rows, FP64
    double N[6] = {0, 0, 0, 0, 0, 0}, c[3] = {0, 0, 0};
    for (int n = o0; n < o1; ++n) {
      if (!valid_idx(n)) continue;
      const double* P = pose_d + 12 * a.kf[n];
      const double* Q = rig_d + 16 * a.cam[n];
      double R[9], t[3];
      for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) R[3 * r + k] = Q[4 + 3 * r] * P[k] + Q[5 + 3 * r] * P[3 + k] + Q[6 + 3 * r] * P[6 + k];
        t[r] = Q[4 + 3 * r] * P[9] + Q[5 + 3 * r] * P[10] + Q[6 + 3 * r] * P[11] + Q[13 + r];
      }
      const double x = ((double)uv[2 * (size_t)n] - Q[2]) / Q[0];
      const double y = ((double)uv[2 * (size_t)n + 1] - Q[3]) / Q[1];
      for (int row = 0; row < 2; ++row) {
        const double s = row == 0 ? x : y;
        double A[3];
        for (int k = 0; k < 3; ++k) A[k] = s * R[6 + k] - R[3 * row + k];
        const double b = t[row] - s * t[2];
        N[0] += A[0] * A[0], N[1] += A[0] * A[1], N[2] += A[0] * A[2];
        N[3] += A[1] * A[1], N[4] += A[1] * A[2], N[5] += A[2] * A[2];
        c[0] += A[0] * b, c[1] += A[1] * b, c[2] += A[2] * b;
      }
    }
    if (!solve3(N, c, p, 1e-14)) {
      st = 2;
    } else {
      // one step of iterative refinement on the linear system (corrected semi-normal
      // equations): N dp = A^T (b - A p) recovers the accuracy the normal equations lose to
      // the squared condition number
      double c2[3] = {0, 0, 0}, dp[3];
      for (int n = o0; n < o1; ++n) {
        if (!valid_idx(n)) continue;
        const double* P = pose_d + 12 * a.kf[n];
        const double* Q = rig_d + 16 * a.cam[n];
        double R[9], t[3];
        for (int r = 0; r < 3; ++r) {
          for (int k = 0; k < 3; ++k) R[3 * r + k] = Q[4 + 3 * r] * P[k] + Q[5 + 3 * r] * P[3 + k] + Q[6 + 3 * r] * P[6 + k];
          t[r] = Q[4 + 3 * r] * P[9] + Q[5 + 3 * r] * P[10] + Q[6 + 3 * r] * P[11] + Q[13 + r];
        }
        const double x = ((double)uv[2 * (size_t)n] - Q[2]) / Q[0];
        const double y = ((double)uv[2 * (size_t)n + 1] - Q[3]) / Q[1];
        for (int row = 0; row < 2; ++row) {
          const double s = row == 0 ? x : y;
          double A[3];
          for (int k = 0; k < 3; ++k) A[k] = s * R[6 + k] - R[3 * row + k];
          const double res = (t[row] - s * t[2]) - (A[0] * p[0] + A[1] * p[1] + A[2] * p[2]);
          c2[0] += A[0] * res, c2[1] += A[1] * res, c2[2] += A[2] * res;
        }
      }
      if (solve3(N, c2, dp, 0.0))
        for (int k = 0; k < 3; ++k) p[k] += dp[k];
    }
  }
  if (a.p_lin) {
    for (int k = 0; k < 3; ++k) a.p_lin[3 * (size_t)j + k] = st == 0 ? p[k] : CUDART_NAN;
  }
  if (st != 0) {
    for (int k = 0; k < 3; ++k) a.p_w[3 * (size_t)j + k] = CUDART_NAN;
    if (a.status) a.status[j] = st;
    return;
  }
  // refinement
  const T zmin = (T)a.zmin, hub = (T)a.huber;
  double lam = a.lam0, nu = 2.0;
  bool need_lin = true;
  double H[6] = {0}, g[3] = {0}, F0 = 0.0, ssq = 0.0;
  int nv = 0, ni = 0;
  for (int it = 0; it < a.iters; ++it) {
    if (need_lin) {
      const T px = (T)p[0], py = (T)p[1], pz = (T)p[2];
      T h[6] = {0, 0, 0, 0, 0, 0}, gg[3] = {0, 0, 0}, F = 0, S = 0;
      nv = 0, ni = 0;
      for (int n = o0; n < o1; ++n) {
        if (!valid_idx(n)) continue;
        T r[2], J[2][3];
        if (!obs_eval<T, true>(pose_t + 12 * a.kf[n], rig_t + 16 * a.cam[n], px, py, pz, uv[2 * (size_t)n],
                               uv[2 * (size_t)n + 1], zmin, r, J))
          continue;
        const T s = r[0] * r[0] + r[1] * r[1];
        const T e = sqrt(s);
        const bool inl = e <= hub;
        const T w = inl ? T(1) : hub / e;
        const T w0[3] = {w * J[0][0], w * J[0][1], w * J[0][2]}, w1[3] = {w * J[1][0], w * J[1][1], w * J[1][2]};
        h[0] += w0[0] * J[0][0] + w1[0] * J[1][0];
        h[1] += w0[0] * J[0][1] + w1[0] * J[1][1];
        h[2] += w0[0] * J[0][2] + w1[0] * J[1][2];
        h[3] += w0[1] * J[0][1] + w1[1] * J[1][1];
        h[4] += w0[1] * J[0][2] + w1[1] * J[1][2];
        h[5] += w0[2] * J[0][2] + w1[2] * J[1][2];
        for (int k = 0; k < 3; ++k) gg[k] += w0[k] * r[0] + w1[k] * r[1];
        F += T(0.5) * (inl ? s : T(2) * hub * e - hub * hub);
        S += s;
        nv += 1;
        ni += inl ? 1 : 0;
      }
      for (int k = 0; k < 6; ++k) H[k] = (double)h[k];
      for (int k = 0; k < 3; ++k) g[k] = (double)gg[k];
      F0 = (double)F;
      ssq = (double)S;
    }
    // Marquardt diagonal floored at 1e-12 of its largest entry
    const double dmax = fmax(H[0], fmax(H[3], H[5]));
    const double D[3] = {fmax(H[0], 1e-12 * dmax), fmax(H[3], 1e-12 * dmax), fmax(H[5], 1e-12 * dmax)};
    const double A[6] = {H[0] + lam * D[0], H[1], H[2], H[3] + lam * D[1], H[4], H[5] + lam * D[2]};
    const double mg[3] = {-g[0], -g[1], -g[2]};
    double delta[3];
    const bool ok = solve3(A, mg, delta, 0.0);
    double F1 = CUDART_NAN, L = CUDART_NAN, gain = CUDART_NAN;
    bool acc = false;
    if (ok) {
      L = 0.0;
      for (int k = 0; k < 3; ++k) L += delta[k] * (lam * D[k] * delta[k] - g[k]);
      L *= 0.5;
      const double q[3] = {p[0] + delta[0], p[1] + delta[1], p[2] + delta[2]};
      const T qx = (T)q[0], qy = (T)q[1], qz = (T)q[2];
      T F = 0;
      for (int n = o0; n < o1; ++n) {
        if (!valid_idx(n)) continue;
        T r[2], J[2][3];
        if (!obs_eval<T, false>(pose_t + 12 * a.kf[n], rig_t + 16 * a.cam[n], qx, qy, qz, uv[2 * (size_t)n],
                                uv[2 * (size_t)n + 1], zmin, r, J))
          continue;
        const T s = r[0] * r[0] + r[1] * r[1];
        const T e = sqrt(s);
        F += T(0.5) * (e <= hub ? s : T(2) * hub * e - hub * hub);
      }
      F1 = (double)F;
      gain = L != 0.0 ? (F0 - F1) / L : CUDART_NAN;
      acc = L > 0.0 && isfinite(F1) && gain > 0.0;
      if (acc)
        for (int k = 0; k < 3; ++k) p[k] = q[k];
    }
    if (a.trace) {
      cvba_lm_record* rec = a.trace + (size_t)j * a.iters + it;
      rec->cost0 = F0;
      rec->cost1 = F1;
      rec->lambda = lam;
      rec->gain = gain;
      rec->pred = L;
      rec->step_norm = ok ? sqrt(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]) : CUDART_NAN;
      rec->rms_px = nv > 0 ? sqrt(ssq / nv) : 0.0;
      rec->accepted = acc ? 1 : 0;
      rec->nonpd = ok ? 0 : 1;
      rec->n_valid = nv;
      rec->n_inlier = ni;
      rec->n_bad_index = n_bad;
      rec->reserved = 0;
    }
    if (acc) {
      lam *= fmax(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) * (2.0 * gain - 1.0) * (2.0 * gain - 1.0));
      nu = 2.0;
    } else {
      lam *= nu;
      nu *= 2.0;
    }
    need_lin = acc;
  }
  for (int k = 0; k < 3; ++k) a.p_w[3 * (size_t)j + k] = p[k];
  if (a.status) a.status[j] = 0;
}

}  // namespace

extern "C" cvba_status cvba_triangulate(int dtype, int n_lm, int n_kf, int n_cams, int n_obs, const void* intr,
                                        const void* T_cb, const double* T_bw, const int32_t* lm_off,
                                        const int32_t* kf, const int32_t* cam, const void* uv, const cvba_opts* opts,
                                        double* p_lin, double* p_w, int32_t* status, cvba_lm_record* trace,
                                        void* stream) {
  if ((dtype != 0 && dtype != 1) || n_lm < 1 || n_kf < 1 || n_kf > kKMax || n_cams < 1 || n_cams > kCMax ||
      n_obs < 0 || !opts)
    return CVBA_ERR_INVALID_ARG;
  if (!intr || !T_cb || !T_bw || !lm_off || !p_w || (n_obs > 0 && (!kf || !cam || !uv))) return CVBA_ERR_INVALID_ARG;
  if (opts->iters < 0 || !(opts->huber_delta > 0.0) || !std::isfinite(opts->huber_delta) ||
      !std::isfinite(opts->z_min) || !(opts->lambda0 > 0.0) || !std::isfinite(opts->lambda0))
    return CVBA_ERR_INVALID_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int32_t> off((size_t)n_lm + 1);
  if (cudaMemcpyAsync(off.data(), lm_off, off.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  if (off[0] != 0 || off[n_lm] != n_obs) return CVBA_ERR_INVALID_ARG;
  for (int j = 0; j < n_lm; ++j)
    if (off[j + 1] < off[j]) return CVBA_ERR_INVALID_ARG;
  TriArgs a{n_lm, n_kf, n_cams, opts->iters, opts->lambda0, opts->huber_delta, opts->z_min, intr, T_cb, T_bw,
            lm_off, kf, cam, uv, p_lin, p_w, status, trace};
  const int grid = (n_lm + kThreads - 1) / kThreads;
  const size_t smem = tri_smem(dtype, n_kf, n_cams);
  cudaError_t e;
  if (dtype == 0) {
    e = cudaFuncSetAttribute(k_triangulate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_triangulate<double><<<grid, kThreads, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_triangulate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_triangulate<float><<<grid, kThreads, smem, s>>>(a);
  }
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  return CVBA_OK;
}
