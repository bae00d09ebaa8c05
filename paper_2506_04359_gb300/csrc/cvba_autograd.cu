// Differentiable robust reprojection cost (cuVSLAM Sec. 2.2, Eq. r^repr and the SBA
// objective): forward F = 1/2 sum_n rho(|r_n|^2) and its hand-written adjoint.
//
// Inputs are caller-owned device arrays in one floating type (FP64 or FP32), in the
// caller's order (no layout): intrinsics (C x 4), rig extrinsics T_cb (C x 12), tangent
// perturbations xi (K x 6, translation first), keyframe poses T_bw (K x 12), landmarks
// (M x 3), observations (kf, cam, lm int32; uv N x 2).  The pose of keyframe i is
// T'_i = Exp(xi_i) T_i (left update), so xi = 0 gives the gradient in the tangent space
// at T_i.  The backward pass recomputes every Jacobian (nothing is stored between the
// passes) and returns
//   dF/dxi   = J_l(xi)^T [g_X; X' x g_X] summed over the keyframe's observations,
//   dF/dT    = R_e^T g_X (x) [p; 1]   (the 3 x 4 matrix entries),
//   dF/dp    = R'^T g_X,
//   dF/dintr = w (r_u X/Z, r_v Y/Z, r_u, r_v),
// with g_X = w A^T r (A = d pi / d X'), all scaled by the upstream gradient, and J_l the
// left Jacobian of SE(3) (Barfoot, "State Estimation for Robotics", 2017).
// Per-keyframe and per-camera sums are per-CTA partials reduced in a fixed order;
// landmark gradients are accumulated with atomics (few observations per landmark).
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/cvba.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxCtas = 1216;           // 8 x 152 SMs: bounds the partial-sum workspace
constexpr int kKfVals = 18;              // per keyframe: left-tangent gradient (6), dF/dT (12)
constexpr double kTaylor = 1e-4;

size_t n_ctas(int n_obs) {
  const size_t c = ((size_t)n_obs + kThreads - 1) / kThreads;
  return c < kMaxCtas ? (c > 0 ? c : 1) : kMaxCtas;
}

// Workspace (doubles): per-CTA cost partial, per-CTA keyframe and camera partials, then
// the K exponentials T'_i (12 each) and the K left Jacobians J_l(xi_i) (36 each).
size_t ws_doubles(int n_obs, int n_kf, int n_cams) {
  const size_t g = n_ctas(n_obs);
  return g + g * ((size_t)n_kf * kKfVals + (size_t)n_cams * 4) + (size_t)n_kf * 12 + (size_t)n_kf * 36 + 8;
}

template <typename T>
__device__ __forceinline__ double ld(const T* p, size_t i) {
  return (double)p[i];
}

// T' = Exp(xi) T (SE(3) exponential: Rodrigues, t' = R_e t + V rho) and, for the backward
// pass, J_l(xi) = [[J, Q], [0, J]] (row-major 6 x 6), J = V the SO(3) left Jacobian,
// Q(rho, phi) from Barfoot (2017) Eq. (7.86).  Thread per keyframe; FP64 throughout.
template <typename T>
__global__ void k_ad_poses(int n_kf, const T* __restrict__ xi, const T* __restrict__ T_bw, T* __restrict__ Tp,
                           double* __restrict__ Jl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_kf) return;
  double rho[3], ph[3];
  for (int k = 0; k < 3; ++k) {
    rho[k] = ld(xi, 6 * (size_t)i + k);
    ph[k] = ld(xi, 6 * (size_t)i + 3 + k);
  }
  const double th2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
  const double th = sqrt(th2);
  double A, B, C, D, E;                            // Rodrigues / V / Q coefficients
  if (th < kTaylor) {
    A = 1.0 - th2 / 6.0;
    B = 0.5 - th2 / 24.0;
    C = 1.0 / 6.0 - th2 / 120.0;
    D = 1.0 / 24.0 - th2 / 720.0;                  // (th^2 + 2 cos th - 2) / (2 th^4)
    E = 1.0 / 120.0 - th2 / 2520.0;                // (2 th - 3 sin th + th cos th) / (2 th^5)
  } else {
    const double s = sin(th), c = cos(th);
    A = s / th;
    B = (1.0 - c) / th2;
    C = (th - s) / (th2 * th);
    D = (th2 + 2.0 * c - 2.0) / (2.0 * th2 * th2);
    E = (2.0 * th - 3.0 * s + th * c) / (2.0 * th2 * th2 * th);
  }
  double P[9] = {0.0, -ph[2], ph[1], ph[2], 0.0, -ph[0], -ph[1], ph[0], 0.0};
  double Rr[9] = {0.0, -rho[2], rho[1], rho[2], 0.0, -rho[0], -rho[1], rho[0], 0.0};
  auto mm = [](const double* a, const double* b, double* c) {
    for (int r = 0; r < 3; ++r)
      for (int q = 0; q < 3; ++q) c[r * 3 + q] = a[r * 3] * b[q] + a[r * 3 + 1] * b[3 + q] + a[r * 3 + 2] * b[6 + q];
  };
  double P2[9], Re[9], V[9];
  mm(P, P, P2);
  for (int k = 0; k < 9; ++k) {
    const double I = (k % 4 == 0) ? 1.0 : 0.0;
    Re[k] = I + A * P[k] + B * P2[k];
    V[k] = I + B * P[k] + C * P2[k];
  }
  double te[3];
  for (int r = 0; r < 3; ++r) te[r] = V[r * 3] * rho[0] + V[r * 3 + 1] * rho[1] + V[r * 3 + 2] * rho[2];
  double T0[12];
  for (int k = 0; k < 12; ++k) T0[k] = ld(T_bw, 12 * (size_t)i + k);   // [R | t] row-major 3 x 4
  T* out = Tp + 12 * (size_t)i;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q)
      out[r * 4 + q] = (T)(Re[r * 3] * T0[q] + Re[r * 3 + 1] * T0[4 + q] + Re[r * 3 + 2] * T0[8 + q]);
    out[r * 4 + 3] = (T)(Re[r * 3] * T0[3] + Re[r * 3 + 1] * T0[7] + Re[r * 3 + 2] * T0[11] + te[r]);
  }
  if (!Jl) return;
  // Q = 1/2 Rr + C (P Rr + Rr P + P Rr P) + D (P2 Rr + Rr P2 - 3 P Rr P) + E (P Rr P2 + P2 Rr P)
  double PR[9], RP[9], PRP[9], P2R[9], RP2[9], PRP2[9], P2RP[9];
  mm(P, Rr, PR);
  mm(Rr, P, RP);
  mm(PR, P, PRP);
  mm(P2, Rr, P2R);
  mm(Rr, P2, RP2);
  mm(PR, P2, PRP2);
  mm(P2R, P, P2RP);
  double Q[9];
  for (int k = 0; k < 9; ++k)
    Q[k] = 0.5 * Rr[k] + C * (PR[k] + RP[k] + PRP[k]) + D * (P2R[k] + RP2[k] - 3.0 * PRP[k]) + E * (PRP2[k] + P2RP[k]);
  double* J = Jl + 36 * (size_t)i;
  for (int r = 0; r < 6; ++r)
    for (int q = 0; q < 6; ++q) {
      double v = 0.0;
      if (r < 3 && q < 3) v = V[r * 3 + q];
      else if (r < 3) v = Q[r * 3 + q - 3];
      else if (q >= 3) v = V[(r - 3) * 3 + q - 3];
      J[r * 6 + q] = v;
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
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
};

// One observation in the compute type T: X' = R' p + t', X_c = R_cb X' + t_cb.  Returns
// false for an index out of range.
template <typename T>
__device__ __forceinline__ bool ad_obs(int n, int n_kf, int n_cams, int n_lm, const T* T_cb, const T* Tp,
                                       const T* p_w, const int32_t* kf, const int32_t* cam, const int32_t* lm,
                                       T X[3], T Xc[3], int& i, int& c, int& j) {
  i = kf[n];
  c = cam[n];
  j = lm[n];
  if (i < 0 || i >= n_kf || c < 0 || c >= n_cams || j < 0 || j >= n_lm) return false;
  const T* P = Tp + 12 * (size_t)i;
  const T p0 = p_w[3 * (size_t)j], p1 = p_w[3 * (size_t)j + 1], p2 = p_w[3 * (size_t)j + 2];
  for (int a = 0; a < 3; ++a) X[a] = P[a * 4] * p0 + P[a * 4 + 1] * p1 + P[a * 4 + 2] * p2 + P[a * 4 + 3];
  const T* Q = T_cb + 12 * (size_t)c;
  for (int a = 0; a < 3; ++a) Xc[a] = Q[a * 4] * X[0] + Q[a * 4 + 1] * X[1] + Q[a * 4 + 2] * X[2] + Q[a * 4 + 3];
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ad_forward(int n_obs, int n_kf, int n_cams, int n_lm,
                                                         const T* intr, const T* T_cb, const T* Tp,
                                                         const T* p_w, const int32_t* kf, const int32_t* cam,
                                                         const int32_t* lm, const T* uv, T hub, T zmin,
                                                         double* part) {
  __shared__ double red[32];
  Acc<T> acc;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_obs; n += gridDim.x * blockDim.x) {
    T X[3], Xc[3];
    int i, c, j;
    if (!ad_obs(n, n_kf, n_cams, n_lm, T_cb, Tp, p_w, kf, cam, lm, X, Xc, i, c, j)) continue;
    if (!(Xc[2] > zmin)) continue;
    const T u = intr[4 * (size_t)c] * Xc[0] / Xc[2] + intr[4 * (size_t)c + 2];
    const T v = intr[4 * (size_t)c + 1] * Xc[1] / Xc[2] + intr[4 * (size_t)c + 3];
    const T r0 = u - uv[2 * (size_t)n], r1 = v - uv[2 * (size_t)n + 1];
    const T s = r0 * r0 + r1 * r1, e = sqrt(s);
    acc.add((T)0.5 * (e <= hub ? s : (T)2 * hub * e - hub * hub));
  }
  double a = warp_sum(acc.value());
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

template <typename T>
__global__ void k_ad_cost_reduce(const double* part, int g, T* out) {
  __shared__ double red[32];
  double v = 0.0;
  for (int k = threadIdx.x; k < g; k += blockDim.x) v += part[k];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
    if (threadIdx.x == 0) *out = (T)s;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_ad_backward(int n_obs, int n_kf, int n_cams, int n_lm,
                                                          const T* intr, const T* T_cb, const T* Tp,
                                                          const T* T_bw, const T* p_w, const int32_t* kf,
                                                          const int32_t* cam, const int32_t* lm, const T* uv,
                                                          T hub, T zmin, const T* grad_out, T* g_p,
                                                          double* kf_part, double* cam_part) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  T* s_acc = reinterpret_cast<T*>(s_raw);          // n_kf * 18 + n_cams * 4
  const int nk = n_kf * kKfVals, na = nk + n_cams * 4;
  for (int k = threadIdx.x; k < na; k += blockDim.x) s_acc[k] = 0;
  __syncthreads();
  const T go = grad_out[0];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < n_obs; n += gridDim.x * blockDim.x) {
    T X[3], Xc[3];
    int i, c, j;
    if (!ad_obs(n, n_kf, n_cams, n_lm, T_cb, Tp, p_w, kf, cam, lm, X, Xc, i, c, j)) continue;
    if (!(Xc[2] > zmin)) continue;
    const T fx = intr[4 * (size_t)c], fy = intr[4 * (size_t)c + 1];
    const T iz = (T)1 / Xc[2], xn = Xc[0] * iz, yn = Xc[1] * iz;
    const T r0 = fx * Xc[0] / Xc[2] + intr[4 * (size_t)c + 2] - uv[2 * (size_t)n];
    const T r1 = fy * Xc[1] / Xc[2] + intr[4 * (size_t)c + 3] - uv[2 * (size_t)n + 1];
    const T s = r0 * r0 + r1 * r1, e = sqrt(s);
    const T w = (e <= hub ? (T)1 : hub / e) * go;
    // g_Xc = J_pi^T (w r), g_X = R_cb^T g_Xc
    const T gxc0 = w * fx * iz * r0, gxc1 = w * fy * iz * r1;
    const T gxc2 = -w * (fx * xn * iz * r0 + fy * yn * iz * r1);
    const T* Q = T_cb + 12 * (size_t)c;
    T gX[3];
    for (int a = 0; a < 3; ++a) gX[a] = Q[a] * gxc0 + Q[4 + a] * gxc1 + Q[8 + a] * gxc2;
    const T* P = Tp + 12 * (size_t)i;
    T u3[3];                                       // R'^T g_X
    for (int a = 0; a < 3; ++a) u3[a] = P[a] * gX[0] + P[4 + a] * gX[1] + P[8 + a] * gX[2];
    if (g_p)
      for (int a = 0; a < 3; ++a) atomicAdd(g_p + 3 * (size_t)j + a, u3[a]);
    T* ka = s_acc + kKfVals * i;
    // left tangent at T': (g_X, X' x g_X)
    atomicAdd(ka + 0, gX[0]);
    atomicAdd(ka + 1, gX[1]);
    atomicAdd(ka + 2, gX[2]);
    atomicAdd(ka + 3, X[1] * gX[2] - X[2] * gX[1]);
    atomicAdd(ka + 4, X[2] * gX[0] - X[0] * gX[2]);
    atomicAdd(ka + 5, X[0] * gX[1] - X[1] * gX[0]);
    // base pose matrix: X' = R_e (R p + t) + t_e, h = R_e^T g_X = R R'^T g_X;
    // dF/dR = h p^T, dF/dt = h
    const T p0 = p_w[3 * (size_t)j], p1 = p_w[3 * (size_t)j + 1], p2 = p_w[3 * (size_t)j + 2];
    const T* B = T_bw + 12 * (size_t)i;
    for (int a = 0; a < 3; ++a) {
      const T h = B[a * 4] * u3[0] + B[a * 4 + 1] * u3[1] + B[a * 4 + 2] * u3[2];
      atomicAdd(ka + 6 + a * 4, h * p0);
      atomicAdd(ka + 6 + a * 4 + 1, h * p1);
      atomicAdd(ka + 6 + a * 4 + 2, h * p2);
      atomicAdd(ka + 6 + a * 4 + 3, h);
    }
    T* ca = s_acc + nk + 4 * c;
    atomicAdd(ca + 0, w * r0 * xn);
    atomicAdd(ca + 1, w * r1 * yn);
    atomicAdd(ca + 2, w * r0);
    atomicAdd(ca + 3, w * r1);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nk; k += blockDim.x) kf_part[(size_t)blockIdx.x * nk + k] = (double)s_acc[k];
  for (int k = threadIdx.x; k < n_cams * 4; k += blockDim.x)
    cam_part[(size_t)blockIdx.x * n_cams * 4 + k] = (double)s_acc[nk + k];
}

// Fixed-order sums of the per-CTA partials: dF/dT and dF/dintr (warp per output).
template <typename T>
__global__ void k_ad_grad_reduce(int g, int n_kf, int n_cams, const double* kf_part, const double* cam_part,
                                 T* g_T, T* g_intr) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nk = n_kf * kKfVals, nc = n_cams * 4;
  if (warp < nk) {
    const int i = warp / kKfVals, k = warp % kKfVals;
    if (k < 6 || !g_T) return;
    double v = 0.0;
    for (int b = lane; b < g; b += 32) v += kf_part[(size_t)b * nk + warp];
    v = warp_sum(v);
    if (lane == 0) g_T[12 * (size_t)i + k - 6] = (T)v;
  } else if (warp < nk + nc) {
    if (!g_intr) return;
    const int q = warp - nk;
    double v = 0.0;
    for (int b = lane; b < g; b += 32) v += cam_part[(size_t)b * nc + q];
    v = warp_sum(v);
    if (lane == 0) g_intr[q] = (T)v;
  }
}

// dF/dxi = J_l(xi)^T (left-tangent gradient at T'); warp per keyframe.
template <typename T>
__global__ void k_ad_apply_jl(int n_kf, int g, const double* kf_part, const double* Jl, T* g_xi) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n_kf) return;
  const int nk = n_kf * kKfVals;
  double gl[6];
  for (int k = 0; k < 6; ++k) {
    double v = 0.0;
    for (int b = lane; b < g; b += 32) v += kf_part[(size_t)b * nk + kKfVals * i + k];
    gl[k] = warp_sum(v);
  }
  if (lane < 6) {
    const double* J = Jl + 36 * (size_t)i;
    double v = 0.0;
    for (int r = 0; r < 6; ++r) v += J[r * 6 + lane] * gl[r];
    g_xi[6 * (size_t)i + lane] = (T)v;
  }
}

// Workspace layout (doubles): part[g] | kf_part[g * K * 18] | cam_part[g * C * 4] | Tp[K * 12]
// (stored in T) | Jl[K * 36].
template <typename T>
cvba_status forward_impl(int n_obs, int n_kf, int n_cams, int n_lm, const void* intr, const void* T_cb,
                         const void* xi, const void* T_bw, const void* p_w, const int32_t* kf, const int32_t* cam,
                         const int32_t* lm, const void* uv, double hub, double zmin, void* out, void* work,
                         cudaStream_t s) {
  double* ws = static_cast<double*>(work);
  const int g = (int)n_ctas(n_obs);
  double* part = ws;
  T* Tp = reinterpret_cast<T*>(ws + g + (size_t)g * ((size_t)n_kf * kKfVals + (size_t)n_cams * 4));
  k_ad_poses<T><<<(n_kf + 127) / 128, 128, 0, s>>>(n_kf, (const T*)xi, (const T*)T_bw, Tp, nullptr);
  k_ad_forward<T><<<g, kThreads, 0, s>>>(n_obs, n_kf, n_cams, n_lm, (const T*)intr, (const T*)T_cb, Tp,
                                         (const T*)p_w, kf, cam, lm, (const T*)uv, (T)hub, (T)zmin, part);
  k_ad_cost_reduce<T><<<1, 256, 0, s>>>(part, g, (T*)out);
  return cudaGetLastError() == cudaSuccess ? CVBA_OK : CVBA_ERR_CUDA;
}

template <typename T>
cvba_status backward_impl(int n_obs, int n_kf, int n_cams, int n_lm, const void* intr, const void* T_cb,
                          const void* xi, const void* T_bw, const void* p_w, const int32_t* kf, const int32_t* cam,
                          const int32_t* lm, const void* uv, double hub, double zmin, const void* grad_out,
                          void* g_xi, void* g_T, void* g_p, void* g_intr, void* work, cudaStream_t s) {
  double* ws = static_cast<double*>(work);
  const int g = (int)n_ctas(n_obs);
  double* kf_part = ws + g;
  double* cam_part = kf_part + (size_t)g * n_kf * kKfVals;
  double* Tpd = cam_part + (size_t)g * n_cams * 4;
  T* Tp = reinterpret_cast<T*>(Tpd);
  double* Jl = Tpd + 12 * (size_t)n_kf;
  if (g_p && cudaMemsetAsync(g_p, 0, sizeof(T) * 3 * (size_t)n_lm, s) != cudaSuccess) return CVBA_ERR_CUDA;
  k_ad_poses<T><<<(n_kf + 127) / 128, 128, 0, s>>>(n_kf, (const T*)xi, (const T*)T_bw, Tp, Jl);
  const size_t sm = sizeof(T) * ((size_t)n_kf * kKfVals + (size_t)n_cams * 4);
  k_ad_backward<T><<<g, kThreads, sm, s>>>(n_obs, n_kf, n_cams, n_lm, (const T*)intr, (const T*)T_cb, Tp,
                                           (const T*)T_bw, (const T*)p_w, kf, cam, lm, (const T*)uv, (T)hub,
                                           (T)zmin, (const T*)grad_out, (T*)g_p, kf_part, cam_part);
  const int warps = n_kf * kKfVals + n_cams * 4;
  k_ad_grad_reduce<T><<<(warps * 32 + 255) / 256, 256, 0, s>>>(g, n_kf, n_cams, kf_part, cam_part, (T*)g_T,
                                                               (T*)g_intr);
  if (g_xi) k_ad_apply_jl<T><<<(n_kf * 32 + 255) / 256, 256, 0, s>>>(n_kf, g, kf_part, Jl, (T*)g_xi);
  return cudaGetLastError() == cudaSuccess ? CVBA_OK : CVBA_ERR_CUDA;
}

bool args_ok(int dtype, int n_obs, int n_kf, int n_cams, int n_lm) {
  // per-CTA keyframe / camera accumulators live in shared memory: K <= 256, C <= 64
  return (dtype == 0 || dtype == 1) && n_obs >= 1 && n_kf >= 1 && n_kf <= 256 && n_cams >= 1 && n_cams <= 64 &&
         n_lm >= 1;
}

}  // namespace

extern "C" size_t cvba_cost_workspace_bytes(int n_obs, int n_kf, int n_cams) {
  if (n_obs < 1 || n_kf < 1 || n_cams < 1) return 0;
  return sizeof(double) * ws_doubles(n_obs, n_kf, n_cams);
}

extern "C" cvba_status cvba_cost_forward(int dtype, int n_obs, int n_kf, int n_cams, int n_lm, const void* intr,
                                         const void* T_cb, const void* xi, const void* T_bw, const void* p_w,
                                         const int32_t* kf, const int32_t* cam, const int32_t* lm, const void* uv,
                                         double huber_delta, double z_min, void* cost, void* work,
                                         size_t work_bytes, void* stream) {
  if (!args_ok(dtype, n_obs, n_kf, n_cams, n_lm)) return CVBA_ERR_INVALID_ARG;
  if (!intr || !T_cb || !xi || !T_bw || !p_w || !kf || !cam || !lm || !uv || !cost || !work)
    return CVBA_ERR_INVALID_ARG;
  if (!(huber_delta > 0.0) || work_bytes < cvba_cost_workspace_bytes(n_obs, n_kf, n_cams)) return CVBA_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  return dtype == 0 ? forward_impl<double>(n_obs, n_kf, n_cams, n_lm, intr, T_cb, xi, T_bw, p_w, kf, cam, lm, uv,
                                           huber_delta, z_min, cost, work, s)
                    : forward_impl<float>(n_obs, n_kf, n_cams, n_lm, intr, T_cb, xi, T_bw, p_w, kf, cam, lm, uv,
                                          huber_delta, z_min, cost, work, s);
}

extern "C" cvba_status cvba_cost_backward(int dtype, int n_obs, int n_kf, int n_cams, int n_lm, const void* intr,
                                          const void* T_cb, const void* xi, const void* T_bw, const void* p_w,
                                          const int32_t* kf, const int32_t* cam, const int32_t* lm, const void* uv,
                                          double huber_delta, double z_min, const void* grad_cost, void* g_xi,
                                          void* g_T_bw, void* g_p_w, void* g_intr, void* work, size_t work_bytes,
                                          void* stream) {
  if (!args_ok(dtype, n_obs, n_kf, n_cams, n_lm)) return CVBA_ERR_INVALID_ARG;
  if (!intr || !T_cb || !xi || !T_bw || !p_w || !kf || !cam || !lm || !uv || !grad_cost || !work)
    return CVBA_ERR_INVALID_ARG;
  if (!(huber_delta > 0.0) || work_bytes < cvba_cost_workspace_bytes(n_obs, n_kf, n_cams)) return CVBA_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == 0)
    return backward_impl<double>(n_obs, n_kf, n_cams, n_lm, intr, T_cb, xi, T_bw, p_w, kf, cam, lm, uv, huber_delta,
                                 z_min, grad_cost, g_xi, g_T_bw, g_p_w, g_intr, work, s);
  return backward_impl<float>(n_obs, n_kf, n_cams, n_lm, intr, T_cb, xi, T_bw, p_w, kf, cam, lm, uv, huber_delta,
                              z_min, grad_cost, g_xi, g_T_bw, g_p_w, g_intr, work, s);
}
