// Pose-graph optimisation (PGO) over keyframe poses.
//
// cuVSLAM (arXiv 2506.04359, Sec. 2.3, Eq. PGO) refines the map by minimising, over the
// edges E of the pose graph with measured deltas D_ij (frontend odometry or loop closures),
//     sum_{(i,j) in E} |Log(D_ij^-1 T_i^-1 T_j)|^2 .
// Readings: T_i are world-from-base poses; Log is the SE(3) logarithm with the twist
// (rho, phi), translation first; plain norm; one pose fixed (gauge); left updates
// T_i <- Exp(xi_i) T_i; the window solve's LM (Marquardt diagonal floored at 1e-12 max,
// Nielsen's update, accept iff L > 0 and gain > 0, exactly `iters` iterations).  With
// E = D^-1 T_i^-1 T_j and r = Log(E), dr/dxi_j = J_r(r)^-1 Ad(T_j^-1) = -dr/dxi_i.
//
// Design (FP64 throughout): per iteration
//   k_pgo_edges     thread per edge: r, J_i, J_j (6 x 6 each) and the edge cost, at the
//                   current poses (only after an accepted step: the linearisation is kept
//                   on a rejected one);
//   k_pgo_assemble  one CTA per structural block of H (each free pose's diagonal block with
//                   its gradient, each distinct pair of free poses joined by edges): sums of
//                   its edges' products in edge order (no atomics, reproducible);
//   k_pgo_load      the dense lower triangle of A = H + lambda D (zero outside the blocks);
//   k_pgo_potrf / k_pgo_trsm / k_pgo_syrk   right-looking Cholesky by 32-column panels: the
//                   diagonal block on one CTA, the panel's rows one warp each, the trailing
//                   update in 16 x 16 tiles over the GPU, each panel only over its envelope
//                   (the rows whose first coupled pose lies in or before the panel: the fill
//                   stays inside this profile);
//   k_pgo_solve     one CTA: L y = -g and L^T delta = y by 32-row panels over the same
//                   envelopes, the predicted reduction and the step norm;
//   k_pgo_candidate thread per pose: Exp(delta_i) T_i;  k_pgo_cost: thread per edge at the
//                   candidate;  k_pgo_decide: one CTA: fixed-order cost sums, gain, accept,
//                   damping, state swap, iteration record.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/cvba.h"

namespace {

constexpr int kPW = 32;   // panel width
constexpr int kPD = 33;   // shared-memory row stride of the diagonal block

struct PgoCtrl {
  int cur, need_lin, nonpd, it;
  double lam, nu, F, pred, step2;
};

// Device view of one solve (pointers into the caller's workspace).
struct Pgo {
  int K, E, nfree, n, npw, fixed, iters, n_pair;
  const int32_t* edges;      // E x 2
  const double* deltas;      // E x 12, [R | t] rows
  double* pose[2];           // K x 12, internal: R row-major (9), t (3)
  double* er;                // E x 6 residuals
  double* eJ;                // E x 72: J_i (6 x 6) then J_j, row-major
  double* ecost;             // E: edge cost at the linearisation point
  double* ccost;             // E: edge cost at the candidate
  double* Hd;                // nfree x 36 diagonal blocks
  double* Ho;                // n_pair x 36 off-diagonal blocks (rows: larger pose)
  double* g;                 // n
  double* D;                 // n Marquardt diagonal
  double* Lw;                // npw x npw factor (lower)
  double* x;                 // npw: y, then delta
  const int32_t* col;        // K: first column of each pose, -1 if fixed
  const int32_t* d_off;      // nfree + 1: (edge, side) contributions of each diagonal block
  const int32_t* d_list;     // 2 E entries: 2 * edge + side
  const int32_t* p_ab;       // n_pair x 2: (a, b) free poses, a > b, by column
  const int32_t* p_off;      // n_pair + 1
  const int32_t* p_list;     // edges of each pair, with side of a in bit 0 (2 * edge + (a is j))
  const int32_t* pend;       // npw / 32: end of each panel's envelope (rows [32 (p + 1), pend[p])
                             // are the only ones with nonzeros in panel p's columns)
  PgoCtrl* ctrl;
  cvba_lm_record* trace;
};

// ------------------------------------------------------------------ SE(3) helpers

__device__ void compose(const double* A, const double* B, double* C) {   // C = A B, internal layout
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
    C[9 + i] = A[3 * i] * B[9] + A[3 * i + 1] * B[10] + A[3 * i + 2] * B[11] + A[9 + i];
  }
}

__device__ void inverse(const double* A, double* B) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B[3 * i + j] = A[3 * j + i];
  for (int i = 0; i < 3; ++i) B[9 + i] = -(B[3 * i] * A[9] + B[3 * i + 1] * A[10] + B[3 * i + 2] * A[11]);
}

__device__ __forceinline__ void hat(const double* v, double* H) {
  H[0] = 0.0, H[1] = -v[2], H[2] = v[1];
  H[3] = v[2], H[4] = 0.0, H[5] = -v[0];
  H[6] = -v[1], H[7] = v[0], H[8] = 0.0;
}

__device__ __forceinline__ void mm3(const double* A, const double* B, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

// Coefficients of the SO(3) / SE(3) series at angle t (t2 = t^2):
// B = (1 - cos t)/t^2, C = (t - sin t)/t^3, Dq = (t^2 + 2 cos t - 2)/(2 t^4),
// Eq = (2 t - 3 sin t + t cos t)/(2 t^5), from Taylor series below t = 0.1.
__device__ void series(double t2, double& A, double& B, double& C, double& Dq, double& Eq) {
  if (t2 < 0.01) {
    A = 1.0 + t2 * (-1.0 / 6 + t2 * (1.0 / 120 + t2 * (-1.0 / 5040 + t2 * (1.0 / 362880))));
    B = 0.5 + t2 * (-1.0 / 24 + t2 * (1.0 / 720 + t2 * (-1.0 / 40320 + t2 * (1.0 / 3628800))));
    C = 1.0 / 6 + t2 * (-1.0 / 120 + t2 * (1.0 / 5040 + t2 * (-1.0 / 362880 + t2 * (1.0 / 39916800))));
    // Dq = sum_{k>=0} (-1)^k t^(2k) / (2k+4)!,  Eq = sum_{k>=0} (-1)^k (k+1) t^(2k) / (2k+5)!
    Dq = 1.0 / 24 + t2 * (-1.0 / 720 + t2 * (1.0 / 40320 + t2 * (-1.0 / 3628800 + t2 * (1.0 / 479001600))));
    Eq = 1.0 / 120 + t2 * (-1.0 / 2520 + t2 * (1.0 / 120960 + t2 * (-1.0 / 9979200 + t2 * (1.0 / 1245404160))));
  } else {
    const double t = sqrt(t2);
    double s, c;
    sincos(t, &s, &c);
    A = s / t;
    B = (1.0 - c) / t2;
    C = (t - s) / (t2 * t);
    Dq = (t2 + 2.0 * c - 2.0) / (2.0 * t2 * t2);
    Eq = (2.0 * t - 3.0 * s + t * c) / (2.0 * t2 * t2 * t);
  }
}

// xi = Log(T): phi from R (series below 1e-4, the largest-diagonal axis near pi), rho = V^-1 t.
__device__ void se3_log(const double* T, double* xi) {
  const double* R = T;
  const double c = fmin(1.0, fmax(-1.0, 0.5 * (R[0] + R[4] + R[8] - 1.0)));
  const double w[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
  const double th = acos(c);
  double phi[3];
  if (th < 1e-4) {
    const double k = 0.5 * (1.0 + th * th / 6.0);
    for (int i = 0; i < 3; ++i) phi[i] = k * w[i];
  } else if (CUDART_PI - th < 1e-6) {
    int k = 0;
    for (int i = 1; i < 3; ++i)
      if (R[4 * i] > R[4 * k]) k = i;
    double ax[3], nrm = 0.0;
    for (int i = 0; i < 3; ++i) ax[i] = 0.5 * (R[3 * i + k] + (i == k ? 1.0 : 0.0));
    for (int i = 0; i < 3; ++i) nrm += ax[i] * ax[i];
    nrm = sqrt(nrm);
    const double sgn = (ax[0] * w[0] + ax[1] * w[1] + ax[2] * w[2]) < 0 ? -1.0 : 1.0;
    for (int i = 0; i < 3; ++i) phi[i] = sgn * th * ax[i] / nrm;
  } else {
    const double k = th / (2.0 * sin(th));
    for (int i = 0; i < 3; ++i) phi[i] = k * w[i];
  }
  // V^-1 = I - 1/2 [phi]x + (1/t^2)(1 - A / (2 B)) [phi]x^2
  const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  double A, B, C, Dq, Eq;
  series(t2, A, B, C, Dq, Eq);
  const double k2 = t2 < 0.01 ? (1.0 / 12 + t2 * (1.0 / 720 + t2 * (1.0 / 30240 + t2 / 1209600.0)))
                              : (1.0 - A / (2.0 * B)) / t2;
  double P[9], P2[9];
  hat(phi, P);
  mm3(P, P, P2);
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) {
      const double vij = (i == j ? 1.0 : 0.0) - 0.5 * P[3 * i + j] + k2 * P2[3 * i + j];
      s += vij * T[9 + j];
    }
    xi[i] = s;
  }
  for (int i = 0; i < 3; ++i) xi[3 + i] = phi[i];
}

// J_r(xi)^-1 = J_l(-xi)^-1 = [[Ji, -Ji Q Ji], [0, Ji]] with J, Q of -xi (Barfoot's closed form).
__device__ void right_jacobian_inverse(const double* xi, double* Jinv /* 36, row-major */) {
  double rho[3] = {-xi[0], -xi[1], -xi[2]}, phi[3] = {-xi[3], -xi[4], -xi[5]};
  const double t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  double A, B, C, Dq, Eq;
  series(t2, A, B, C, Dq, Eq);
  double P[9], R[9], PP[9], PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  hat(phi, P);
  hat(rho, R);
  mm3(P, P, PP);
  mm3(P, R, PR);
  mm3(R, P, RP);
  mm3(PR, P, PRP);
  mm3(PP, R, PPR);
  mm3(RP, P, RPP);
  mm3(PRP, P, PRPP);
  mm3(PP, RP, PPRP);
  double Q[9];
  for (int k = 0; k < 9; ++k)
    Q[k] = 0.5 * R[k] + C * (PR[k] + RP[k] + PRP[k]) + Dq * (PPR[k] + RPP[k] - 3.0 * PRP[k]) + Eq * (PRPP[k] + PPRP[k]);
  // SO(3) J_l^-1(phi) = I - 1/2 [phi]x + (1/t^2)(1 - A/(2B)) [phi]x^2
  const double k2 = t2 < 0.01 ? (1.0 / 12 + t2 * (1.0 / 720 + t2 * (1.0 / 30240 + t2 / 1209600.0)))
                              : (1.0 - A / (2.0 * B)) / t2;
  double Ji[9];
  for (int k = 0; k < 9; ++k) Ji[k] = (k % 4 == 0 ? 1.0 : 0.0) - 0.5 * P[k] + k2 * PP[k];
  double T1[9], T2[9];
  mm3(Ji, Q, T1);
  mm3(T1, Ji, T2);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
      if (i < 3 && j < 3) v = Ji[3 * i + j];
      else if (i < 3) v = -T2[3 * i + j - 3];
      else if (j >= 3) v = Ji[3 * (i - 3) + j - 3];
      Jinv[6 * i + j] = v;
    }
}

// Ad(T) = [[R, [t]x R], [0, R]]
__device__ void adjoint(const double* T, double* Ad) {
  double H[9], HR[9];
  hat(T + 9, H);
  mm3(H, T, HR);
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      double v = 0.0;
      if (i < 3 && j < 3) v = T[3 * i + j];
      else if (i < 3) v = HR[3 * i + j - 3];
      else if (j >= 3) v = T[3 * (i - 3) + j - 3];
      Ad[6 * i + j] = v;
    }
}

__device__ void load_delta(const double* d, double* D) {   // [R | t] rows -> internal
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) D[3 * r + k] = d[4 * r + k];
    D[9 + r] = d[4 * r + 3];
  }
}

__device__ double edge_residual(const Pgo& p, const double* P, int e, double* r) {
  const int i = p.edges[2 * e], j = p.edges[2 * e + 1];
  double D[12], Dinv[12], Tiinv[12], A[12], E[12];
  load_delta(p.deltas + 12 * (size_t)e, D);
  inverse(D, Dinv);
  inverse(P + 12 * i, Tiinv);
  compose(Tiinv, P + 12 * j, A);
  compose(Dinv, A, E);
  se3_log(E, r);
  double s = 0.0;
  for (int k = 0; k < 6; ++k) s += r[k] * r[k];
  return 0.5 * s;
}

// Left update T1 = Exp(xi) T0 (coefficients as in series()).
__device__ void pose_plus(const double* T0, const double* xi, double* T1) {
  const double t2 = xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5];
  double A, B, C, Dq, Eq;
  series(t2, A, B, C, Dq, Eq);
  double P[9], PP[9];
  hat(xi + 3, P);
  mm3(P, P, PP);
  double Re[12];
  for (int k = 0; k < 9; ++k) Re[k] = (k % 4 == 0 ? 1.0 : 0.0) + A * P[k] + B * PP[k];
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += ((i == j ? 1.0 : 0.0) + B * P[3 * i + j] + C * PP[3 * i + j]) * xi[j];
    Re[9 + i] = s;
  }
  compose(Re, T0, T1);
}

// ------------------------------------------------------------------------ kernels

__global__ void k_pgo_init(Pgo p, const double* user, double lam0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < p.K)
    for (int r = 0; r < 3; ++r) {
      for (int q = 0; q < 3; ++q) p.pose[0][12 * k + 3 * r + q] = user[12 * (size_t)k + 4 * r + q];
      p.pose[0][12 * k + 9 + r] = user[12 * (size_t)k + 4 * r + 3];
    }
  if (k == 0) {
    PgoCtrl* c = p.ctrl;
    c->cur = 0, c->need_lin = 1, c->nonpd = 0, c->it = 0;
    c->lam = lam0, c->nu = 2.0, c->F = 0.0, c->pred = 0.0, c->step2 = 0.0;
  }
}

__global__ void k_pgo_edges(Pgo p) {
  if (!p.ctrl->need_lin) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.E) return;
  const double* P = p.pose[p.ctrl->cur];
  double r[6];
  p.ecost[e] = edge_residual(p, P, e, r);
  double Jri[36], Tjinv[12], Ad[36];
  right_jacobian_inverse(r, Jri);
  inverse(P + 12 * p.edges[2 * e + 1], Tjinv);
  adjoint(Tjinv, Ad);
  double* J = p.eJ + 72 * (size_t)e;
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      double s = 0.0;
      for (int k = 0; k < 6; ++k) s += Jri[6 * a + k] * Ad[6 * k + b];
      J[36 + 6 * a + b] = s;       // J_j
      J[6 * a + b] = -s;           // J_i
    }
  for (int k = 0; k < 6; ++k) p.er[6 * (size_t)e + k] = r[k];
}

// Block (a, b) of H: blockIdx.x < nfree: diagonal block of free pose blockIdx.x (and its
// gradient); otherwise off-diagonal pair blockIdx.x - nfree.  36 threads, one entry each.
__global__ void k_pgo_assemble(Pgo p) {
  if (!p.ctrl->need_lin) return;
  const int t = threadIdx.x;
  const int r = t / 6, c = t % 6;
  if (blockIdx.x < p.nfree) {
    const int a = blockIdx.x;
    if (t < 36) {
      double s = 0.0;
      for (int q = p.d_off[a]; q < p.d_off[a + 1]; ++q) {
        const int e = p.d_list[q] >> 1, side = p.d_list[q] & 1;
        const double* J = p.eJ + 72 * (size_t)e + 36 * side;
        for (int k = 0; k < 6; ++k) s += J[6 * k + r] * J[6 * k + c];
      }
      p.Hd[36 * (size_t)a + t] = s;
    } else if (t < 42) {
      const int rr = t - 36;
      double s = 0.0;
      for (int q = p.d_off[a]; q < p.d_off[a + 1]; ++q) {
        const int e = p.d_list[q] >> 1, side = p.d_list[q] & 1;
        const double* J = p.eJ + 72 * (size_t)e + 36 * side;
        for (int k = 0; k < 6; ++k) s += J[6 * k + rr] * p.er[6 * (size_t)e + k];
      }
      p.g[6 * a + rr] = s;
    }
  } else if (t < 36) {
    const int q0 = blockIdx.x - p.nfree;
    double s = 0.0;
    for (int q = p.p_off[q0]; q < p.p_off[q0 + 1]; ++q) {
      const int e = p.p_list[q] >> 1, a_is_j = p.p_list[q] & 1;
      const double* Ja = p.eJ + 72 * (size_t)e + 36 * a_is_j;
      const double* Jb = p.eJ + 72 * (size_t)e + 36 * (1 - a_is_j);
      for (int k = 0; k < 6; ++k) s += Ja[6 * k + r] * Jb[6 * k + c];
    }
    p.Ho[36 * (size_t)q0 + t] = s;
  }
}

// Dense lower triangle of A = H + lambda D; padding rows and columns hold the identity.
__global__ void k_pgo_load(Pgo p) {
  const double lam = p.ctrl->lam;
  const size_t total = (size_t)p.npw * p.npw;
  // Marquardt diagonal from the diagonal blocks, floored at 1e-12 of its maximum
  __shared__ double s_max[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < p.n; i += blockDim.x) m = fmax(m, p.Hd[36 * (i / 6) + 7 * (i % 6)]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, s_max[w]);
  const double floor_ = 1e-12 * m;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / p.npw), j = (int)(e % p.npw);
    double v = 0.0;
    if (j <= i) {
      if (i >= p.n) {
        v = i == j ? 1.0 : 0.0;
      } else if (i / 6 == j / 6) {
        v = p.Hd[36 * (i / 6) + 6 * (i % 6) + j % 6];
        if (i == j) {
          const double d = fmax(v, floor_);
          v += lam * d;
          p.D[i] = d;
        }
      }
    }
    p.Lw[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->nonpd = 0;
}

// Off-diagonal blocks into the loaded matrix (after k_pgo_load): pair q at rows of a, columns of b.
__global__ void k_pgo_load_pairs(Pgo p) {
  const int q = blockIdx.x, t = threadIdx.x;
  if (t >= 36) return;
  const int a = p.p_ab[2 * q], b = p.p_ab[2 * q + 1];
  p.Lw[(size_t)(6 * a + t / 6) * p.npw + 6 * b + t % 6] = p.Ho[36 * (size_t)q + t];
}

__global__ void __launch_bounds__(256) k_pgo_potrf(Pgo p, int pan) {
  __shared__ double A[kPW * kPD];
  __shared__ int s_bad;
  if (p.ctrl->nonpd) return;
  const int o = pan * kPW, tid = threadIdx.x;
  for (int e = tid; e < kPW * kPW; e += blockDim.x) {
    const int i = e / kPW, j = e % kPW;
    A[i * kPD + j] = j <= i ? p.Lw[(size_t)(o + i) * p.npw + o + j] : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < kPW; ++j) {
    const double d = A[j * kPD + j];
    const bool ok = d > 0.0 && isfinite(d);
    const double l = ok ? sqrt(d) : 1.0;
    __syncthreads();
    if (tid == 0) {
      if (!ok) s_bad = 1;
      A[j * kPD + j] = l;
    }
    if (tid > j && tid < kPW) A[tid * kPD + j] /= l;
    __syncthreads();
    // trailing update of the block: A_ik -= L_ij L_kj for j < k <= i
    const int R = kPW - j - 1;
    for (int e = tid; e < R * R; e += blockDim.x) {
      const int i = j + 1 + e / R, k = j + 1 + e % R;
      if (k <= i) A[i * kPD + k] -= A[i * kPD + j] * A[k * kPD + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < kPW * kPW; e += blockDim.x) {
    const int i = e / kPW, j = e % kPW;
    if (j <= i) p.Lw[(size_t)(o + i) * p.npw + o + j] = A[i * kPD + j];
  }
  if (tid == 0 && s_bad) p.ctrl->nonpd = 1;
}

// One warp per row below the panel: L_ip = A_ip L_pp^-T.
__global__ void __launch_bounds__(256) k_pgo_trsm(Pgo p, int pan) {
  __shared__ double Lp[kPW * kPD];
  if (p.ctrl->nonpd) return;
  const int o = pan * kPW, tid = threadIdx.x;
  for (int e = tid; e < kPW * kPW; e += blockDim.x) {
    const int i = e / kPW, j = e % kPW;
    Lp[i * kPD + j] = j <= i ? p.Lw[(size_t)(o + i) * p.npw + o + j] : 0.0;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int row = o + kPW + blockIdx.x * 8 + warp;
  if (row >= p.npw) return;
  double* a = p.Lw + (size_t)row * p.npw + o;
  double u = a[lane];
  for (int m = 0; m < kPW; ++m) {
    const double x = __shfl_sync(0xffffffffu, u, m) / Lp[m * kPD + m];
    if (lane == m) u = x;
    if (lane > m) u -= x * Lp[lane * kPD + m];
  }
  a[lane] = u;
}

// Trailing update after panel pan: 16 x 16 tile (ti, tj), ti >= tj, below the panel.
__global__ void __launch_bounds__(256) k_pgo_syrk(Pgo p, int pan) {
  __shared__ double sa[16 * kPD], sb[16 * kPD];
  if (p.ctrl->nonpd) return;
  const int o = pan * kPW, o2 = o + kPW, tid = threadIdx.x;
  int t = (int)((sqrtf(8.0f * (float)blockIdx.x + 1.0f) - 1.0f) * 0.5f);
  while (t * (t + 1) / 2 > (int)blockIdx.x) --t;
  while ((t + 1) * (t + 2) / 2 <= (int)blockIdx.x) ++t;
  const int ti = t, tj = blockIdx.x - t * (t + 1) / 2;
  for (int e = tid; e < 16 * kPW; e += blockDim.x) {
    const int r = e / kPW, m = e % kPW;
    sa[r * kPD + m] = p.Lw[(size_t)(o2 + 16 * ti + r) * p.npw + o + m];
    sb[r * kPD + m] = p.Lw[(size_t)(o2 + 16 * tj + r) * p.npw + o + m];
  }
  __syncthreads();
  const int r = tid / 16, c = tid % 16;
  const int gi = o2 + 16 * ti + r, gj = o2 + 16 * tj + c;
  if (gj > gi) return;
  double acc = 0.0;
  for (int m = 0; m < kPW; ++m) acc += sa[r * kPD + m] * sb[c * kPD + m];
  p.Lw[(size_t)gi * p.npw + gj] -= acc;
}

// L y = -g, then L^T delta = y; predicted reduction and step norm.  One CTA of 1024.
__global__ void __launch_bounds__(1024) k_pgo_solve(Pgo p) {
  if (p.ctrl->nonpd) return;
  const int tid = threadIdx.x, npw = p.npw, lane = tid & 31;
  double* x = p.x;
  for (int i = tid; i < npw; i += blockDim.x) x[i] = i < p.n ? -p.g[i] : 0.0;
  __syncthreads();
  const int npan = npw / kPW;
  __shared__ double s_part[1024];
  for (int pan = 0; pan < npan; ++pan) {
    const int o = pan * kPW, end = p.pend[pan];
    if (tid < 32) {
      double v = x[o + lane];
      for (int m = 0; m < kPW; ++m) {
        const double xm = __shfl_sync(0xffffffffu, v, m) / p.Lw[(size_t)(o + m) * npw + o + m];
        if (lane == m) v = xm;
        if (lane > m) v -= xm * p.Lw[(size_t)(o + lane) * npw + o + m];
      }
      x[o + lane] = v;
    }
    __syncthreads();
    for (int i = o + kPW + tid; i < end; i += blockDim.x) {   // rows of the panel's envelope
      double s = 0.0;
      for (int m = 0; m < kPW; ++m) s += p.Lw[(size_t)i * npw + o + m] * x[o + m];
      x[i] -= s;
    }
    __syncthreads();
  }
  for (int pan = npan - 1; pan >= 0; --pan) {
    const int o = pan * kPW, end = p.pend[pan];
    // x_p -= L_{below, p}^T x_below over the panel's envelope: thread (g, c) sums column c over
    // the rows o + 32 + g + 32 k (a warp reads whole row segments), then the 32 partials of
    // each column are added in order g = 0..31
    {
      const int c = tid & 31, g = tid >> 5;
      double s = 0.0;
      for (int i = o + kPW + g; i < end; i += 32) s += p.Lw[(size_t)i * npw + o + c] * x[i];
      s_part[g * 32 + c] = s;
    }
    __syncthreads();
    if (tid < kPW) {
      double s = 0.0;
      for (int g = 0; g < 32; ++g) s += s_part[g * 32 + tid];
      x[o + tid] -= s;
    }
    __syncthreads();
    if (tid < 32) {
      double v = x[o + lane];
      for (int m = kPW - 1; m >= 0; --m) {
        const double xm = __shfl_sync(0xffffffffu, v, m) / p.Lw[(size_t)(o + m) * npw + o + m];
        if (lane == m) v = xm;
        if (lane < m) v -= xm * p.Lw[(size_t)(o + m) * npw + o + lane];
      }
      x[o + lane] = v;
    }
    __syncthreads();
  }
  // L = 1/2 delta^T (lam D delta - g), |delta|^2: fixed-order block sums
  __shared__ double s1[32], s2[32];
  double a = 0.0, b = 0.0;
  const double lam = p.ctrl->lam;
  for (int i = tid; i < p.n; i += blockDim.x) {
    a += x[i] * (lam * p.D[i] * x[i] - p.g[i]);
    b += x[i] * x[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if (lane == 0) s1[tid >> 5] = a, s2[tid >> 5] = b;
  __syncthreads();
  if (tid == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sa += s1[w], sb += s2[w];
    p.ctrl->pred = 0.5 * sa;
    p.ctrl->step2 = sb;
    bool fin = isfinite(sa) && isfinite(sb);
    if (!fin) p.ctrl->nonpd = 1;
  }
}

__global__ void k_pgo_candidate(Pgo p) {
  if (p.ctrl->nonpd) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.K) return;
  const int cur = p.ctrl->cur;
  const double* T0 = p.pose[cur] + 12 * k;
  double* T1 = p.pose[cur ^ 1] + 12 * k;
  if (p.col[k] < 0) {
    for (int q = 0; q < 12; ++q) T1[q] = T0[q];
  } else {
    pose_plus(T0, p.x + p.col[k], T1);
  }
}

__global__ void k_pgo_cost(Pgo p) {
  if (p.ctrl->nonpd) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.E) return;
  double r[6];
  p.ccost[e] = edge_residual(p, p.pose[p.ctrl->cur ^ 1], e, r);
}

__device__ double block_sum_ordered(const double* v, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(256) k_pgo_decide(Pgo p) {
  __shared__ double red[8];
  PgoCtrl* c = p.ctrl;
  const bool relin = c->need_lin;
  const double F0 = relin ? block_sum_ordered(p.ecost, p.E, red) : c->F;
  const bool nonpd = c->nonpd;
  const double F1 = nonpd ? CUDART_NAN : block_sum_ordered(p.ccost, p.E, red);
  if (threadIdx.x != 0) return;
  c->F = F0;
  const double L = nonpd ? CUDART_NAN : c->pred;
  const double gain = nonpd ? CUDART_NAN : (L != 0.0 ? (F0 - F1) / L : CUDART_NAN);
  const bool acc = !nonpd && L > 0.0 && isfinite(F1) && gain > 0.0;
  if (p.trace) {
    cvba_lm_record* r = p.trace + c->it;
    r->cost0 = F0;
    r->cost1 = F1;
    r->lambda = c->lam;
    r->gain = gain;
    r->pred = L;
    r->step_norm = nonpd ? CUDART_NAN : sqrt(c->step2);
    r->rms_px = sqrt(2.0 * F0 / fmax(1.0, (double)p.E));
    r->accepted = acc ? 1 : 0;
    r->nonpd = nonpd ? 1 : 0;
    r->n_valid = p.E;
    r->n_inlier = p.E;
    r->n_bad_index = 0;
    r->reserved = 0;
  }
  if (acc) {
    c->lam *= fmax(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) * (2.0 * gain - 1.0) * (2.0 * gain - 1.0));
    c->nu = 2.0;
    c->cur ^= 1;
  } else {
    c->lam *= c->nu;
    c->nu *= 2.0;
  }
  c->need_lin = acc ? 1 : 0;
  c->nonpd = 0;
  c->it++;
}

__global__ void k_pgo_store(Pgo p, double* user) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p.K) return;
  const double* T = p.pose[p.ctrl->cur] + 12 * k;
  for (int r = 0; r < 3; ++r) {
    for (int q = 0; q < 3; ++q) user[12 * (size_t)k + 4 * r + q] = T[3 * r + q];
    user[12 * (size_t)k + 4 * r + 3] = T[9 + r];
  }
}

// ------------------------------------------------------------------ host side

struct Layout {
  size_t ctrl, pose0, pose1, er, eJ, ecost, ccost, Hd, Ho, g, D, Lw, x, col, d_off, d_list, p_ab, p_off, p_list, pend,
      total;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

Layout plan(int K, int E, int n_pair) {
  const int nfree = K - 1, n = 6 * nfree, npw = (n + kPW - 1) / kPW * kPW;
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.ctrl = take(sizeof(PgoCtrl));
  L.pose0 = take(sizeof(double) * 12 * K);
  L.pose1 = take(sizeof(double) * 12 * K);
  L.er = take(sizeof(double) * 6 * (size_t)E);
  L.eJ = take(sizeof(double) * 72 * (size_t)E);
  L.ecost = take(sizeof(double) * (size_t)E);
  L.ccost = take(sizeof(double) * (size_t)E);
  L.Hd = take(sizeof(double) * 36 * (size_t)nfree);
  L.Ho = take(sizeof(double) * 36 * (size_t)std::max(n_pair, 1));
  L.g = take(sizeof(double) * (size_t)n);
  L.D = take(sizeof(double) * (size_t)npw);
  L.Lw = take(sizeof(double) * (size_t)npw * npw);
  L.x = take(sizeof(double) * (size_t)npw);
  L.col = take(sizeof(int32_t) * K);
  L.d_off = take(sizeof(int32_t) * (size_t)(nfree + 1));
  L.d_list = take(sizeof(int32_t) * 2 * (size_t)E);
  L.p_ab = take(sizeof(int32_t) * 2 * (size_t)std::max(n_pair, 1));
  L.p_off = take(sizeof(int32_t) * (size_t)(n_pair + 1));
  L.p_list = take(sizeof(int32_t) * (size_t)std::max(E, 1));
  L.pend = take(sizeof(int32_t) * (size_t)(npw / kPW));
  L.total = o;
  return L;
}

}  // namespace

extern "C" size_t cvba_pgo_workspace_bytes(int n_poses, int n_edges) {
  if (n_poses < 2 || n_edges < 0) return 0;
  // the off-diagonal pairs are at most the edges
  return plan(n_poses, n_edges, n_edges).total;
}

extern "C" cvba_status cvba_pgo_solve(int n_poses, int n_edges, const int32_t* edges, const double* deltas,
                                      double* poses, int fixed, const cvba_opts* opts, cvba_lm_record* trace,
                                      void* work, size_t work_bytes, void* stream) {
  const int K = n_poses, E = n_edges;
  if (K < 2 || E < 1 || fixed < 0 || fixed >= K || !edges || !deltas || !poses || !opts || !work)
    return CVBA_ERR_INVALID_ARG;
  if (opts->iters < 0 || !(opts->lambda0 > 0.0) || !std::isfinite(opts->lambda0)) return CVBA_ERR_INVALID_ARG;
  if (work_bytes < cvba_pgo_workspace_bytes(K, E)) return CVBA_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return CVBA_ERR_INVALID_ARG;
  if (cudaPeekAtLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the graph's structure: read back, checked, and turned into the block contribution lists
  std::vector<int32_t> ed(2 * (size_t)E);
  if (cudaMemcpyAsync(ed.data(), edges, ed.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  std::vector<int32_t> col(K);
  for (int k = 0, c = 0; k < K; ++k) col[k] = k == fixed ? -1 : 6 * c++;
  std::vector<int> seen(K, 0);
  for (int e = 0; e < E; ++e) {
    const int i = ed[2 * e], j = ed[2 * e + 1];
    if (i < 0 || i >= K || j < 0 || j >= K || i == j) return CVBA_ERR_INDEX;
    seen[i] = seen[j] = 1;
  }
  for (int k = 0; k < K; ++k)
    if (k != fixed && !seen[k]) return CVBA_ERR_INVALID_ARG;        // a free pose with no edge
  const int nfree = K - 1;
  std::vector<int32_t> d_off(nfree + 1, 0), d_list;
  {
    std::vector<std::vector<int32_t>> per(nfree);
    for (int e = 0; e < E; ++e)
      for (int side = 0; side < 2; ++side) {
        const int k = ed[2 * e + side];
        if (col[k] >= 0) per[col[k] / 6].push_back(2 * e + side);
      }
    for (int a = 0; a < nfree; ++a) {
      d_off[a + 1] = d_off[a] + (int32_t)per[a].size();
      d_list.insert(d_list.end(), per[a].begin(), per[a].end());
    }
  }
  std::vector<int32_t> p_ab, p_off(1, 0), p_list;
  {
    std::map<std::pair<int, int>, std::vector<int32_t>> pairs;   // (a, b) by column, a > b
    for (int e = 0; e < E; ++e) {
      const int i = ed[2 * e], j = ed[2 * e + 1];
      if (col[i] < 0 || col[j] < 0) continue;
      const int bi = col[i] / 6, bj = col[j] / 6;
      const int a = std::max(bi, bj), b = std::min(bi, bj);
      pairs[{a, b}].push_back(2 * e + (a == bj ? 1 : 0));
    }
    for (auto& kv : pairs) {
      p_ab.push_back(kv.first.first);
      p_ab.push_back(kv.first.second);
      p_list.insert(p_list.end(), kv.second.begin(), kv.second.end());
      p_off.push_back((int32_t)p_list.size());
    }
  }
  const int n_pair = (int)p_off.size() - 1;
  // envelope of the factor by 32-column panel: the first column of each row is that of its
  // pose's first coupled pose (the Cholesky fill stays inside this profile), so the rows below
  // panel p with nonzeros in its columns end at the last row whose first column is in or
  // before the panel
  const int n_c = 6 * nfree, npw_h = (n_c + kPW - 1) / kPW * kPW, npan_h = npw_h / kPW;
  std::vector<int32_t> pend(npan_h);
  {
    std::vector<int> first(nfree);
    for (int a = 0; a < nfree; ++a) first[a] = a;
    for (int q = 0; q < n_pair; ++q) first[p_ab[2 * q]] = std::min(first[p_ab[2 * q]], p_ab[2 * q + 1]);
    for (int pn = 0; pn < npan_h; ++pn) {
      const int end_col = kPW * pn + kPW - 1;
      int last = kPW * (pn + 1) - 1;
      for (int r = kPW * (pn + 1); r < n_c; ++r)
        if (6 * first[r / 6] <= end_col) last = r;
      pend[pn] = std::min(npw_h, (last + 1 + kPW - 1) / kPW * kPW);
    }
  }
  const Layout L = plan(K, E, n_pair);
  unsigned char* w = static_cast<unsigned char*>(work);
  Pgo p{};
  p.K = K, p.E = E, p.nfree = nfree, p.n = 6 * nfree, p.npw = (p.n + kPW - 1) / kPW * kPW, p.fixed = fixed;
  p.iters = opts->iters, p.n_pair = n_pair;
  p.edges = edges, p.deltas = deltas;
  p.pose[0] = reinterpret_cast<double*>(w + L.pose0);
  p.pose[1] = reinterpret_cast<double*>(w + L.pose1);
  p.er = reinterpret_cast<double*>(w + L.er);
  p.eJ = reinterpret_cast<double*>(w + L.eJ);
  p.ecost = reinterpret_cast<double*>(w + L.ecost);
  p.ccost = reinterpret_cast<double*>(w + L.ccost);
  p.Hd = reinterpret_cast<double*>(w + L.Hd);
  p.Ho = reinterpret_cast<double*>(w + L.Ho);
  p.g = reinterpret_cast<double*>(w + L.g);
  p.D = reinterpret_cast<double*>(w + L.D);
  p.Lw = reinterpret_cast<double*>(w + L.Lw);
  p.x = reinterpret_cast<double*>(w + L.x);
  p.col = reinterpret_cast<const int32_t*>(w + L.col);
  p.d_off = reinterpret_cast<const int32_t*>(w + L.d_off);
  p.d_list = reinterpret_cast<const int32_t*>(w + L.d_list);
  p.p_ab = reinterpret_cast<const int32_t*>(w + L.p_ab);
  p.p_off = reinterpret_cast<const int32_t*>(w + L.p_off);
  p.p_list = reinterpret_cast<const int32_t*>(w + L.p_list);
  p.pend = reinterpret_cast<const int32_t*>(w + L.pend);
  p.ctrl = reinterpret_cast<PgoCtrl*>(w + L.ctrl);
  p.trace = trace;
  auto up = [&](size_t off, const std::vector<int32_t>& v) {
    return v.empty() ? cudaSuccess
                     : cudaMemcpyAsync(w + off, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  };
  cudaError_t e = up(L.col, col);
  if (e == cudaSuccess) e = up(L.d_off, d_off);
  if (e == cudaSuccess) e = up(L.d_list, d_list);
  if (e == cudaSuccess) e = up(L.p_ab, p_ab);
  if (e == cudaSuccess) e = up(L.p_off, p_off);
  if (e == cudaSuccess) e = up(L.p_list, p_list);
  if (e == cudaSuccess) e = up(L.pend, pend);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);     // the host lists go out of scope
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  const int tb = 128;
  k_pgo_init<<<(K + tb - 1) / tb, tb, 0, s>>>(p, poses, opts->lambda0);
  const int npan = p.npw / kPW;
  const unsigned n_load = (unsigned)std::min<size_t>(((size_t)p.npw * p.npw + 255) / 256, 152 * 8);
  for (int it = 0; it < opts->iters; ++it) {
    k_pgo_edges<<<(E + tb - 1) / tb, tb, 0, s>>>(p);
    k_pgo_assemble<<<nfree + n_pair, 64, 0, s>>>(p);
    k_pgo_load<<<n_load, 256, 0, s>>>(p);
    if (n_pair > 0) k_pgo_load_pairs<<<n_pair, 64, 0, s>>>(p);
    for (int pan = 0; pan < npan; ++pan) {
      k_pgo_potrf<<<1, 256, 0, s>>>(p, pan);
      const int below = pend[pan] - kPW * (pan + 1);   // rows of the panel's envelope
      if (below == 0) continue;
      k_pgo_trsm<<<below / 8, 256, 0, s>>>(p, pan);
      const int nt = below / 16;
      k_pgo_syrk<<<nt * (nt + 1) / 2, 256, 0, s>>>(p, pan);
    }
    k_pgo_solve<<<1, 1024, 0, s>>>(p);
    k_pgo_candidate<<<(K + tb - 1) / tb, tb, 0, s>>>(p);
    k_pgo_cost<<<(E + tb - 1) / tb, tb, 0, s>>>(p);
    k_pgo_decide<<<1, 256, 0, s>>>(p);
  }
  k_pgo_store<<<(K + tb - 1) / tb, tb, 0, s>>>(p, poses);
  if (cudaGetLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  return CVBA_OK;
}
