// cvba_evaluate_noalloc: the robust reprojection cost of a window, computed from plain
// device arrays without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are running, for
// example a robot's tracking thread whose GPU memory budget is fixed at start-up (an
// allocation can block on the device, can fail under memory pressure from other
// processes, and is forbidden after initialisation in some real-time or certified
// software), or a host program whose GPU memory is entirely owned by another allocator.
// They cannot create a cvba_ctx (which allocates its layout), so this entry point takes
// every input and output as a caller-owned device pointer and keeps its only scratch, the
// per-block partial sums, in a fixed file-scope device array.
//
// The scratch array is shared by every call in the process on a given GPU and keeps the
// last call's contents; each call overwrites the entries it reads, so nothing needs
// clearing between calls.  Calls whose kernels overlap on the GPU (different streams, or
// other threads) race on it: serialise them.  The array (640 KB) lives in this library's
// device module: with lazy module loading (the CUDA default) the module, and with it the
// array, is loaded onto a GPU by the first call there, which therefore may allocate; with
// CUDA_MODULE_LOADING=EAGER it is loaded with the context.  Either way it stays until the
// context is destroyed.  The array's device address is looked up on every call, so a
// module reloaded after a device reset is found at its new address.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/cvba.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 16384;
constexpr int kMaxObs = kMaxBlocks * kThreads;   // 4,194,304 observations per call
constexpr int kParts = 5;                        // cost, sum r^2, n_valid, n_inlier, n_bad_index

// Host code must not pass this name to a kernel: on the host it is only a stand-in, and
// kernels are given the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) double g_partials[kMaxBlocks * kParts];

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum of kParts values; result in thread 0.
__device__ void block_sum(double v[kParts], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < kParts; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
    for (int k = 0; k < kParts; ++k) red[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0)
    for (int k = 0; k < kParts; ++k) v[k] = warp_sum(lane < nw ? red[k * 32 + lane] : 0.0);
}

// One thread per observation: r = pi(T^cb_k T^bw_i p^w_j) - o (cuVSLAM Sec. 2.2, Eq. r^repr),
// Huber cost 1/2 rho(|r|^2) on valid observations (camera depth > z_min), with the same
// operation order as the library's evaluation kernel so results agree to rounding of the
// final sums.  Observations with an index out of range are skipped and counted.
__global__ void __launch_bounds__(kThreads) k_eval_obs(int n_obs, int n_kf, int n_cams, int n_lm,
                                                       const double* __restrict__ intr, const double* __restrict__ T_cb,
                                                       const double* __restrict__ T_bw, const double* __restrict__ p_w,
                                                       const int32_t* __restrict__ kf, const int32_t* __restrict__ cam,
                                                       const int32_t* __restrict__ lm, const double* __restrict__ uv,
                                                       double hub, double zmin, double* __restrict__ partials) {
  __shared__ double red[kParts * 32];
  double v[kParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < n_obs) {
    const int i = kf[n], c = cam[n], j = lm[n];
    if (i < 0 || i >= n_kf || c < 0 || c >= n_cams || j < 0 || j >= n_lm) {
      v[4] = 1.0;
    } else {
      const double* P = T_bw + 12 * i;   // [R | t] row-major
      const double px = p_w[3 * j], py = p_w[3 * j + 1], pz = p_w[3 * j + 2];
      double X[3];
      for (int r = 0; r < 3; ++r)
        X[r] = fma(P[4 * r], px, fma(P[4 * r + 1], py, fma(P[4 * r + 2], pz, P[4 * r + 3])));
      const double* Q = T_cb + 12 * c;
      const double xc = fma(Q[0], X[0], fma(Q[1], X[1], fma(Q[2], X[2], Q[3])));
      const double yc = fma(Q[4], X[0], fma(Q[5], X[1], fma(Q[6], X[2], Q[7])));
      const double zc = fma(Q[8], X[0], fma(Q[9], X[1], fma(Q[10], X[2], Q[11])));
      if (zc > zmin) {
        const double iz = 1.0 / zc;
        const double xn = xc * iz, yn = yc * iz;
        const double r0 = fma(intr[4 * c], xn, intr[4 * c + 2]) - uv[2 * n];
        const double r1 = fma(intr[4 * c + 1], yn, intr[4 * c + 3]) - uv[2 * n + 1];
        const double s = fma(r0, r0, r1 * r1);
        const double e = sqrt(s);
        const bool inl = e <= hub;
        v[0] = 0.5 * (inl ? s : fma(2.0 * hub, e, -hub * hub));
        v[1] = s;
        v[2] = 1.0;
        v[3] = inl ? 1.0 : 0.0;
      }
    }
  }
  block_sum(v, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < kParts; ++k) partials[blockIdx.x * kParts + k] = v[k];
}

// Fixed-order sum of the per-block partials into the caller's output.
__global__ void __launch_bounds__(kThreads) k_eval_obs_reduce(const double* __restrict__ partials, int n_blocks,
                                                              double* __restrict__ out) {
  __shared__ double red[kParts * 32];
  double v[kParts] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_blocks; b += blockDim.x)
    for (int k = 0; k < kParts; ++k) v[k] += partials[b * kParts + k];
  block_sum(v, red);
  if (threadIdx.x == 0)
    for (int k = 0; k < kParts; ++k) out[k] = v[k];
}

// Device address of the scratch array on the current device, looked up with that device
// current.  Not cached: after a device reset (or in another context on the same ordinal)
// the module is loaded again and the array can sit at a new address.  The lookup is cheap
// once the module is loaded and allocates nothing then.
cvba_status scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return CVBA_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return CVBA_OK;
}

}  // namespace

extern "C" cvba_status cvba_evaluate_noalloc(int n_obs, int n_kf, int n_cams, int n_lm, const double* intr,
                                             const double* T_cb, const double* T_bw, const double* p_w,
                                             const int32_t* kf, const int32_t* cam, const int32_t* lm,
                                             const double* uv, double huber_delta, double z_min, double* out,
                                             void* stream) {
  if (n_obs < 1 || n_obs > kMaxObs || n_kf < 1 || n_cams < 1 || n_lm < 1) return CVBA_ERR_INVALID_ARG;
  if (!intr || !T_cb || !T_bw || !p_w || !kf || !cam || !lm || !uv || !out) return CVBA_ERR_INVALID_ARG;
  if (!(huber_delta > 0.0) || !std::isfinite(huber_delta) || !std::isfinite(z_min)) return CVBA_ERR_INVALID_ARG;
  // An error left pending by the caller's own earlier work is not ours: launch nothing,
  // leave it pending for the caller, and report it.
  if (cudaPeekAtLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  double* partials = nullptr;
  const cvba_status st = scratch_address(&partials);
  if (st != CVBA_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_blocks = (n_obs + kThreads - 1) / kThreads;
  k_eval_obs<<<n_blocks, kThreads, 0, s>>>(n_obs, n_kf, n_cams, n_lm, intr, T_cb, T_bw, p_w, kf, cam, lm, uv,
                                           huber_delta, z_min, partials);
  if (cudaGetLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  k_eval_obs_reduce<<<1, kThreads, 0, s>>>(partials, n_blocks, out);
  if (cudaGetLastError() != cudaSuccess) return CVBA_ERR_CUDA;
  return CVBA_OK;
}
