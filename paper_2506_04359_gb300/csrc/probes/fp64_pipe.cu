// Standalone measurement program (not part of the library; the library build compiles only the
// files of the directory above): throughput and dependent latency of FP64 FMA against the FP64
// matrix multiply-accumulate mma.sync.m8n8k4.f64 on one GPU, to decide whether the FP64
// trailing updates of the reduced-system factorisation gain from the MMA form.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_pipe fp64_pipe.cu && ./fp64_pipe
// Every thread writes one double to out[] (sized to the grid), so nothing is read or written
// out of bounds; the loops have fixed trip counts.
#include <cstdio>
#include <cuda_runtime.h>

constexpr int ITER = 4096;

__global__ void k_dfma(double* out, double b, double c) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITER; ++i) {
    a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
    a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

__global__ void k_dfma_chain(double* out, double b, double c) {     // one dependent chain
  double a0 = threadIdx.x;
  for (int i = 0; i < ITER; ++i) a0 = fma(a0, b, c);
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0;
}

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
}

__global__ void k_dmma(double* out, double a, double b) {
  double c[8][2];
#pragma unroll
  for (int k = 0; k < 8; ++k) c[k][0] = c[k][1] = threadIdx.x + k;
  for (int i = 0; i < ITER / 8; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) dmma(c[k][0], c[k][1], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += c[k][0] + c[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dmma_chain(double* out, double a, double b) {
  double c0 = threadIdx.x, c1 = c0 + 1;
  for (int i = 0; i < ITER / 8; ++i) dmma(c0, c1, a, b);
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1;
}

template <typename F>
float time_ms(F f) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f();
  cudaDeviceSynchronize();
  cudaEventRecord(e0);
  for (int r = 0; r < 5; ++r) f();
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / 5;
}

int main() {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, 0);
  const int sms = prop.multiProcessorCount;
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  const int blocks = sms * 4, threads = 256;
  double* out;
  cudaMalloc(&out, sizeof(double) * blocks * threads);
  const double b = 0.999999, c = 1e-7;
  // throughput: FMAs = threads x ITER x 8 (DFMA); warps x (ITER/8) x 8 mma x 256 FMA (DMMA)
  const double n_dfma = (double)blocks * threads * ITER * 8;
  const double n_dmma = (double)blocks * (threads / 32) * (ITER / 8) * 8 * 256;
  float t1 = time_ms([&] { k_dfma<<<blocks, threads>>>(out, b, c); });
  float t2 = time_ms([&] { k_dmma<<<blocks, threads>>>(out, b, c); });
  // latency: one warp, one dependent chain
  float t3 = time_ms([&] { k_dfma_chain<<<1, 32>>>(out, b, c); });
  float t4 = time_ms([&] { k_dmma_chain<<<1, 32>>>(out, b, c); });
  cudaError_t err = cudaDeviceSynchronize();
  const double ghz = clk_khz * 1e-6;
  printf("device %s, %d SMs, clock %.3f GHz, status %s\n", prop.name, sms, ghz, cudaGetErrorString(err));
  printf("DFMA throughput: %.1f GFMA/s = %.3f TFLOP/s, %.2f FMA/clk/SM (%.3f ms)\n", n_dfma / t1 / 1e6,
         2 * n_dfma / t1 / 1e9, n_dfma / (t1 * 1e-3) / (sms * ghz * 1e9), t1);
  printf("DMMA throughput: %.1f GFMA/s = %.3f TFLOP/s, %.2f FMA/clk/SM (%.3f ms)\n", n_dmma / t2 / 1e6,
         2 * n_dmma / t2 / 1e9, n_dmma / (t2 * 1e-3) / (sms * ghz * 1e9), t2);
  printf("DFMA dependent latency: %.1f cycles per FMA (%.3f ms)\n", t3 * 1e-3 * ghz * 1e9 / ITER, t3);
  printf("DMMA dependent latency: %.1f cycles per mma (%.3f ms)\n", t4 * 1e-3 * ghz * 1e9 / (ITER / 8), t4);
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
