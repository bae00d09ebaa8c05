// Stand-in for the CUDA runtime and the library's kernel launchers, for CPU tests of the host
// layer (cvba_host.cpp): device memory is host memory (fresh buffers filled with 0xCD bytes),
// copies and fills are memcpy and memset, streams, events and graphs are tokens, and the
// launchers do nothing.  Pinned host memory is allocated at exactly the requested size, so an
// overrun shows up under AddressSanitizer.  Counters let a test see how often a graph was
// instantiated and how often an elapsed time was read; the elapsed times themselves can be
// scripted (g_elapsed_script, consumed in order, 0 when exhausted).
//
// Include after cvba_host.cpp, in exactly one translation unit of a test driver.
#pragma once
#include <cstdlib>
#include <cstring>
#include <vector>

int g_instantiate_count = 0;
int g_elapsed_calls = 0;
std::vector<float> g_elapsed_script;

namespace {
char g_token[64];  // streams, events and graphs are addresses inside this array
template <typename T>
T token(int i) {
  return reinterpret_cast<T>(g_token + i);
}
}  // namespace

extern "C" {
cudaError_t cudaMalloc(void** p, size_t n) {
  *p = std::malloc(n ? n : 1);
  if (!*p) return cudaErrorMemoryAllocation;
  std::memset(*p, 0xCD, n);
  return cudaSuccess;
}
cudaError_t cudaFree(void* p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMallocHost(void** p, size_t n) {
  *p = std::malloc(n ? n : 1);  // exact size: an overrun of the staging is a heap overflow
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFreeHost(void* p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMemcpy(void* dst, const void* src, size_t n, enum cudaMemcpyKind) {
  if (n) std::memcpy(dst, src, n);
  return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t n, enum cudaMemcpyKind, cudaStream_t) {
  if (n) std::memcpy(dst, src, n);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t) {
  if (n) std::memset(p, v, n);
  return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned int) {
  *s = token<cudaStream_t>(1);
  return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamBeginCapture(cudaStream_t, enum cudaStreamCaptureMode) { return cudaSuccess; }
cudaError_t cudaStreamEndCapture(cudaStream_t, cudaGraph_t* g) {
  *g = token<cudaGraph_t>(2);
  return cudaSuccess;
}
cudaError_t cudaGraphInstantiate(cudaGraphExec_t* e, cudaGraph_t, unsigned long long) {
  *e = token<cudaGraphExec_t>(3);
  ++g_instantiate_count;
  return cudaSuccess;
}
cudaError_t cudaGraphLaunch(cudaGraphExec_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t) { return cudaSuccess; }
cudaError_t cudaGraphDestroy(cudaGraph_t) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t* e) {
  *e = token<cudaEvent_t>(4);
  return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned int) {
  *e = token<cudaEvent_t>(5);
  return cudaSuccess;
}
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t) {
  *ms = g_elapsed_calls < (int)g_elapsed_script.size() ? g_elapsed_script[g_elapsed_calls] : 0.f;
  ++g_elapsed_calls;
  return cudaSuccess;
}
cudaError_t cudaGetDeviceCount(int* n) {
  *n = 1;
  return cudaSuccess;
}
cudaError_t cudaGetDevice(int* d) {
  *d = 0;
  return cudaSuccess;
}
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDeviceProperties(struct cudaDeviceProp* p, int) {
  std::memset(p, 0, sizeof(*p));
  std::strcpy(p->name, "host stand-in");
  p->major = 10;
  p->minor = 3;
  p->multiProcessorCount = 152;
  p->sharedMemPerBlockOptin = 232448;
  return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "host stand-in"; }
}

// ---------------------------------------------------------------- launchers: no work
namespace cvba {
void batch_plan_sizes(Dev*, int, BatchLaunch&) {}
cudaError_t enqueue_batch_init(const BatchLaunch&, double, double, double, int, int, int, cudaStream_t) {
  return cudaSuccess;
}
cudaError_t enqueue_batch_iteration(const BatchLaunch&, cudaStream_t) { return cudaSuccess; }
int batch_kernels_per_iteration(const BatchLaunch&) { return 0; }
int solve_kernels_per_iteration(const Dev&) { return 0; }
cudaError_t enqueue_solve_init(const Dev&, double, double, double, int, int, int, cudaStream_t) { return cudaSuccess; }
cudaError_t enqueue_iteration(const Dev&, cudaStream_t, cudaEvent_t*, const SideStream*) { return cudaSuccess; }
int profile_parts() { return 1; }
const char* profile_names() { return "none"; }
cudaError_t enqueue_state_io(const Dev&, int, double*, const int32_t*, cudaStream_t) { return cudaSuccess; }
int kernels_per_iteration() { return 0; }
int kernels_per_solve_init() { return 0; }
cudaError_t enqueue_evaluate(const Dev&, double, double, double*, cudaStream_t) { return cudaSuccess; }
cudaError_t set_kernel_attributes() { return cudaSuccess; }
}  // namespace cvba
