// aew_dot_noalloc: the FP64 inner product of aew_dot for callers that cannot allocate
// device memory.  Some callers run where cudaMalloc is not allowed or not wanted: inside
// an application that owns every device allocation through its own pool, a framework
// hook that must not change the device memory footprint while it runs, or code that
// must not take the allocator's locks.  aew_dot allocates a small partial-sum buffer on
// every call; this variant keeps that buffer in a fixed array in device global memory
// instead and calls no allocating routine.
//
// Scratch: g_dot_partials, a file-scope __device__ array of kMaxPartials doubles
// (512 KiB).  Every GPU that loads the library holds it until the process exits.
// One block reduces kChunk elements, so n may be at most kMaxPartials * kChunk = 2^32.
// All calls share the array: calls that overlap on the GPU (on different streams, or
// from different host threads) race on it and must be serialised by the caller.  Each
// call writes every partial it later reads, so no clearing is needed between calls.
//
// The host cannot use the array's name as a device address: at the first call on each
// device (with that device current) the library looks up its address with
// cudaGetSymbolAddress and caches it, keyed by the device's current context (its
// process-unique ID), so that a context created anew -- after cudaDeviceReset, say --
// gets its own lookup instead of a stale address.  That first call on a device (and on
// each new context) must therefore not happen while a stream is being captured.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include "../../include/aewave.h"

namespace {

constexpr long long kChunk = 65536;     // elements reduced by one block
constexpr int kMaxPartials = 65536;     // blocks per call => n <= 2^32
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dot_partials[kMaxPartials];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {};
unsigned long long g_ctx[kMaxDevices] = {};   // ID of the context g_addr belongs to

__global__ void dot_chunks_kernel(const float* __restrict__ a, const float* __restrict__ b,
                                  size_t n, double* part) {
  const size_t lo = (size_t)blockIdx.x * kChunk;
  const size_t hi = lo + kChunk < n ? lo + kChunk : n;
  double acc = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += kThreads) acc += (double)a[i] * (double)b[i];
  __shared__ double sw[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sw[w];
    part[blockIdx.x] = s;
  }
}

__global__ void dot_sum_kernel(const double* part, int nblk, double* out_dev) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
  __shared__ double sw[1024 / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += sw[w];
    *out_dev = s;
  }
}

// ID of the calling thread's current context (0 if none is current or the driver
// entry points are unavailable), through the driver entry points the runtime exposes
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && f && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && f && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// device address of the scratch array on the current device, looked up once per device
// and context (the lookup makes the device's primary context current if none was)
double* scratch_on_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long id = current_context_id();
  if (!g_addr[dev] || id == 0 || id != g_ctx[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dot_partials) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_addr[dev] = static_cast<double*>(p);
    g_ctx[dev] = current_context_id();
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int aew_dot_noalloc(const float* a_dev, const float* b_dev, size_t n, double* out_dev,
                               void* stream) {
  if (!a_dev || !b_dev || !out_dev) return AEW_E_ARG;
  if (n > (size_t)kMaxPartials * (size_t)kChunk) return AEW_E_ARG;   // beyond the scratch
  double* part = scratch_on_current_device();
  if (!part) return AEW_E_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nblk = (int)((n + kChunk - 1) / kChunk);
  if (nblk > 0) dot_chunks_kernel<<<nblk, kThreads, 0, s>>>(a_dev, b_dev, n, part);
  dot_sum_kernel<<<1, 1024, 0, s>>>(part, nblk, out_dev);
  return cudaGetLastError() == cudaSuccess ? AEW_OK : AEW_E_CUDA;
}
