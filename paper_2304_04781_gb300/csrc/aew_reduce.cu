// Elementwise preparation, FP64 reductions and gradient finalisation.
//
// FP64 is used only for the time-summed gradient accumulator, the misfit and the
// inner products of the adjoint-identity / finite-difference checks.  Reductions are
// two-pass (fixed per-block partial sums, then one block) so results are
// deterministic run to run.
#include "aew_internal.cuh"

#include <cmath>

namespace aew {
namespace {

constexpr int RT = 256;

__device__ __forceinline__ bool finite_f(float v) { return isfinite(v); }

__global__ void prep_m_kernel(const float* __restrict__ c, float* __restrict__ m, size_t n,
                              FieldCheck* chk) {
  unsigned int bad = 0, neg = 0;
  float mx = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = c[i];
    m[i] = v * v;
    if (!finite_f(v)) {
      ++bad;
    } else {
      if (v <= 0.f) ++neg;
      mx = fmaxf(mx, v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
    neg += __shfl_xor_sync(0xffffffffu, neg, o);
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicAdd(&chk->nonfinite, bad);
    if (neg) atomicAdd(&chk->cneg, neg);
    atomicMax(&chk->cmax_bits, __float_as_uint(mx));
  }
}

__global__ void prep_dm_kernel(const float* __restrict__ c, const float* __restrict__ dc,
                               float* __restrict__ dm, size_t n, FieldCheck* chk) {
  unsigned int bad = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float v = dc[i];
    if (!finite_f(v)) ++bad;
    dm[i] = 2.f * c[i] * v;
  }
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&chk->nonfinite, bad);
}

// block-level FP64 sum into part[blockIdx.x]
__device__ void block_sum_store(double v, double* part) {
  __shared__ double sw[RT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RT / 32; ++w) s += sw[w];
    part[blockIdx.x] = s;
  }
}

__global__ void residual_kernel(const float* __restrict__ d, const float* __restrict__ dobs,
                                float* __restrict__ r, size_t n_row0, size_t n, double* part) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (i >= n_row0) {
      v = d[i] - dobs[i];
      acc += (double)v * (double)v;
    }
    r[i] = v;
  }
  block_sum_store(acc, part);
}

__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n,
                           double* part) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    acc += (double)a[i] * (double)b[i];
  block_sum_store(acc, part);
}

__global__ void sum_partials_kernel(const double* part, int nblk, double scale, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) acc += part[i];
  __shared__ double sw[RT / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RT / 32; ++w) s += sw[w];
    out[0] = scale * s;
  }
}

__global__ void finalize_grad_kernel(const float* __restrict__ c, const double* __restrict__ acc,
                                     float* __restrict__ g, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    g[i] = (float)(2.0 * (double)c[i] * acc[i]);
}

// full Newton HVP in c: H dc = 2 c (accA + accB) + (dc / c) g, with g = 2 c dJ/dm the
// gradient of the same c (so (dc / c) g = 2 dc dJ/dm)
__global__ void finalize_hvp_full_kernel(const float* __restrict__ c, const float* __restrict__ dc,
                                         const double* __restrict__ a, const double* __restrict__ b,
                                         const float* __restrict__ g, float* __restrict__ out,
                                         size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const double ci = (double)c[i];
    out[i] = (float)(2.0 * ci * (a[i] + b[i]) + (double)dc[i] / ci * (double)g[i]);
  }
}

int grid_for(size_t n) {
  size_t b = (n + RT - 1) / RT;
  if (b > 152 * 8) b = 152 * 8;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_prep_m(const float* c, float* m, size_t n, FieldCheck* chk, cudaStream_t s) {
  prep_m_kernel<<<grid_for(n), RT, 0, s>>>(c, m, n, chk);
  return cudaGetLastError();
}
cudaError_t launch_prep_dm(const float* c, const float* dc, float* dm, size_t n, FieldCheck* chk,
                           cudaStream_t s) {
  prep_dm_kernel<<<grid_for(n), RT, 0, s>>>(c, dc, dm, n, chk);
  return cudaGetLastError();
}
cudaError_t launch_residual(const float* d, const float* dobs, float* r, size_t n_row0, size_t n,
                            double* part, int nblk, cudaStream_t s) {
  residual_kernel<<<nblk, RT, 0, s>>>(d, dobs, r, n_row0, n, part);
  return cudaGetLastError();
}
cudaError_t launch_dot_partials(const float* a, const float* b, size_t n, double* part, int nblk,
                                cudaStream_t s) {
  dot_kernel<<<nblk, RT, 0, s>>>(a, b, n, part);
  return cudaGetLastError();
}
cudaError_t launch_sum_partials(const double* part, int nblk, double scale, double* out,
                                cudaStream_t s) {
  sum_partials_kernel<<<1, RT, 0, s>>>(part, nblk, scale, out);
  return cudaGetLastError();
}
cudaError_t launch_finalize_grad(const float* c, const double* acc64, float* g, size_t n,
                                 cudaStream_t s) {
  finalize_grad_kernel<<<grid_for(n), RT, 0, s>>>(c, acc64, g, n);
  return cudaGetLastError();
}
cudaError_t launch_finalize_hvp_full(const float* c, const float* dc, const double* a,
                                     const double* b, const float* g, float* out, size_t n,
                                     cudaStream_t s) {
  finalize_hvp_full_kernel<<<grid_for(n), RT, 0, s>>>(c, dc, a, b, g, out, n);
  return cudaGetLastError();
}

}  // namespace aew
