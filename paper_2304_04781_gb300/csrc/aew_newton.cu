// MAP estimation with the BiLaplacian prior (Sec. 2) by inexact Newton-CG, and the
// DIAS active subspace (Sec. 4.3), built on the gradient and Hessian-vector solves of
// aew_api.cu.
//
// The solves dominate: one Newton iteration is a gradient plus up to cg_max
// Hessian-vector products, each two or three wave solves over the whole history.
// What runs here besides them is HBM-bound vector work: the prior operator (a 7-point
// stencil with zero-flux boundaries, one thread per node, neighbours through L1/L2), the
// projection onto the inactive subspace, CG updates, and FP64-accumulated inner
// products.  Arithmetic is FP32 -- GB300's FP64 rate is a small fraction of its FP32
// rate -- with FP64 only in the reductions.
//
// Prior solve A x = w: conjugate gradients whose scalars never leave the device.  Each
// kernel that needs rr or p^T A p sums the previous kernel's per-block FP64 partials
// itself (every block in the same order, so all blocks agree), so an iteration is three
// launches and the host reads the residual only every 8 iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/aewave.h"
#include "aew_internal.cuh"
#include "aew_pca.h"
#include "aew_solver.h"

namespace aew {
namespace {

constexpr int NT = 256;
constexpr int kVecBlocks = 152 * 4;   // grid of the vector kernels (grid-stride)
constexpr int kMaxN = 64;             // DIAS gradient samples
constexpr int kMaxR = 32;             // DIAS active subspace dimension
constexpr int kGramTile = 64;         // nodes per Gram tile

struct Grid {
  int nx, ny, nz;
  size_t C;
};

int vec_grid(size_t n) {
  const size_t b = (n + NT - 1) / NT;
  return (int)std::max<size_t>(1, std::min<size_t>(b, kVecBlocks));
}

// block-level FP64 sum of v into part[blockIdx.x]
__device__ void block_store(double v, double* part) {
  __shared__ double sw[NT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sw[w];
    part[blockIdx.x] = s;
  }
  __syncthreads();
}

// sum of part[0..n) by the whole block, in a fixed order (all blocks agree)
__device__ double block_sum_of(const double* __restrict__ part, int n) {
  __shared__ double sw[NT / 32];
  __shared__ double total;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) v += part[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sw[w];
    total = s;
  }
  __syncthreads();
  return total;
}

// The prior solve's reductions keep each thread's terms in FP32 and move them into an
// FP64 accumulator every kFlush terms: one FP64 add per kFlush elements instead of one
// FP64 FMA per element (GB300's FP64 rate would otherwise bound these passes below HBM
// speed).  That is safe there because the solve works on vectors scaled to unit rms;
// the Newton driver's vectors (gradients near 1e-20 per node) would underflow in FP32
// squares, so its inner products multiply in FP64.
constexpr int kFlush = 16;

struct Acc {
  double d = 0.0;
  float f = 0.f;
  int n = 0;
  __device__ __forceinline__ void add(float x) {
    f += x;
    if (++n == kFlush) {
      d += (double)f;
      f = 0.f;
      n = 0;
    }
  }
  __device__ __forceinline__ double total() const { return d + (double)f; }
};

// y = A x (+ yadd) with A x = alpha x - alpha theta / h^2 * sum over the neighbours a node
// has of (x_nb - x); optional partials of sum wdot . (A x).  One warp per grid row
// (k, y), each lane four consecutive nodes (nx is a multiple of 4 and the vectors are
// 16-byte aligned): one float4 load per row below, above, in front and behind, and the
// x neighbours by shuffle, the row's ends of each 128-node stretch loaded by lanes 0 and
// 31.  y may be yadd; x must not overlap y.
__device__ __forceinline__ float f4c(const float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__global__ void prior_kernel(const float* __restrict__ x, float* y, const float* yadd, Grid g,
                             float alpha, float at, const float* __restrict__ wdot, double* part) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * NT) >> 5;
  const int nrow = g.ny * g.nz;
  const int nq = g.nx >> 2;   // float4 per row
  const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  Acc acc;
  for (int row = (blockIdx.x * NT + threadIdx.x) >> 5; row < nrow; row += warps) {
    const int j = row % g.ny, k = row / g.ny;
    const size_t base = (size_t)row * g.nx;
    for (int q0 = 0; q0 < nq; q0 += 32) {   // the same trip count in every lane
      const int q = q0 + lane;
      const bool in = q < nq;
      const size_t n = base + 4 * (size_t)q;
      const float4 xc = in ? *reinterpret_cast<const float4*>(x + n) : z4;
      float xl = __shfl_up_sync(0xffffffffu, xc.w, 1);     // node 4q - 1
      float xr = __shfl_down_sync(0xffffffffu, xc.x, 1);   // node 4q + 4
      if (!in) continue;
      const int i = 4 * q;
      if (lane == 0 && i > 0) xl = x[n - 1];
      if (lane == 31 && q + 1 < nq) xr = x[n + 4];
      const float4 ym = j > 0 ? *reinterpret_cast<const float4*>(x + n - sy) : z4;
      const float4 yp = j + 1 < g.ny ? *reinterpret_cast<const float4*>(x + n + sy) : z4;
      const float4 zm = k > 0 ? *reinterpret_cast<const float4*>(x + n - sz) : z4;
      const float4 zp = k + 1 < g.nz ? *reinterpret_cast<const float4*>(x + n + sz) : z4;
      float v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float xn = f4c(xc, c);
        float lap = 0.f;
        if (i + c > 0) lap += (c == 0 ? xl : f4c(xc, c - 1)) - xn;
        if (i + c + 1 < g.nx) lap += (c == 3 ? xr : f4c(xc, c + 1)) - xn;
        if (j > 0) lap += f4c(ym, c) - xn;
        if (j + 1 < g.ny) lap += f4c(yp, c) - xn;
        if (k > 0) lap += f4c(zm, c) - xn;
        if (k + 1 < g.nz) lap += f4c(zp, c) - xn;
        v[c] = alpha * xn - at * lap;
      }
      if (part) {
        const float4 w = *reinterpret_cast<const float4*>(wdot + n);
        acc.add(w.x * v[0]);
        acc.add(w.y * v[1]);
        acc.add(w.z * v[2]);
        acc.add(w.w * v[3]);
      }
      if (yadd) {
        const float4 ya = *reinterpret_cast<const float4*>(yadd + n);
        v[0] += ya.x;
        v[1] += ya.y;
        v[2] += ya.z;
        v[3] += ya.w;
      }
      *reinterpret_cast<float4*>(y + n) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
  if (part) block_store(acc.total(), part);
}

// out = a x + b y (either of x, y may be out); n a multiple of 4
__global__ void axpby_kernel(float a, const float* x, float b, const float* y, float* out,
                             size_t n) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* y4 = reinterpret_cast<const float4*>(y);
  float4* o4 = reinterpret_cast<float4*>(out);
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * NT) {
    const float4 u = x4[i], v = y4[i];
    o4[i] = make_float4(a * u.x + b * v.x, a * u.y + b * v.y, a * u.z + b * v.z, a * u.w + b * v.w);
  }
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}

// FP64 products and sums (any magnitudes)
__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, size_t n,
                           double* part) {
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * NT) {
    const float4 u = a4[i], v = b4[i];
    acc += (double)u.x * v.x + (double)u.y * v.y + (double)u.z * v.z + (double)u.w * v.w;
  }
  block_store(acc, part);
}

// CG for A x = w, FP32 vectors, scalars from FP64 partials (see the file comment).
// update: a = rr / pAp; x += a p; r -= a Ap; partials of r.r into prr_new
__global__ void cg_update_kernel(float* __restrict__ x, float* __restrict__ r,
                                 const float* __restrict__ p, const float* __restrict__ Ap,
                                 size_t n, const double* ppap, const double* prr, int nblk,
                                 double* prr_new) {
  const double pap = block_sum_of(ppap, nblk);
  const double rr = block_sum_of(prr, nblk);
  const float a = pap > 0.0 ? (float)(rr / pap) : 0.f;
  float4* x4 = reinterpret_cast<float4*>(x);
  float4* r4 = reinterpret_cast<float4*>(r);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(Ap);
  Acc acc;
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * NT) {
    const float4 pi = p4[i], qi = q4[i];
    float4 xi = x4[i], ri = r4[i];
    xi.x += a * pi.x; xi.y += a * pi.y; xi.z += a * pi.z; xi.w += a * pi.w;
    ri.x -= a * qi.x; ri.y -= a * qi.y; ri.z -= a * qi.z; ri.w -= a * qi.w;
    x4[i] = xi;
    r4[i] = ri;
    acc.add(dot4(ri, ri));
  }
  block_store(acc.total(), prr_new);
}

// direction: p = r + (rr_new / rr_old) p
__global__ void cg_dir_kernel(float* __restrict__ p, const float* __restrict__ r, size_t n,
                              const double* prr_old, const double* prr_new, int nblk) {
  const double ro = block_sum_of(prr_old, nblk);
  const double rn = block_sum_of(prr_new, nblk);
  const float b = ro > 0.0 ? (float)(rn / ro) : 0.f;
  float4* p4 = reinterpret_cast<float4*>(p);
  const float4* r4 = reinterpret_cast<const float4*>(r);
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * NT) {
    const float4 ri = r4[i];
    float4 pi = p4[i];
    pi.x = ri.x + b * pi.x; pi.y = ri.y + b * pi.y; pi.z = ri.z + b * pi.z; pi.w = ri.w + b * pi.w;
    p4[i] = pi;
  }
}

// projection: partial dots of v with the r rows of W1, part[k][nblk]
__global__ void proj_dots_kernel(const float* __restrict__ W1, int r, const float* __restrict__ v,
                                 size_t n, double* part) {
  const float4* v4 = reinterpret_cast<const float4*>(v);
  for (int k = 0; k < r; ++k) {
    const float4* w4 = reinterpret_cast<const float4*>(W1 + (size_t)k * n);
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n / 4; i += (size_t)gridDim.x * NT) {
      const float4 u = w4[i], x = v4[i];
      acc += (double)u.x * x.x + (double)u.y * x.y + (double)u.z * x.z + (double)u.w * x.w;
    }
    block_store(acc, part + (size_t)k * gridDim.x);
  }
}

// out = v - sum_k (W1_k . v) W1_k, the coefficients summed from proj_dots_kernel's partials
__global__ void proj_apply_kernel(const float* __restrict__ W1, int r, const float* v, float* out,
                                  size_t n, const double* part, int nblk) {
  __shared__ float coef[kMaxR];
  for (int k = 0; k < r; ++k) {
    const double s = block_sum_of(part + (size_t)k * nblk, nblk);
    if (threadIdx.x == 0) coef[k] = (float)s;
  }
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    float acc = v[i];
    for (int k = 0; k < r; ++k) acc -= coef[k] * W1[(size_t)k * n + i];
    out[i] = acc;
  }
}

// Gram matrix of the N rows of G: per block, FP32 sums over 64-node tiles staged in
// shared memory, accumulated in FP64; part[block][pair], pairs (a <= b) row-major
__global__ void gram_kernel(const float* __restrict__ G, int N, size_t n, double* part) {
  __shared__ float tile[kMaxN][kGramTile + 1];
  const int npair = N * (N + 1) / 2;
  constexpr int kPer = (kMaxN * (kMaxN + 1) / 2 + NT - 1) / NT;
  double acc[kPer];
  int pa[kPer], pb[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    acc[q] = 0.0;
    int p = threadIdx.x + q * NT, a = 0;
    pa[q] = -1;
    pb[q] = -1;
    if (p < npair) {
      while (p >= N - a) {   // row a holds pairs (a, a..N-1)
        p -= N - a;
        ++a;
      }
      pa[q] = a;
      pb[q] = a + p;
    }
  }
  const size_t ntile = (n + kGramTile - 1) / kGramTile;
  for (size_t t = blockIdx.x; t < ntile; t += gridDim.x) {
    const size_t base = t * kGramTile;
    __syncthreads();
    for (int e = threadIdx.x; e < N * kGramTile; e += NT) {
      const int row = e / kGramTile, col = e % kGramTile;
      const size_t i = base + col;
      tile[row][col] = i < n ? G[(size_t)row * n + i] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      if (pa[q] < 0) continue;
      float s = 0.f;
      for (int c = 0; c < kGramTile; ++c) s += tile[pa[q]][c] * tile[pb[q]][c];
      acc[q] += (double)s;
    }
  }
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int p = threadIdx.x + q * NT;
    if (p < npair) part[(size_t)blockIdx.x * npair + p] = acc[q];
  }
}

// M[a][b] = M[b][a] = scale * sum over blocks of part[.][pair]
__global__ void gram_sum_kernel(const double* part, int nblk, int N, double scale, double* M) {
  const int npair = N * (N + 1) / 2;
  for (int p = blockIdx.x * NT + threadIdx.x; p < npair; p += gridDim.x * NT) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * npair + p];
    int a = 0, q = p;
    while (q >= N - a) {
      q -= N - a;
      ++a;
    }
    M[a * N + a + q] = scale * s;
    M[(a + q) * N + a] = scale * s;
  }
}

// W1[k][i] = sum_j coef[j][k] G[j][i]
__global__ void combine_kernel(const float* __restrict__ G, int N, size_t n,
                               const float* __restrict__ coef, int r, float* __restrict__ W1) {
  __shared__ float cs[kMaxN * kMaxR];
  for (int e = threadIdx.x; e < N * r; e += NT) cs[e] = coef[e];
  __syncthreads();
  for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
    float acc[kMaxR];
#pragma unroll
    for (int k = 0; k < kMaxR; ++k) acc[k] = 0.f;
    for (int j = 0; j < N; ++j) {
      const float gj = G[(size_t)j * n + i];
#pragma unroll
      for (int k = 0; k < kMaxR; ++k)
        if (k < r) acc[k] += cs[j * r + k] * gj;
    }
#pragma unroll
    for (int k = 0; k < kMaxR; ++k)
      if (k < r) W1[(size_t)k * n + i] = acc[k];
  }
}

// ---------------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------------
#define NW_CK(expr)                                                         \
  do {                                                                      \
    cudaError_t _e = (expr);                                                \
    if (_e != cudaSuccess)                                                  \
      return set_error(h, AEW_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// device buffers of one call, freed when it returns
struct Work {
  std::vector<void*> ptrs;
  ~Work() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  bool alloc(T** p, size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return false;
    }
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
  }
};

struct Ops {
  aew_handle* h;
  Grid g;
  cudaStream_t s;
  double* part;        // [kVecBlocks] FP64 partials
  double* ppart;       // [kMaxR][kVecBlocks] projection partials
  std::vector<double> hp;

  int grid() const { return vec_grid(g.C); }

  int axpby(float a, const float* x, float b, const float* y, float* out) {
    axpby_kernel<<<grid(), NT, 0, s>>>(a, x, b, y, out, g.C);
    NW_CK(cudaGetLastError());
    return AEW_OK;
  }
  int copy(const float* x, float* out) {
    NW_CK(cudaMemcpyAsync(out, x, g.C * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return AEW_OK;
  }
  // host FP64 inner product (synchronises)
  int dot(const float* a, const float* b, double* out) {
    const int nb = grid();
    dot_kernel<<<nb, NT, 0, s>>>(a, b, g.C, part);
    NW_CK(cudaGetLastError());
    hp.resize(nb);
    NW_CK(cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    NW_CK(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int i = 0; i < nb; ++i) acc += hp[i];
    *out = acc;
    return AEW_OK;
  }
  // y = A x (+ yadd)
  int prior(double alpha, double theta, double hh, const float* x, float* y,
            const float* yadd = nullptr) {
    prior_kernel<<<grid(), NT, 0, s>>>(x, y, yadd, g, (float)alpha,
                                       (float)(alpha * theta / (hh * hh)), nullptr, nullptr);
    NW_CK(cudaGetLastError());
    return AEW_OK;
  }
  // out = P v = v - W1^T (W1 v)  (out may be v)
  int project(const float* W1, int r, const float* v, float* out) {
    const int nb = grid();
    proj_dots_kernel<<<nb, NT, 0, s>>>(W1, r, v, g.C, ppart);
    NW_CK(cudaGetLastError());
    proj_apply_kernel<<<nb, NT, 0, s>>>(W1, r, v, out, g.C, ppart, nb);
    NW_CK(cudaGetLastError());
    return AEW_OK;
  }
};

// every grid vector is read as float4
bool aligned16(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int prior_args_ok(aew_handle* h, double alpha, double theta) {
  if (!(alpha > 0.0) || !std::isfinite(alpha))
    return set_error(h, AEW_E_ARG, "prior alpha must be positive and finite");
  if (!(theta >= 0.0) || !std::isfinite(theta))
    return set_error(h, AEW_E_ARG, "prior theta must be non-negative and finite");
  return AEW_OK;
}

// CG on A x = w (device scalars); x_dev written
int prior_cg(aew_handle* h, const Grid& g, double hh, double alpha, double theta,
             const float* w, float* x, double rtol, int max_iter, int* iters, cudaStream_t s) {
  Work ws;
  float *r, *p, *Ap;
  double* part;   // [3][kVecBlocks]: p.Ap, rr (two parities)
  if (!ws.alloc(&r, g.C) || !ws.alloc(&p, g.C) || !ws.alloc(&Ap, g.C) ||
      !ws.alloc(&part, 3 * (size_t)kVecBlocks))
    return set_error(h, AEW_E_NOMEM, "prior solve: work vectors do not fit");
  const int nb = vec_grid(g.C);
  double* ppap = part;
  double* prr[2] = {part + kVecBlocks, part + 2 * kVecBlocks};
  const float fa = (float)alpha, fat = (float)(alpha * theta / (hh * hh));
  dot_kernel<<<nb, NT, 0, s>>>(w, w, g.C, prr[0]);
  NW_CK(cudaGetLastError());
  std::vector<double> hp(nb);
  auto host_sum = [&](const double* dpart, double* out) -> int {
    NW_CK(cudaMemcpyAsync(hp.data(), dpart, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    NW_CK(cudaStreamSynchronize(s));
    double a = 0.0;
    for (int i = 0; i < nb; ++i) a += hp[i];
    *out = a;
    return AEW_OK;
  };
  double ww = 0.0;
  int rc = host_sum(prr[0], &ww);
  if (rc) return rc;
  if (iters) *iters = 0;
  if (ww == 0.0) {   // w = 0: x = 0
    NW_CK(cudaMemsetAsync(x, 0, g.C * sizeof(float), s));
    return AEW_OK;
  }
  // solve for the unit-rms right-hand side sc w (the iteration's FP32 squares then stay
  // far from FP32's range limits), and scale x back at the end
  const double sc = std::sqrt((double)g.C / ww);
  NW_CK(cudaMemsetAsync(x, 0, g.C * sizeof(float), s));
  axpby_kernel<<<nb, NT, 0, s>>>((float)sc, w, 0.f, w, r, g.C);
  axpby_kernel<<<nb, NT, 0, s>>>((float)sc, w, 0.f, w, p, g.C);
  NW_CK(cudaGetLastError());
  dot_kernel<<<nb, NT, 0, s>>>(r, r, g.C, prr[0]);
  NW_CK(cudaGetLastError());
  if ((rc = host_sum(prr[0], &ww))) return rc;
  const double tol2 = rtol * rtol * ww;
  int it = 0;
  for (; it < max_iter; ++it) {
    const int cur = it & 1, nxt = cur ^ 1;
    prior_kernel<<<nb, NT, 0, s>>>(p, Ap, nullptr, g, fa, fat, p, ppap);
    cg_update_kernel<<<nb, NT, 0, s>>>(x, r, p, Ap, g.C, ppap, prr[cur], nb, prr[nxt]);
    cg_dir_kernel<<<nb, NT, 0, s>>>(p, r, g.C, prr[cur], prr[nxt], nb);
    NW_CK(cudaGetLastError());
    if ((it & 7) == 7 || it + 1 == max_iter) {
      double rr = 0.0;
      if ((rc = host_sum(prr[nxt], &rr))) return rc;
      if (rr <= tol2) {
        ++it;
        if (iters) *iters = it;
        axpby_kernel<<<nb, NT, 0, s>>>((float)(1.0 / sc), x, 0.f, x, x, g.C);
        NW_CK(cudaGetLastError());
        return AEW_OK;
      }
    }
  }
  if (iters) *iters = it;
  axpby_kernel<<<nb, NT, 0, s>>>((float)(1.0 / sc), x, 0.f, x, x, g.C);
  NW_CK(cudaGetLastError());
  char buf[160];
  std::snprintf(buf, sizeof buf, "prior solve: relative residual above %.3g after %d iterations",
                rtol, max_iter);
  return set_error(h, AEW_E_NOCONVERGE, buf);
}

}  // namespace
}  // namespace aew

using aew::Grid;
using aew::set_error;

extern "C" {

int aew_prior_apply(aew_handle* h, double alpha, double theta, const float* q_dev,
                    float* out_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!q_dev || !out_dev) return set_error(h, AEW_E_ARG, "NULL vector");
  if (!aew::aligned16(q_dev) || !aew::aligned16(out_dev))
    return set_error(h, AEW_E_ARG, "vectors must be 16-byte aligned");
  int rc = aew::prior_args_ok(h, alpha, theta);
  if (rc) return rc;
  const aew::GridInfo gi = aew::grid_of(h);
  const Grid g{gi.nx, gi.ny, gi.nz, gi.C};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  aew::prior_kernel<<<aew::vec_grid(g.C), aew::NT, 0, s>>>(
      q_dev, out_dev, nullptr, g, (float)alpha, (float)(alpha * theta / (gi.h * gi.h)), nullptr,
      nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(h, AEW_E_CUDA, cudaGetErrorString(e));
  return AEW_OK;
}

int aew_prior_solve(aew_handle* h, double alpha, double theta, const float* w_dev, float* x_dev,
                    double rtol, int max_iter, int* iters_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!w_dev || !x_dev) return set_error(h, AEW_E_ARG, "NULL vector");
  if (!aew::aligned16(w_dev) || !aew::aligned16(x_dev))
    return set_error(h, AEW_E_ARG, "vectors must be 16-byte aligned");
  if (!(rtol > 0.0) || max_iter < 1) return set_error(h, AEW_E_ARG, "rtol > 0, max_iter >= 1");
  int rc = aew::prior_args_ok(h, alpha, theta);
  if (rc) return rc;
  const aew::GridInfo gi = aew::grid_of(h);
  const Grid g{gi.nx, gi.ny, gi.nz, gi.C};
  return aew::prior_cg(h, g, gi.h, alpha, theta, w_dev, x_dev, rtol, max_iter, iters_host,
                       static_cast<cudaStream_t>(stream));
}

int aew_newton_cg(aew_handle* h, float* c_dev, const float* d_obs_dev, const float* c0_dev,
                  const aew_newton_cfg* cfg, const float* W1_dev, int r,
                  aew_newton_iter* hist_host, int* iters_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!c_dev || !c0_dev || !cfg) return set_error(h, AEW_E_ARG, "NULL argument");
  if (!aew::aligned16(c_dev) || !aew::aligned16(c0_dev) || !aew::aligned16(W1_dev))
    return set_error(h, AEW_E_ARG, "c, c0 and W1 must be 16-byte aligned");
  int rc = aew::prior_args_ok(h, cfg->alpha, cfg->theta);
  if (rc) return rc;
  if (cfg->newton_iters < 1 || cfg->cg_max < 1 || cfg->max_backtracks < 1 ||
      !(cfg->c1 > 0.0 && cfg->c1 < 1.0) || !(cfg->eta_max > 0.0) || !(cfg->gtol >= 0.0))
    return set_error(h, AEW_E_ARG, "bad Newton-CG settings");
  if (W1_dev ? (r < 1 || r > aew::kMaxR) : r != 0)
    return set_error(h, AEW_E_ARG, "W1 needs 1 <= r <= 32 rows (r = 0 without W1)");
  if (iters_host) *iters_host = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const aew::GridInfo gi = aew::grid_of(h);
  const Grid g{gi.nx, gi.ny, gi.nz, gi.C};
  const double al = cfg->alpha, th = cfg->theta, hh = gi.h;

  aew::Work ws;
  float *g_tot, *gm, *x, *res, *d, *Hd, *t1, *t2, *ct;
  double *part, *ppart;
  if (!ws.alloc(&g_tot, g.C) || !ws.alloc(&gm, g.C) || !ws.alloc(&x, g.C) ||
      !ws.alloc(&res, g.C) || !ws.alloc(&d, g.C) || !ws.alloc(&Hd, g.C) || !ws.alloc(&t1, g.C) ||
      !ws.alloc(&t2, g.C) || !ws.alloc(&ct, g.C) || !ws.alloc(&part, aew::kVecBlocks) ||
      !ws.alloc(&ppart, (size_t)aew::kMaxR * aew::kVecBlocks))
    return set_error(h, AEW_E_NOMEM, "Newton-CG: work vectors do not fit");
  aew::Ops op{h, g, s, part, ppart, {}};

  // R(c) = 1/2 |A P (c - c0)|^2 and, with grad, grad = P A^2 P (c - c0)
  auto reg = [&](const float* c, double* R, float* grad) -> int {
    int e = op.axpby(1.f, c, -1.f, c0_dev, t1);
    if (!e && W1_dev) e = op.project(W1_dev, r, t1, t1);
    if (!e) e = op.prior(al, th, hh, t1, t2);
    if (!e) e = op.dot(t2, t2, R);
    if (e) return e;
    *R *= 0.5;
    if (!grad) return AEW_OK;
    if ((e = op.prior(al, th, hh, t2, grad))) return e;
    if (W1_dev) e = op.project(W1_dev, r, grad, grad);
    return e;
  };
  // Hd = H_misfit v + P A^2 P v
  auto hess = [&](const float* v, float* out) -> int {
    int e = cfg->full_hessian ? aew_hessvec_full(h, v, out, stream) : aew_hessvec(h, v, out, stream);
    if (e) return e;
    const float* vin = v;
    if (W1_dev) {
      if ((e = op.project(W1_dev, r, v, t1))) return e;
      vin = t1;
    }
    if ((e = op.prior(al, th, hh, vin, t2))) return e;
    if (W1_dev) {
      if ((e = op.prior(al, th, hh, t2, t1))) return e;
      if ((e = op.project(W1_dev, r, t1, t1))) return e;
      return op.axpby(1.f, out, 1.f, t1, out);
    }
    return op.prior(al, th, hh, t2, out, out);
  };

  double Jm = 0.0;
  bool ok = true;
  if ((rc = aew::gradient_gated(h, c_dev, d_obs_dev, gm, INFINITY, &Jm, &ok, s))) return rc;
  double g0n = -1.0;
  for (int it = 0; it < cfg->newton_iters; ++it) {
    double R = 0.0;
    if ((rc = reg(c_dev, &R, g_tot))) return rc;
    if ((rc = op.axpby(1.f, gm, 1.f, g_tot, g_tot))) return rc;
    double gg = 0.0;
    if ((rc = op.dot(g_tot, g_tot, &gg))) return rc;
    const double gn = std::sqrt(gg), J = Jm + R;
    if (g0n < 0.0) g0n = gn;
    if (cfg->gtol > 0.0 && gn <= cfg->gtol * g0n) break;
    const double eta = std::min(cfg->eta_max, std::sqrt(g0n > 0.0 ? gn / g0n : 0.0));

    // CG on H x = -g from x = 0
    NW_CK(cudaMemsetAsync(x, 0, g.C * sizeof(float), s));
    if ((rc = op.axpby(-1.f, g_tot, 0.f, g_tot, res))) return rc;
    if ((rc = op.copy(res, d))) return rc;
    double rr = gg;
    int k = 0;
    for (k = 1; k <= cfg->cg_max; ++k) {
      if ((rc = hess(d, Hd))) return rc;
      double dHd = 0.0;
      if ((rc = op.dot(d, Hd, &dHd))) return rc;
      if (!(dHd > 0.0)) {   // negative (or no) curvature: keep the current iterate
        --k;
        break;
      }
      const double a = rr / dHd;
      if ((rc = op.axpby((float)a, d, 1.f, x, x))) return rc;
      if ((rc = op.axpby((float)-a, Hd, 1.f, res, res))) return rc;
      double rr_new = 0.0;
      if ((rc = op.dot(res, res, &rr_new))) return rc;
      if (std::sqrt(rr_new) <= eta * gn) break;
      if ((rc = op.axpby(1.f, res, (float)(rr_new / rr), d, d))) return rc;
      rr = rr_new;
    }
    if (k > cfg->cg_max) k = cfg->cg_max;
    if (k == 0 && (rc = op.axpby(-1.f, g_tot, 0.f, g_tot, x))) return rc;   // steepest descent
    double slope = 0.0;
    if ((rc = op.dot(g_tot, x, &slope))) return rc;

    // Armijo backtracking; each trial's gradient stops after its forward solve if the
    // misfit already fails the test.  A trial outside the stability bound (or with
    // c <= 0) fails like a cost increase.
    double step = 1.0, Jm_t = 0.0;
    int bt = 0;
    bool accepted = false;
    for (; bt < cfg->max_backtracks; ++bt) {
      if ((rc = op.axpby((float)step, x, 1.f, c_dev, ct))) return rc;
      double Rt = 0.0;
      if ((rc = reg(ct, &Rt, nullptr))) return rc;
      const double gate = J + cfg->c1 * step * slope - Rt;
      rc = aew::gradient_gated(h, ct, d_obs_dev, gm, gate, &Jm_t, &accepted, s);
      if (rc == AEW_E_CFL || rc == AEW_E_CONFIG) {
        accepted = false;
        rc = AEW_OK;
      }
      if (rc) return rc;
      if (accepted) break;
      step *= 0.5;
    }
    if (!accepted) {   // no sufficient decrease along x: stop at the current iterate
      if (hist_host) hist_host[it] = aew_newton_iter{J, J - R, R, gn, k, bt, 0.0};
      if (iters_host) *iters_host = it + 1;
      break;
    }
    if ((rc = op.copy(ct, c_dev))) return rc;
    Jm = Jm_t;
    if (hist_host) hist_host[it] = aew_newton_iter{J, J - R, R, gn, k, bt, step};
    if (iters_host) *iters_host = it + 1;
  }
  aew::set_error(h, AEW_OK, "");
  NW_CK(cudaStreamSynchronize(s));
  return AEW_OK;
}

int aew_dias_subspace(aew_handle* h, const float* c_dev, const float* d_obs_dev,
                      const float* noise_dev, int N, double alpha, double theta, int r,
                      float* G_dev, float* W1_dev, double* lambda_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!c_dev || !noise_dev || !G_dev || !W1_dev || !lambda_host)
    return set_error(h, AEW_E_ARG, "NULL argument");
  if (!aew::aligned16(c_dev) || !aew::aligned16(noise_dev) || !aew::aligned16(G_dev) ||
      !aew::aligned16(W1_dev))
    return set_error(h, AEW_E_ARG, "c, noise, G and W1 must be 16-byte aligned");
  if (N < 1 || N > aew::kMaxN || r < 1 || r > N || r > aew::kMaxR)
    return set_error(h, AEW_E_ARG, "need 1 <= r <= N <= 64 and r <= 32");
  int rc = aew::prior_args_ok(h, alpha, theta);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const aew::GridInfo gi = aew::grid_of(h);
  const Grid g{gi.nx, gi.ny, gi.nz, gi.C};
  aew::Work ws;
  float *cs, *coef;
  double *part, *M;
  const int npair = N * (N + 1) / 2;
  const int gb = aew::vec_grid(g.C);
  if (!ws.alloc(&cs, g.C) || !ws.alloc(&coef, (size_t)N * r) ||
      !ws.alloc(&part, (size_t)gb * npair) || !ws.alloc(&M, (size_t)N * N))
    return set_error(h, AEW_E_NOMEM, "DIAS: work vectors do not fit");
  aew::Ops op{h, g, s, nullptr, nullptr, {}};
  // CG iterations for rtol 1e-6 grow with sqrt of A's condition number
  const double kappa = 1.0 + 12.0 * theta / (gi.h * gi.h);
  const int max_iter = (int)std::min(100000.0, 1000.0 + 40.0 * std::sqrt(kappa));
  for (int i = 0; i < N; ++i) {
    float* gi_dev = G_dev + (size_t)i * g.C;
    if ((rc = aew::prior_cg(h, g, gi.h, alpha, theta, noise_dev + (size_t)i * g.C, cs, 1e-6,
                            max_iter, nullptr, s)))
      return rc;
    if ((rc = op.axpby(1.f, c_dev, 1.f, cs, cs))) return rc;
    double J = 0.0;
    bool ok = true;
    if ((rc = aew::gradient_gated(h, cs, d_obs_dev, gi_dev, INFINITY, &J, &ok, s))) return rc;
  }
  aew::gram_kernel<<<gb, aew::NT, 0, s>>>(G_dev, N, g.C, part);
  aew::gram_sum_kernel<<<(npair + aew::NT - 1) / aew::NT, aew::NT, 0, s>>>(part, gb, N, 1.0 / N, M);
  NW_CK(cudaGetLastError());
  std::vector<double> Mh((size_t)N * N), V((size_t)N * N), w(N);
  NW_CK(cudaMemcpyAsync(Mh.data(), M, Mh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  NW_CK(cudaStreamSynchronize(s));
  if (!aew::sym_eig(N, Mh.data(), w.data(), V.data()))
    return set_error(h, AEW_E_ARG, "DIAS: eigensolver did not converge");
  for (int j = 0; j < N; ++j) lambda_host[j] = w[j];
  if (!(w[r - 1] > 0.0)) return set_error(h, AEW_E_ARG, "DIAS: fewer than r positive eigenvalues");
  std::vector<float> ch((size_t)N * r);
  for (int j = 0; j < N; ++j)
    for (int k = 0; k < r; ++k)
      ch[(size_t)j * r + k] = (float)(V[(size_t)j * N + k] / std::sqrt(N * w[k]));
  NW_CK(cudaMemcpyAsync(coef, ch.data(), ch.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  aew::combine_kernel<<<gb, aew::NT, 0, s>>>(G_dev, N, g.C, coef, r, W1_dev);
  NW_CK(cudaGetLastError());
  NW_CK(cudaStreamSynchronize(s));
  return AEW_OK;
}

}  // extern "C"
