// Per-block autoencoder codec on tcgen05 tensor cores (compression in space, Sec. 3.1;
// dense layers sigma(y W + b) of Eq. (5), Sec. 3.3), plus the snapshot packing of
// Algorithm 1.
//
// Block vector of an 8x8x8-node block: k = z*256 + f*64 + y*8 + x (f = e, vx, vy, vz);
// block b = (bz*NBy + by)*NBx + bx.  Each field of each block is divided by its
// power-of-two scale s_{b,f} = 2^max(e, -100), m 2^e (m in [1/2, 1)) the block's max |f|
// (exact in BF16).  Inside the gradient the forward step packs and normalises the
// vectors itself; the entry points here pack a given state (pack_raw_kernel, then
// normalise_kernel).
//
// Encoder: A = normalised BF16 block vectors, times W1 (2048 x 512) -> +b1, GELU -> H
// (BF16), times W2 (512 x n_lat) -> +b2 -> FP16 latent.  Decoder: latent (FP16) times W3
// (FP16, n_lat x 512) -> +b3, GELU -> H (BF16), times W4 (BF16, 512 x 2048, or only its
// 512 strain columns inside the adjoint) -> +b4, times s_{b,e}, scattered back to the grid.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "aew_codec.cuh"
#include "aew_codec_state.cuh"
#include "aew_dec.cuh"
#include "aew_gemm2.cuh"
#include "aew_gemm.cuh"

namespace aew {


namespace {

// the four weight transposes of codec_refresh in one launch: a block takes one 32 x 32
// tile of one matrix (tile prefix per matrix)
struct Transposes {
  const float* src[4];
  uint16_t* dst[4];
  int rows[4], cols[4], fp16[4];
  int tiles[5];
};
__global__ void transpose_multi_kernel(Transposes t) {
  __shared__ float tile[32][33];
  int m = 0;
  while (m < 3 && (int)blockIdx.x >= t.tiles[m + 1]) ++m;
  const int rows = t.rows[m], cols = t.cols[m];
  const int tx = (cols + 31) / 32;
  const int b = blockIdx.x - t.tiles[m];
  const int c0 = (b % tx) * 32, r0 = (b / tx) * 32;
  const float* src = t.src[m];
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * cols + c] : 0.f;
  }
  __syncthreads();
  uint16_t* dst = t.dst[m];
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float v = tile[threadIdx.x][i];
      uint16_t bits;
      if (t.fp16[m]) {
        __half hv = __float2half_rn(v);
        bits = *reinterpret_cast<uint16_t*>(&hv);
      } else {
        bits = gemm::bf16_bits(v);
      }
      dst[(size_t)c * rows + r] = bits;
    }
  }
}

// ---------------------------------------------------------------------------------
// Epilogues
// ---------------------------------------------------------------------------------
// hidden-layer activation of the inference epilogues: GELU (ACT 0) or the paper's ELU
// (ACT 1: e^a - 1 below 0, a above)
template <int ACT>
__device__ __forceinline__ float act_fwd(float a) {
  if (ACT == 1) return a > 0.f ? a : expm1f(a);
  return gemm::gelu_fast(a);
}
// bf16x2 of (act(x0), act(x1)); GELU on the paired FP32 lanes
template <int ACT>
__device__ __forceinline__ uint32_t act_pack2(float x0, float x1) {
  if (ACT == 0) gemm::gelu_fast_pair(x0, x1);
  else x0 = act_fwd<ACT>(x0), x1 = act_fwd<ACT>(x1);
  return gemm::pack_bf16(x0, x1);
}
// (x0 + b0, x1 + b1) and (x0 s + b0, x1 s + b1) on the paired lanes
__device__ __forceinline__ void add2(float& x0, float& x1, float b0, float b1) {
  gemm::f2::split(gemm::f2::add(gemm::f2::make(x0, x1), gemm::f2::make(b0, b1)), x0, x1);
}
__device__ __forceinline__ void fma2(float& x0, float& x1, float s, float b0, float b1) {
  gemm::f2::split(gemm::f2::fma(gemm::f2::make(x0, x1), gemm::f2::splat(s), gemm::f2::make(b0, b1)),
                  x0, x1);
}

// H[row][col..] = bf16(act(acc + bias)), row stride ld
template <int ACT>
struct EpBiasAct {
  const float* bias;
  uint16_t* H;
  long long M;
  int ld;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    const float4* bq = reinterpret_cast<const float4*>(bias + col);
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      const float4 b = __ldg(bq + j / 4);
      float x0 = v[j], x1 = v[j + 1], x2 = v[j + 2], x3 = v[j + 3];
      add2(x0, x1, b.x, b.y);
      add2(x2, x3, b.z, b.w);
      pk[j / 2] = act_pack2<ACT>(x0, x1);
      pk[j / 2 + 1] = act_pack2<ACT>(x2, x3);
    }
    uint16_t* dst = H + row * ld + col;   // 32-byte aligned: ld and col multiples of 32
    gemm::st_global_32B(dst, pk[0], pk[1], pk[2], pk[3], pk[4], pk[5], pk[6], pk[7]);
    gemm::st_global_32B(dst + 16, pk[8], pk[9], pk[10], pk[11], pk[12], pk[13], pk[14], pk[15]);
  }
};

using EpBiasGeluH = EpBiasAct<0>;

// Encoder layer 1 of the time codec on raw (unnormalised) BF16 window vectors:
// H[row][col..] = bf16(act(acc / s_row + bias)), s_row the vector's power-of-two scale
// from its max |e| (vmax, float bits).  Dividing the FP32 sum by a power of two equals
// summing the normalised products (the scale commutes with every rounding involved).
template <int ACT>
struct EpScaleAct {
  const float* bias;
  const unsigned* vmax;
  uint16_t* H;
  long long M;
  int ld;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    const float is = gemm::block_inv_scale(__uint_as_float(__ldg(vmax + row)));
    const float4* bq = reinterpret_cast<const float4*>(bias + col);
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      const float4 b = __ldg(bq + j / 4);
      float x0 = v[j], x1 = v[j + 1], x2 = v[j + 2], x3 = v[j + 3];
      fma2(x0, x1, is, b.x, b.y);
      fma2(x2, x3, is, b.z, b.w);
      pk[j / 2] = act_pack2<ACT>(x0, x1);
      pk[j / 2 + 1] = act_pack2<ACT>(x2, x3);
    }
    uint16_t* dst = H + row * ld + col;   // 32-byte aligned: ld and col multiples of 32
    gemm::st_global_32B(dst, pk[0], pk[1], pk[2], pk[3], pk[4], pk[5], pk[6], pk[7]);
    gemm::st_global_32B(dst + 16, pk[8], pk[9], pk[10], pk[11], pk[12], pk[13], pk[14], pk[15]);
  }
};

// Decoder layer 2 of the time codec, scattered to the window's strain slices:
// column n = t*128 + z*64 + y*8 + x of vector row (bz, by, bx) -> slice t, node
// (2bz + z, 8by + y, 8bx + x); e = (acc + b4[n]) * s_row, 0 on boundary nodes.
// A 32-column group is 4 rows of 8 nodes: two float4 stores per row.
struct EpDecWindow {
  const float* b4;
  const unsigned* vmax;
  float* e;               // slice 0 of [16][nz][ny][nx]
  int nx, ny, nz, NBx, NBy;
  long long M;            // vectors (< 2^31)
  size_t slice;           // nx ny nz
  const double* mn;       // min-max normalisation (else null): offset and range
  const double* rr;
  bool bf16;              // write the slices as BF16 ([16][nz][ny][nx] uint16 from e)
  __device__ __forceinline__ void operator()(long long rw, int col, const float (&v)[32]) const {
    if (rw >= M) return;
    const int r = (int)rw;
    const int bx = r % NBx, q = r / NBx;
    const int by = q % NBy, bz = q / NBy;
    const float sc = rr ? (float)__ldg(rr + r) : gemm::block_scale(__uint_as_float(__ldg(vmax + r)));
    const float off = rr ? (float)__ldg(mn + r) : 0.f;
    const int t = col >> 7, z = (col >> 6) & 1, y0 = (col & 63) >> 3;
    const int kz = 2 * bz + z;
    const bool zb = kz == 0 || kz == nz - 1;
    const bool xlo = bx == 0, xhi = bx == NBx - 1;
    float* base = e + (size_t)t * slice + ((size_t)kz * ny + 8 * by + y0) * nx + 8 * bx;
    const float4* bq = reinterpret_cast<const float4*>(b4 + col);
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
      const int jy = 8 * by + y0 + yy;
      const bool yb = zb || jy == 0 || jy == ny - 1;
      const float4 blo = __ldg(bq + 2 * yy), bhi = __ldg(bq + 2 * yy + 1);
      const float bv[8] = {blo.x, blo.y, blo.z, blo.w, bhi.x, bhi.y, bhi.z, bhi.w};
      float o[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const float val = fmaf(v[yy * 8 + x] + bv[x], sc, off);
        o[x] = (yb || (x == 0 && xlo) || (x == 7 && xhi)) ? 0.f : val;
      }
      if (bf16) {   // the same element index in the BF16 view: one 16-byte store
        const size_t idx = (size_t)(base - e) + (size_t)yy * nx;
        *reinterpret_cast<uint4*>(reinterpret_cast<uint16_t*>(e) + idx) =
            make_uint4(gemm::pack_bf16(o[0], o[1]), gemm::pack_bf16(o[2], o[3]),
                       gemm::pack_bf16(o[4], o[5]), gemm::pack_bf16(o[6], o[7]));
      } else {
        float4* dst = reinterpret_cast<float4*>(base + (size_t)yy * nx);
        dst[0] = make_float4(o[0], o[1], o[2], o[3]);
        dst[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
  }
};

// latent = fp16(acc + bias), flag overflow
struct EpLatent {
  const float* bias;
  uint16_t* lat;
  int nl;
  long long M;
  int* ovf;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M || col >= nl) return;
    const float4* bq = reinterpret_cast<const float4*>(bias + col);
    uint32_t pk[16];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
      const float4 b = __ldg(bq + j / 4);
      const float a[4] = {v[j] + b.x, v[j + 1] + b.y, v[j + 2] + b.z, v[j + 3] + b.w};
#pragma unroll
      for (int h = 0; h < 4; h += 2) {
        const __half2 hv = __floats2half2_rn(a[h], a[h + 1]);
        bad |= !(fabsf(a[h]) <= 65504.f) || !(fabsf(a[h + 1]) <= 65504.f);
        pk[(j + h) / 2] = *reinterpret_cast<const uint32_t*>(&hv);
      }
    }
    if (bad) atomicOr(ovf, 1);
    uint16_t* dst = lat + row * nl + col;   // 32-byte aligned: nl and col multiples of 32
    gemm::st_global_32B(dst, pk[0], pk[1], pk[2], pk[3], pk[4], pk[5], pk[6], pk[7]);
    gemm::st_global_32B(dst + 16, pk[8], pk[9], pk[10], pk[11], pk[12], pk[13], pk[14], pk[15]);
  }
};

// strain part of the decoder output, scattered to the grid:
// column n = z*64 + y*8 + x of block row -> node (8bz+z, 8by+y, 8bx+x);
// e = (acc + b4[z*256 + y*8 + x]) * s_b (power-of-two block scale), 0 on boundary nodes.
// The row's block coordinates and scale are found once per row (Row), then each
// 32-column group is stored through it.
struct EpDecGrid {
  const float* b4;
  const unsigned* bmax;   // [nblocks][4] maxima of |f| (float bits); field 0 = strain
  float* e;
  int nx, ny, nz, NBx, NBy;
  long long M;            // number of blocks (< 2^31, checked by the launcher)
  struct Row {
    float* base;          // node (8bz, 8by, 8bx)
    float s;
    int kz0, jy0;         // 8bz, 8by
    bool live, xlo, xhi;  // row in range; block on the x = 0 / x = nx - 1 face
  };
  __device__ __forceinline__ Row row(long long rw) const {
    Row c;
    c.live = rw < M;
    if (!c.live) return c;
    const int r = (int)rw;
    const int bx = r % NBx, t = r / NBx;
    const int by = t % NBy, bz = t / NBy;
    c.s = gemm::block_scale(__uint_as_float(__ldg(bmax + (size_t)r * 4)));
    c.kz0 = 8 * bz;
    c.jy0 = 8 * by;
    c.base = e + ((size_t)c.kz0 * ny + c.jy0) * nx + 8 * bx;
    c.xlo = bx == 0;
    c.xhi = bx == NBx - 1;
    return c;
  }
  // b4 of a 32-column group (4 rows of 8 nodes): b4[z*256 + y*8 + x], 32 consecutive
  // floats from z*256 + y0*8
  struct Bias {
    float4 q[8];
  };
  __device__ __forceinline__ void bias(int col, Bias& bb) const {
    const float4* bq = reinterpret_cast<const float4*>(b4 + (col >> 6) * 256 + (col & 63));
#pragma unroll
    for (int j = 0; j < 8; ++j) bb.q[j] = __ldg(bq + j);
  }
  __device__ __forceinline__ void operator()(const Row& c, int col, const Bias& bb,
                                             const float (&v)[32]) const {
    if (!c.live) return;
    const int z = col >> 6, y0 = (col & 63) >> 3;
    const int kz = c.kz0 + z;
    const bool zb = (kz == 0 || kz == nz - 1);
    float* pz = c.base + (size_t)z * ny * nx;
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
      const int jy = c.jy0 + y0 + yy;
      const bool yb = zb || jy == 0 || jy == ny - 1;
      const float4 blo = bb.q[2 * yy], bhi = bb.q[2 * yy + 1];
      const float bv[8] = {blo.x, blo.y, blo.z, blo.w, bhi.x, bhi.y, bhi.z, bhi.w};
      float o[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const float val = (v[yy * 8 + x] + bv[x]) * c.s;
        o[x] = (yb || (x == 0 && c.xlo) || (x == 7 && c.xhi)) ? 0.f : val;
      }
      float4* dst = reinterpret_cast<float4*>(pz + (size_t)(y0 + yy) * nx);
      dst[0] = make_float4(o[0], o[1], o[2], o[3]);
      dst[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
};

// out[row][col..] = acc + bias (FP32 vectors)
struct EpVec {
  const float* bias;
  float* out;
  long long ld;
  long long M;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    float4* dst = reinterpret_cast<float4*>(out + row * ld + col);
    const float4* bq = reinterpret_cast<const float4*>(bias + col);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 b = __ldg(bq + q);
      dst[q] = make_float4(v[4 * q] + b.x, v[4 * q + 1] + b.y, v[4 * q + 2] + b.z, v[4 * q + 3] + b.w);
    }
  }
};


bool ensure_X(Codec* c, size_t rows) {
  if (c->X_rows >= rows) return true;
  if (c->X) cudaFree(c->X);
  c->X = nullptr;
  c->X_rows = 0;
  if (cudaMalloc(&c->X, rows * kNIn * sizeof(uint16_t)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->X_rows = rows;
  return true;
}

bool ensure_H(Codec* c, size_t rows) {
  if (c->H_rows >= rows) return true;
  if (c->H) cudaFree(c->H);
  c->H = nullptr;
  c->H_rows = 0;
  if (cudaMalloc(&c->H, rows * (size_t)c->n_hid * sizeof(uint16_t)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->H_rows = rows;
  return true;
}

// ---------------------------------------------------------------------------------
// Algorithm 1 packing: BF16 normalised block vectors
// ---------------------------------------------------------------------------------
// Raw BF16 block vectors of a grid state and the per-block, per-field maxima of |f|.
// One thread per float4 of a grid row: consecutive threads read consecutive x
// (coalesced) and write 8-byte pieces; the two threads of a block row combine their
// maxima by shuffle before the atomicMax.
__global__ void pack_raw_kernel(const float* f0, const float* f1, const float* f2,
                                const float* f3, int nx, int ny, int NBx, int NBy,
                                long long nblk, unsigned* bmax, uint16_t* out) {
  const int xq_n = nx >> 2;
  const long long total = nblk / NBx * 256LL * xq_n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long iters = (total + stride - 1) / stride;
  for (long long q = 0; q < iters; ++q) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x + q * stride;
    const bool live = t < total;
    const int xq = live ? (int)(t % xq_n) : 0;
    const long long r = live ? t / xq_n : 0;
    const int y = (int)(r & 7), f = (int)((r >> 3) & 3), z = (int)((r >> 5) & 7);
    const long long slab = r >> 8;               // (bz, by)
    const long long by = slab % NBy, bz = slab / NBy;
    const long long b = slab * NBx + (xq >> 1);
    float m = 0.f;
    if (live) {
      const float* src = f == 0 ? f0 : (f == 1 ? f1 : (f == 2 ? f2 : f3));
      const float4 a = *reinterpret_cast<const float4*>(
          src + ((size_t)(8 * bz + z) * ny + (size_t)(8 * by + y)) * nx + 4 * (size_t)xq);
      *reinterpret_cast<uint2*>(out + b * kNIn + z * 256 + f * 64 + y * 8 + 4 * (xq & 1)) =
          make_uint2(gemm::pack_bf16(a.x, a.y), gemm::pack_bf16(a.z, a.w));
      m = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
    }
    // xq and xq ^ 1 are adjacent lanes (xq_n is even) and share block b and field f
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if (live && (xq & 1) == 0 && m > 0.f) atomicMax(bmax + b * 4 + f, __float_as_uint(m));
  }
}

// y = x * 2^-e per block-field (exact), from raw BF16 vectors and block maxima; out may
// be raw itself (each thread rewrites only the 16 bytes it read)
__global__ void normalise_kernel(const uint16_t* raw, const unsigned* __restrict__ bmax,
                                 long long n, uint16_t* out) {
  const long long total = n * (kNIn / 8);   // 16-byte pieces
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / (kNIn / 8);
    const int k = (int)(t % (kNIn / 8)) * 8;
    const int f = (k >> 6) & 3;
    const float sc = gemm::block_inv_scale(__uint_as_float(bmax[b * 4 + f]));
    uint4 v = *reinterpret_cast<const uint4*>(raw + b * kNIn + k);
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      w[j] = gemm::pack_bf16(__uint_as_float(w[j] << 16) * sc, __uint_as_float(w[j] & 0xffff0000u) * sc);
    *reinterpret_cast<uint4*>(out + b * kNIn + k) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Strain fields e[t][nz][ny][nx] (t < nsteps; later slots 0) -> raw BF16 window
// vectors [nvec][2048], k = t*128 + z*64 + y*8 + x, and max |e| per vector (atomicMax;
// vmax zeroed by the caller).  One thread per float4 of a grid row; the two threads of
// an 8-node row combine their maxima by shuffle.
__global__ void window_pack_kernel(const float* __restrict__ e, int nsteps, int nx, int ny,
                                   int nz, uint16_t* __restrict__ raw, unsigned* vmax) {
  const int xq_n = nx >> 2;
  const long long total = (long long)kTSteps * nz * ny * xq_n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long iters = (total + stride - 1) / stride;
  const int NBx = nx >> 3, NBy = ny >> 3;
  for (long long q = 0; q < iters; ++q) {
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x + q * stride;
    const bool live = t0 < total;
    const int xq = live ? (int)(t0 % xq_n) : 0;
    long long r = live ? t0 / xq_n : 0;
    const int y = (int)(r % ny);
    r /= ny;
    const int z = (int)(r % nz);
    const int t = (int)(r / nz);
    const long long v = ((long long)(z >> 1) * NBy + (y >> 3)) * NBx + (xq >> 1);
    float m = 0.f;
    if (live) {
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
      if (t < nsteps)
        a = *reinterpret_cast<const float4*>(e + (((size_t)t * nz + z) * ny + y) * nx + 4 * (size_t)xq);
      *reinterpret_cast<uint2*>(raw + v * kNIn + t * 128 + (z & 1) * 64 + (y & 7) * 8 + 4 * (xq & 1)) =
          make_uint2(gemm::pack_bf16(a.x, a.y), gemm::pack_bf16(a.z, a.w));
      m = fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
    }
    // xq and xq ^ 1 are adjacent lanes (xq_n is even) and share vector v
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    if (live && (xq & 1) == 0 && m > 0.f) atomicMax(vmax + v, __float_as_uint(m));
  }
}

// y = x * 2^-e per vector (exact), from raw BF16 window vectors and their maxima; out
// may be raw itself (each thread rewrites only the 16 bytes it read)
__global__ void window_normalise_kernel(const uint16_t* raw, const unsigned* __restrict__ vmax,
                                        long long n, uint16_t* out) {
  const long long total = n * (kNIn / 8);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long b = t / (kNIn / 8);
    const int k = (int)(t % (kNIn / 8)) * 8;
    const float sc = gemm::block_inv_scale(__uint_as_float(vmax[b]));
    uint4 v = *reinterpret_cast<const uint4*>(raw + b * kNIn + k);
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 4; ++j)
      w[j] = gemm::pack_bf16(__uint_as_float(w[j] << 16) * sc, __uint_as_float(w[j] & 0xffff0000u) * sc);
    *reinterpret_cast<uint4*>(out + b * kNIn + k) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Moments of the PCA initialisation.  YT[i][v] = bf16(sqrt(w[n0 + v]) Y[n0 + v][i]) for
// v < nc, 0 for nc <= v < ncp (32 x 32 tiles through shared memory).
__global__ void moment_transpose_kernel(const uint16_t* __restrict__ Y, long long n0, int nc,
                                        int ncp, const float* __restrict__ w,
                                        uint16_t* __restrict__ YT, int ldT) {
  __shared__ uint16_t tile[32][34];
  const int i0 = blockIdx.x * 32, v0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int v = v0 + r, i = i0 + threadIdx.x;
    uint16_t b = 0;
    if (v < nc) {
      const uint16_t y = Y[(size_t)(n0 + v) * kNIn + i];
      b = w ? gemm::bf16_bits(gemm::bf16_val(y) * sqrtf(w[n0 + v])) : y;
    }
    tile[r][threadIdx.x] = b;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, v = v0 + threadIdx.x;
    if (v < ncp) YT[(size_t)i * ldT + v] = tile[threadIdx.x][r];
  }
}

// per-block partial sums part[b][0..2047] = sum_v w_v y_v, part[b][2048] = sum_v w_v over
// the vectors v = b, b + gridDim.x, ...; thread t owns columns 8t .. 8t + 7
__global__ void moment_sum_kernel(const uint16_t* __restrict__ Y, long long n,
                                  const float* __restrict__ w, double* __restrict__ part) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double sw = 0.0;
  for (long long v = blockIdx.x; v < n; v += gridDim.x) {
    const double wv = w ? (double)w[v] : 1.0;
    const uint4 q = *reinterpret_cast<const uint4*>(Y + (size_t)v * kNIn + 8 * threadIdx.x);
    const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[2 * j] += wv * (double)__uint_as_float(u[j] << 16);
      acc[2 * j + 1] += wv * (double)__uint_as_float(u[j] & 0xffff0000u);
    }
    sw += wv;
  }
  double* out = part + (size_t)blockIdx.x * (kNIn + 1);
#pragma unroll
  for (int j = 0; j < 8; ++j) out[8 * threadIdx.x + j] = acc[j];
  if (threadIdx.x == 0) out[kNIn] = sw;
}

// s64[i] = sum over blocks of part[b][i], in block order (deterministic)
__global__ void moment_reduce_kernel(const double* __restrict__ part, int nblk,
                                     double* __restrict__ s64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > kNIn) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (kNIn + 1) + i];
  s64[i] = s;
}

// Decoded-error sums of a chunk of vectors: acc[f] += sum (yh - y)^2, acc[4 + f] +=
// sum y^2, acc[8 + f] and acc[12 + f] the same times s^2 (physical units), per field f
// (time codec: every column is field 0).  One warp per vector, grid-stride; one set of
// atomics per block.
__global__ void eval_err_kernel(const uint16_t* __restrict__ Y, const float* __restrict__ Yh,
                                const float* __restrict__ mx, int time, int nc,
                                double* __restrict__ acc) {
  __shared__ double sh[8][16];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double a[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = 0.0;
  for (int v = blockIdx.x * 8 + wid; v < nc; v += gridDim.x * 8) {
    // time == 2 (min-max): mx is [n][2] = (offset, range), x = y r + offset
    float sc[4];
    const float off = time == 2 ? mx[2 * (size_t)v] : 0.f;
#pragma unroll
    for (int f = 0; f < 4; ++f)
      sc[f] = time == 2 ? mx[2 * (size_t)v + 1]
                        : gemm::block_scale(time ? mx[v] : mx[(size_t)v * 4 + f]);
    for (int k = lane; k < kNIn; k += 32) {
      const int f = time ? 0 : ((k >> 6) & 3);
      const double y = (double)gemm::bf16_val(Y[(size_t)v * kNIn + k]);
      const double d = (double)Yh[(size_t)v * kNIn + k] - y;
      const double s2 = (double)sc[f] * (double)sc[f];
      const double x = y * (double)sc[f] + (double)off;
#pragma unroll
      for (int g = 0; g < 4; ++g)
        if (g == f) {
          a[g] += d * d;
          a[4 + g] += y * y;
          a[8 + g] += d * d * s2;
          a[12 + g] += x * x;
        }
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    for (int o = 16; o > 0; o >>= 1) a[j] += __shfl_xor_sync(0xffffffffu, a[j], o);
  if (lane == 0)
    for (int j = 0; j < 16; ++j) sh[wid][j] = a[j];
  __syncthreads();
  if (threadIdx.x < 16) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, t);
  }
}

// The paper's min-max normalisation of raw BF16 window vectors, one warp per vector:
// min and max of its 2048 values, r = max(max - min, beta), y = (x - min) / r in FP32,
// one rounding to BF16 (in place allowed: each lane rewrites what it read); the offset
// and range are kept in FP64.
__global__ void window_minmax_kernel(const uint16_t* raw, long long nvec, double beta,
                                     uint16_t* out, double* __restrict__ mn,
                                     double* __restrict__ rr, float2* __restrict__ pair32) {
  const int lane = threadIdx.x & 31;
  for (long long v = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; v < nvec;
       v += ((long long)gridDim.x * blockDim.x) >> 5) {
    const uint4* src = reinterpret_cast<const uint4*>(raw + (size_t)v * kNIn);
    uint4 q[8];
    float lo = INFINITY, hi = -INFINITY;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      q[k] = src[k * 32 + lane];
      const uint32_t w[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float a = __uint_as_float(w[j] << 16), b = __uint_as_float(w[j] & 0xffff0000u);
        lo = fminf(lo, fminf(a, b));
        hi = fmaxf(hi, fmaxf(a, b));
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double r = fmax((double)hi - (double)lo, beta);
    const float fl = lo, ir = (float)(1.0 / r);
    uint4* dst = reinterpret_cast<uint4*>(out + (size_t)v * kNIn);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      uint32_t w[4] = {q[k].x, q[k].y, q[k].z, q[k].w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        w[j] = gemm::pack_bf16((__uint_as_float(w[j] << 16) - fl) * ir,
                               (__uint_as_float(w[j] & 0xffff0000u) - fl) * ir);
      dst[k * 32 + lane] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (lane == 0) {
      if (mn) mn[v] = (double)lo;
      if (rr) rr[v] = r;
      if (pair32) pair32[v] = make_float2(lo, (float)r);
    }
  }
}

__global__ void vector_weights_kernel(const float* __restrict__ mx, long long n, int pw,
                                      float* __restrict__ w) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const float sc = gemm::block_scale(mx[v]);
    w[v] = pw == 1 ? sc : sc * sc;
  }
}

// G64[row][col..] += acc (one tile owns each element: no atomics)
struct EpGramAcc {
  double* G;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= kNIn) return;
    double* g = G + row * kNIn + col;
#pragma unroll
    for (int j = 0; j < 32; ++j) g[j] += (double)v[j];
  }
};

// strain rows of W4t (vector index z*256 + j, j < 64) packed as W4e [512][512]
__global__ void strain_rows_kernel(const uint16_t* __restrict__ W4t, uint16_t* __restrict__ W4e) {
  const int r = blockIdx.x, k = threadIdx.x;
  const int src = (r >> 6) * 256 + (r & 63);
  for (int q = k; q < kNHid; q += blockDim.x) W4e[(size_t)r * kNHid + q] = W4t[(size_t)src * kNHid + q];
}


}  // namespace

// =================================================================================
namespace gemm {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        fn == nullptr || q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  return encode;
}

CUresult make_tmap(CUtensorMap* map, const void* base, bool fp16, long long rows, int K,
                   long long ld, int box_rows, bool swizzle128) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return CUDA_ERROR_NOT_FOUND;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {swizzle128 ? 64u : 8u, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return encode(map, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace gemm

// the inference epilogues' GELU and the training kernels' GELU derivative, element by
// element (test hook)
__global__ void activation_probe_kernel(const float* __restrict__ x, float* __restrict__ y,
                                        float* __restrict__ dy, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = x[i];
    // GELU as the epilogues evaluate it, on the pair (x[2k], x[2k+1]) that holds x[i];
    // NaN where it differs in any bit from the scalar form
    const long long j = i ^ 1;
    const float w = j < n ? x[j] : v;
    float lo = (i & 1) ? w : v, hi = (i & 1) ? v : w;
    gemm::gelu_fast_pair(lo, hi);
    const float yp = (i & 1) ? hi : lo;
    y[i] = __float_as_uint(yp) == __float_as_uint(gemm::gelu_fast(v)) ? yp
                                                                      : __uint_as_float(0x7fc00000u);
    dy[i] = gemm::gelu_prime_f(v);
  }
}
cudaError_t launch_activation_probe(const float* x, float* y, float* dy, long long n,
                                    cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + 255) / 256;
  const int grid = (int)(want < 152 * 8 ? want : 152 * 8);
  activation_probe_kernel<<<grid, 256, 0, s>>>(x, y, dy, n);
  return cudaGetLastError();
}

Codec* codec_new(int n_lat, bool time) {
  Codec* c = new Codec();
  c->n_lat = n_lat;
  c->time = time;
  c->n_hid = time ? 2 * n_lat : kNHid;
  const size_t nl = (size_t)n_lat, nh = (size_t)c->n_hid;
  const size_t sz[8] = {(size_t)kNIn * nh, nh, nh * nl, nl, nl * nh, nh, nh * kNIn, kNIn};
  bool ok = true;
  for (int i = 0; i < 8 && ok; ++i) {
    c->wn[i] = sz[i];
    ok = cudaMalloc(&c->w[i], sz[i] * sizeof(float)) == cudaSuccess;
    c->bytes += sz[i] * sizeof(float);
  }
  ok = ok && cudaMalloc(&c->W1t, (size_t)kNIn * nh * 2) == cudaSuccess &&
       cudaMalloc(&c->W2t, nl * nh * 2) == cudaSuccess &&
       cudaMalloc(&c->W3t, nl * nh * 2) == cudaSuccess &&
       cudaMalloc(&c->W4t, (size_t)kNIn * nh * 2) == cudaSuccess &&
       (time || cudaMalloc(&c->W4e, (size_t)512 * kNHid * 2) == cudaSuccess) &&
       cudaMalloc(&c->err, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&c->sc_tmp, 4 * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    codec_free(c);
    return nullptr;
  }
  cudaMemset(c->err, 0, sizeof(int));
  if (const char* env = getenv("AEW_GEMM_CTAS")) c->max_ctas = atoi(env);   // tuning override
  if (const char* env = getenv("AEW_GEMM_STAGES")) c->max_stages = atoi(env);   // tuning override
  if (const char* env = getenv("AEW_GEMM_PAIR")) c->pair_gemm = atoi(env) != 0;  // tuning override
  c->bytes += ((size_t)2 * kNIn * nh + 2 * nl * nh + (time ? 0 : (size_t)512 * kNHid)) * 2;
  return c;
}

void codec_free(Codec* c) {
  if (!c) return;
  for (float* p : c->w) cudaFree(p);
  cudaFree(c->W1t);
  cudaFree(c->W2t);
  cudaFree(c->W3t);
  cudaFree(c->W4t);
  cudaFree(c->W4e);
  cudaFree(c->H);
  cudaFree(c->X);
  cudaFree(c->sc_tmp);
  cudaFree(c->err);
  if (c->train) train_state_free(c->train);
  delete c;
}

int codec_nlat(const Codec* c) { return c->n_lat; }
int codec_nhid(const Codec* c) { return c->n_hid; }
void codec_reset_training(Codec* c) {
  if (c->train) train_state_free(c->train);
  c->train = nullptr;
}

int* codec_err_flag(Codec* c) { return c->err; }

bool codec_take_error(Codec* c, cudaStream_t s) {
  int v = 0;
  if (cudaMemcpyAsync(&v, c->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return true;
  if (v) cudaMemsetAsync(c->err, 0, sizeof(int), s);
  return v != 0;
}
size_t codec_device_bytes(const Codec* c) {
  return c->bytes + c->H_rows * (size_t)c->n_hid * 2 + c->X_rows * kNIn * 2 +
         (c->train ? train_state_bytes(c->train) : 0);
}
bool codec_ready(const Codec* c) { return c && c->ready; }

// refresh the tensor-core operand copies from the FP32 masters
cudaError_t codec_refresh(Codec* c, cudaStream_t s) {
  const int nl = c->n_lat, nh = c->n_hid;
  cudaError_t e;
  Transposes t{{c->w[0], c->w[2], c->w[4], c->w[6]}, {c->W1t, c->W2t, c->W3t, c->W4t},
               {kNIn, nh, nl, nh}, {nh, nl, nh, kNIn}, {0, 0, 1, 0}, {0, 0, 0, 0, 0}};
  for (int m = 0; m < 4; ++m)
    t.tiles[m + 1] = t.tiles[m] + ((t.rows[m] + 31) / 32) * ((t.cols[m] + 31) / 32);
  transpose_multi_kernel<<<t.tiles[4], dim3(32, 8), 0, s>>>(t);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (c->time) return cudaSuccess;
  strain_rows_kernel<<<512, 128, 0, s>>>(c->W4t, c->W4e);
  return cudaGetLastError();
}

cudaError_t codec_set_weights(Codec* c, const float* const w[8]) {
  for (int i = 0; i < 8; ++i) {
    cudaError_t e = cudaMemcpy(c->w[i], w[i], c->wn[i] * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = codec_refresh(c, 0);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(0);
  if (e == cudaSuccess) c->ready = true;
  return e;
}

cudaError_t codec_get_weights(const Codec* c, float* const w[8]) {
  cudaError_t e = cudaDeviceSynchronize();
  for (int i = 0; i < 8 && e == cudaSuccess; ++i)
    e = cudaMemcpy(w[i], c->w[i], c->wn[i] * sizeof(float), cudaMemcpyDeviceToHost);
  return e;
}

cudaError_t codec_encode_grid(Codec* c, const float* const f[4], int nx, int ny, int nz,
                              unsigned* bmax, uint16_t* lat, int* overflow, cudaStream_t s) {
  const long long nb = (long long)(nx / 8) * (ny / 8) * (nz / 8);
  if (!ensure_X(c, (size_t)nb)) return cudaErrorMemoryAllocation;
  // raw BF16 block vectors and block maxima, then normalised in place
  cudaError_t e = snapshot_pack(f, nx, ny, nz, bmax, c->X, c->X, s);
  if (e != cudaSuccess) return e;
  return codec_encode_vectors(c, c->X, nb, lat, overflow, s);
}


static int ctas_of(const Codec* c, int ctas) { return ctas > 0 ? ctas : c->max_ctas; }

// the time codec's products are all wide (N >= 512, hundreds of thousands of rows): they
// run on SM pairs, whose 256 x 256 tiles pull a third fewer operand bytes per SM
static bool pair_wide(const Codec* c) { return c->time && c->pair_gemm && c->max_stages == 0; }

// encoder layer 2: latents = fp16(H W2 + b2) from the hidden activations in c->H
static cudaError_t encode_layer2(Codec* c, long long n, uint16_t* lat, int* overflow,
                                 cudaStream_t s, int g) {
  const int nl = c->n_lat, nh = c->n_hid;
  EpLatent e2{c->w[3], lat, nl, n, overflow};
  const gemm::Mat a2{c->H, n, nh}, b2{c->W2t, nl, nh};
  if (pair_wide(c)) return gemm2::launch<true>(n, nl, nh, a2, b2, e2, c->err, s, g);
  if (nl == 64) return gemm::launch<64, true>(n, nl, nh, a2, b2, e2, c->err, s, g, c->max_stages);
  if (nl == 32) return gemm::launch<32, true>(n, nl, nh, a2, b2, e2, c->err, s, g, c->max_stages);
  return gemm::launch<256, true>(n, nl, nh, a2, b2, e2, c->err, s, g, c->max_stages);
}

// encoder layer 1 on normalised vectors with epilogue EP (bias + activation)
template <class EP>
static cudaError_t encode_layer1(Codec* c, const uint16_t* vec, long long n, const EP& ep,
                                 cudaStream_t s, int g) {
  const int nh = c->n_hid;
  const gemm::Mat a1{vec, n, kNIn}, b1{c->W1t, nh, kNIn};
  return c->pair_gemm && c->max_stages == 0
             ? gemm2::launch<true>(n, nh, kNIn, a1, b1, ep, c->err, s, g)
             : gemm::launch<256, true>(n, nh, kNIn, a1, b1, ep, c->err, s, g, c->max_stages);
}

cudaError_t codec_encode_vectors(Codec* c, const uint16_t* vec, long long n, uint16_t* lat,
                                 int* overflow, cudaStream_t s, int ctas) {
  if (!ensure_H(c, (size_t)n)) return cudaErrorMemoryAllocation;
  const int g = ctas_of(c, ctas);
  const int nh = c->n_hid;
  cudaError_t e = c->act == 1 ? encode_layer1(c, vec, n, EpBiasAct<1>{c->w[1], c->H, n, nh}, s, g)
                              : encode_layer1(c, vec, n, EpBiasAct<0>{c->w[1], c->H, n, nh}, s, g);
  if (e != cudaSuccess) return e;
  return encode_layer2(c, n, lat, overflow, s, g);
}

template <int ACT>
static cudaError_t decode_hidden_t(Codec* c, const uint16_t* lat, long long nb, cudaStream_t s,
                                   int ctas) {
  const int nl = c->n_lat, nh = c->n_hid;
  EpBiasAct<ACT> ep{c->w[5], c->H, nb, nh};
  if (pair_wide(c))
    return gemm2::launch<false>(nb, nh, nl, gemm::Mat{lat, nb, nl}, gemm::Mat{c->W3t, nh, nl}, ep,
                                c->err, s, ctas_of(c, ctas));
  return gemm::launch<256, false>(nb, nh, nl, gemm::Mat{lat, nb, nl},
                                  gemm::Mat{c->W3t, nh, nl}, ep, c->err, s, ctas_of(c, ctas),
                                  c->max_stages);
}

static cudaError_t decode_hidden(Codec* c, const uint16_t* lat, long long nb, cudaStream_t s,
                                 int ctas) {
  if (!ensure_H(c, (size_t)nb)) return cudaErrorMemoryAllocation;
  return c->act == 1 ? decode_hidden_t<1>(c, lat, nb, s, ctas) : decode_hidden_t<0>(c, lat, nb, s, ctas);
}

// strain decode in one kernel: layer 1, GELU, layer 2 with H kept in shared memory
static cudaError_t decode_e_fused(Codec* c, const uint16_t* lat, long long nb, const EpDecGrid& ep,
                                  cudaStream_t s, int ctas) {
  static const cudaError_t attr = cudaFuncSetAttribute(
      dec::dec2_kernel<EpDecGrid>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dec::kSmem);
  if (attr != cudaSuccess) return attr;
  const int sms = gemm::sm_count();
  const int nl = c->n_lat;
  CUtensorMap tz, tw3, tw4;
  if (gemm::make_tmap(&tz, lat, true, nb, nl, nl, dec::kRows, true) != CUDA_SUCCESS ||
      gemm::make_tmap(&tw3, c->W3t, true, kNHid, nl, nl, 256, true) != CUDA_SUCCESS ||
      gemm::make_tmap(&tw4, c->W4e, false, 512, kNHid, kNHid, 256, true) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if (nb >= (1LL << 31)) return cudaErrorInvalidValue;
  const long long tiles = (nb + dec::kRows - 1) / dec::kRows;
  const int g = ctas_of(c, ctas);
  const int cap = (g > 0 && g < sms) ? g : sms;
  const int grid = (int)(tiles < cap ? tiles : cap);
  dec::dec2_kernel<EpDecGrid><<<grid, dec::kThreads, dec::kSmem, s>>>(tz, tw3, tw4, (int)nb,
                                                                      c->w[5], ep, c->err);
  return cudaGetLastError();
}

cudaError_t codec_decode_grid_e(Codec* c, const uint16_t* lat, int nx, int ny, int nz,
                                const unsigned* bmax, float* e_out, cudaStream_t s, int ctas) {
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 8;
  const long long nb = (long long)NBx * NBy * NBz;
  EpDecGrid ep{c->w[7], bmax, e_out, nx, ny, nz, NBx, NBy, nb};
  return decode_e_fused(c, lat, nb, ep, s, ctas);
}

cudaError_t codec_decode_vectors(Codec* c, const uint16_t* lat, long long nvec, float* out,
                                 cudaStream_t s) {
  cudaError_t e = decode_hidden(c, lat, nvec, s, 0);
  if (e != cudaSuccess) return e;
  const int nh = c->n_hid;
  EpVec ep{c->w[7], out, kNIn, nvec};
  return gemm::launch<256, true>(nvec, kNIn, nh, gemm::Mat{c->H, nvec, nh},
                                 gemm::Mat{c->W4t, kNIn, nh}, ep, c->err, s, c->max_ctas, c->max_stages);
}

// ---------------------------------------------------------------------------------
// Compression in time
// ---------------------------------------------------------------------------------
cudaError_t codec_encode_window(Codec* c, uint16_t* raw, const unsigned* vmax,
                                long long nvec, uint16_t* lat, int* overflow, cudaStream_t s,
                                int ctas, double* mn, double* rr) {
  if (!ensure_H(c, (size_t)nvec)) return cudaErrorMemoryAllocation;
  const int g = ctas_of(c, ctas);
  const int nh = c->n_hid;
  cudaError_t e;
  if (c->norm == 1) {   // the paper's min-max normalisation, then the plain layer 1
    if (!mn || !rr) return cudaErrorInvalidValue;
    if ((e = window_minmax(raw, nvec, c->beta, raw, mn, rr, s)) != cudaSuccess) return e;
    e = c->act == 1 ? encode_layer1(c, raw, nvec, EpBiasAct<1>{c->w[1], c->H, nvec, nh}, s, g)
                    : encode_layer1(c, raw, nvec, EpBiasAct<0>{c->w[1], c->H, nvec, nh}, s, g);
  } else {
    e = c->act == 1 ? encode_layer1(c, raw, nvec, EpScaleAct<1>{c->w[1], vmax, c->H, nvec, nh}, s, g)
                    : encode_layer1(c, raw, nvec, EpScaleAct<0>{c->w[1], vmax, c->H, nvec, nh}, s, g);
  }
  if (e != cudaSuccess) return e;
  return encode_layer2(c, nvec, lat, overflow, s, g);
}

cudaError_t codec_decode_window(Codec* c, const uint16_t* lat, const unsigned* vmax, int nx,
                                int ny, int nz, float* e_out, cudaStream_t s, int ctas,
                                const double* mn, const double* rr, bool bf16_out) {
  if (c->norm == 1 && (!mn || !rr)) return cudaErrorInvalidValue;
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 2;
  const long long nvec = (long long)NBx * NBy * NBz;
  if (nvec >= (1LL << 31)) return cudaErrorInvalidValue;
  cudaError_t e = decode_hidden(c, lat, nvec, s, ctas);
  if (e != cudaSuccess) return e;
  const int nh = c->n_hid;
  EpDecWindow ep{c->w[7], vmax, e_out, nx, ny, nz, NBx, NBy, nvec, (size_t)nx * ny * nz,
                 c->norm == 1 ? mn : nullptr, c->norm == 1 ? rr : nullptr, bf16_out};
  if (pair_wide(c))
    return gemm2::launch<true>(nvec, kNIn, nh, gemm::Mat{c->H, nvec, nh},
                               gemm::Mat{c->W4t, kNIn, nh}, ep, c->err, s, ctas_of(c, ctas));
  return gemm::launch<256, true>(nvec, kNIn, nh, gemm::Mat{c->H, nvec, nh},
                                 gemm::Mat{c->W4t, kNIn, nh}, ep, c->err, s, ctas_of(c, ctas),
                                 c->max_stages);
}

cudaError_t window_pack(const float* e, int nsteps, int nx, int ny, int nz, uint16_t* raw,
                        unsigned* vmax, cudaStream_t s) {
  const long long nvec = (long long)(nx / 8) * (ny / 8) * (nz / 2);
  cudaError_t err = cudaMemsetAsync(vmax, 0, (size_t)nvec * sizeof(unsigned), s);
  if (err != cudaSuccess) return err;
  const long long total = (long long)kTSteps * nz * ny * (nx / 4);
  long long blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  window_pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(e, nsteps, nx, ny, nz, raw, vmax);
  return cudaGetLastError();
}

cudaError_t codec_moments(Codec* c, const uint16_t* Y, long long n, const float* w, double* G64,
                          double* s64, cudaStream_t s) {
  constexpr int kChunk = 32768;   // vectors per GEMM (K); 128 MB of transposed BF16
  constexpr int kPartBlocks = 1024;
  uint16_t* YT = nullptr;
  double* part = nullptr;
  cudaError_t e = cudaMalloc(&YT, (size_t)kNIn * kChunk * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&part, (size_t)kPartBlocks * (kNIn + 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemsetAsync(G64, 0, (size_t)kNIn * kNIn * sizeof(double), s);
  if (e == cudaSuccess && n > 0) {
    moment_sum_kernel<<<kPartBlocks, kNIn / 8, 0, s>>>(Y, n, w, part);
    e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(part, 0, (size_t)kPartBlocks * (kNIn + 1) * sizeof(double), s);
  }
  if (e == cudaSuccess) {
    moment_reduce_kernel<<<(kNIn + 1 + 255) / 256, 256, 0, s>>>(part, kPartBlocks, s64);
    e = cudaGetLastError();
  }
  for (long long n0 = 0; e == cudaSuccess && n0 < n; n0 += kChunk) {
    const int nc = (int)std::min<long long>(kChunk, n - n0);
    const int ncp = (nc + 63) / 64 * 64;
    dim3 grid(kNIn / 32, ncp / 32), block(32, 8);
    moment_transpose_kernel<<<grid, block, 0, s>>>(Y, n0, nc, ncp, w, YT, kChunk);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = gemm::launch<256, true>(kNIn, kNIn, ncp, gemm::Mat{YT, kNIn, kChunk},
                                  gemm::Mat{YT, kNIn, kChunk}, EpGramAcc{G64}, c->err, s);
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  cudaFree(YT);
  cudaFree(part);
  return e;
}

cudaError_t vector_weights(const float* mx, long long n, int pw, float* w, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  vector_weights_kernel<<<152 * 8, 256, 0, s>>>(mx, n, pw, w);
  return cudaGetLastError();
}

cudaError_t codec_eval(Codec* c, const uint16_t* Y, const float* maxima, long long n,
                       double* out, cudaStream_t s) {
  constexpr int kChunk = 16384;
  uint16_t* lat = nullptr;
  float* dec = nullptr;
  double* acc = nullptr;
  int* ovf = nullptr;
  cudaError_t e = cudaMalloc(&lat, (size_t)kChunk * c->n_lat * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&dec, (size_t)kChunk * kNIn * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&acc, 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&ovf, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 16 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ovf, 0, sizeof(int), s);
  for (long long n0 = 0; e == cudaSuccess && n0 < n; n0 += kChunk) {
    const int nc = (int)std::min<long long>(kChunk, n - n0);
    e = codec_encode_vectors(c, Y + (size_t)n0 * kNIn, nc, lat, ovf, s);
    if (e == cudaSuccess) e = codec_decode_vectors(c, lat, nc, dec, s);
    if (e == cudaSuccess) {
      eval_err_kernel<<<1024, 256, 0, s>>>(Y + (size_t)n0 * kNIn, dec,
                                           maxima + (size_t)n0 * (c->time ? (c->norm == 1 ? 2 : 1) : 4),
                                           c->time ? (c->norm == 1 ? 2 : 1) : 0, nc, acc);
      e = cudaGetLastError();
    }
  }
  double h[16] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  cudaFree(lat);
  cudaFree(dec);
  cudaFree(acc);
  cudaFree(ovf);
  if (e != cudaSuccess) return e;
  auto rel = [](double num, double den) { return den > 0 ? std::sqrt(num / den) : 0.0; };
  double nd = 0, nn = 0, pd = 0, pn = 0;
  for (int f = 0; f < 4; ++f) {
    out[f] = rel(h[f], h[4 + f]);
    out[5 + f] = rel(h[8 + f], h[12 + f]);
    nd += h[f];
    nn += h[4 + f];
    pd += h[8 + f];
    pn += h[12 + f];
  }
  out[4] = rel(nd, nn);
  out[9] = rel(pd, pn);
  return cudaSuccess;
}

cudaError_t window_minmax(const uint16_t* raw, long long nvec, double beta, uint16_t* out,
                          double* mn, double* rr, cudaStream_t s, float* pair32) {
  if (nvec <= 0) return cudaSuccess;
  long long blocks = (nvec * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  window_minmax_kernel<<<(unsigned)blocks, 256, 0, s>>>(raw, nvec, beta, out, mn, rr,
                                                        reinterpret_cast<float2*>(pair32));
  return cudaGetLastError();
}

void codec_set_variant(Codec* c, int norm, int act, double beta) {
  c->norm = norm;
  c->act = act;
  c->beta = beta;
}
bool codec_minmax(const Codec* c) { return c->norm == 1; }
double codec_beta(const Codec* c) { return c->beta; }

cudaError_t window_normalise(const uint16_t* raw, const unsigned* vmax, long long nvec,
                             uint16_t* out, cudaStream_t s) {
  if (nvec <= 0) return cudaSuccess;
  window_normalise_kernel<<<152 * 8, 256, 0, s>>>(raw, vmax, nvec, out);
  return cudaGetLastError();
}

cudaError_t snapshot_pack(const float* const f[4], int nx, int ny, int nz, unsigned* bmax,
                          uint16_t* raw, uint16_t* out, cudaStream_t s) {
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 8;
  const long long nb = (long long)NBx * NBy * NBz;
  cudaError_t e = cudaMemsetAsync(bmax, 0, (size_t)nb * 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const long long threads = nb * 256 * 2;
  long long blocks = (threads + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  pack_raw_kernel<<<(unsigned)blocks, 256, 0, s>>>(f[0], f[1], f[2], f[3], nx, ny, NBx, NBy, nb,
                                                   bmax, raw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (out) {
    normalise_kernel<<<152 * 8, 256, 0, s>>>(raw, bmax, nb, out);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace aew
