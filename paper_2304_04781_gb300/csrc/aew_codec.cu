// Per-block autoencoder codec on tcgen05 tensor cores (compression in space, Sec. 3.1;
// dense layers sigma(y W + b) of Eq. (5), Sec. 3.3), plus the snapshot packing of
// Algorithm 1.
//
// Block vector of an 8x8x8-node block: k = z*256 + f*64 + y*8 + x (f = e, vx, vy, vz);
// block b = (bz*NBy + by)*NBx + bx.  Each field is divided by its scale s_f (the
// running maximum of |f|).
//
// Encoder: A = normalised block vectors gathered straight from the four FP32 grid
// fields (BF16, RNE), times W1 (2048 x 512) -> +b1, GELU -> H (BF16), times W2
// (512 x n_lat) -> +b2 -> FP16 latent.  Decoder: latent (FP16) times W3 (FP16,
// n_lat x 512) -> +b3, GELU -> H (BF16), times W4 (BF16, 512 x 2048, or only its 512
// strain columns inside the adjoint) -> +b4, times s_e, scattered back to the grid.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <vector>

#include "aew_codec.cuh"
#include "aew_codec_state.cuh"
#include "aew_gemm.cuh"

namespace aew {


namespace {

__global__ void transpose_to16_kernel(const float* __restrict__ src, int rows, int cols,
                                      uint16_t* __restrict__ dst, int fp16) {
  // dst[c][r] = round(src[r][c])
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) {
      const float v = tile[threadIdx.x][i];
      uint16_t b;
      if (fp16) {
        __half hv = __float2half_rn(v);
        b = *reinterpret_cast<uint16_t*>(&hv);
      } else {
        b = gemm::bf16_bits(v);
      }
      dst[(size_t)c * rows + r] = b;
    }
  }
}

cudaError_t transpose16(const float* src, int rows, int cols, uint16_t* dst, bool fp16,
                        cudaStream_t s) {
  dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
  transpose_to16_kernel<<<grid, block, 0, s>>>(src, rows, cols, dst, fp16 ? 1 : 0);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Epilogues
// ---------------------------------------------------------------------------------
// H[row][col..] = bf16(gelu(acc + bias))
struct EpBiasGeluH {
  const float* bias;
  uint16_t* H;
  long long M;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const float a0 = v[j] + __ldg(bias + col + j), a1 = v[j + 1] + __ldg(bias + col + j + 1);
      pk[j / 2] = gemm::pack_bf16(gemm::gelu_f(a0), gemm::gelu_f(a1));
    }
    uint4* dst = reinterpret_cast<uint4*>(H + row * kNHid + col);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
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
    uint32_t pk[16];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const float a0 = v[j] + __ldg(bias + col + j), a1 = v[j + 1] + __ldg(bias + col + j + 1);
      const __half2 hv = __floats2half2_rn(a0, a1);
      bad |= !(fabsf(a0) <= 65504.f) || !(fabsf(a1) <= 65504.f);
      pk[j / 2] = *reinterpret_cast<const uint32_t*>(&hv);
    }
    if (bad) atomicOr(ovf, 1);
    uint4* dst = reinterpret_cast<uint4*>(lat + row * nl + col);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
  }
};

// strain part of the decoder output, scattered to the grid:
// column n = z*64 + y*8 + x of block row -> node (8bz+z, 8by+y, 8bx+x);
// e = (acc + b4[z*256 + y*8 + x]) * s_e, 0 on boundary nodes
struct EpDecGrid {
  const float* b4;
  const float* scale_e;
  float* e;
  int nx, ny, nz, NBx, NBy;
  long long M;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    const float s = __ldg(scale_e);
    const long long bx = row % NBx, t = row / NBx;
    const long long by = t % NBy, bz = t / NBy;
    const int z = col >> 6, y0 = (col & 63) >> 3;
    const int kz = (int)(8 * bz) + z;
    const bool zb = (kz == 0 || kz == nz - 1);
#pragma unroll
    for (int yy = 0; yy < 4; ++yy) {
      const int jy = (int)(8 * by) + y0 + yy;
      const bool yb = zb || jy == 0 || jy == ny - 1;
      float o[8];
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        const int ix = (int)(8 * bx) + x;
        const float bv = __ldg(b4 + z * 256 + (y0 + yy) * 8 + x);
        const float val = (v[yy * 8 + x] + bv) * s;
        o[x] = (yb || ix == 0 || ix == nx - 1) ? 0.f : val;
      }
      float4* dst = reinterpret_cast<float4*>(e + ((size_t)kz * ny + jy) * nx + 8 * bx);
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
#pragma unroll
    for (int q = 0; q < 8; ++q)
      dst[q] = make_float4(v[4 * q] + __ldg(bias + col + 4 * q), v[4 * q + 1] + __ldg(bias + col + 4 * q + 1),
                           v[4 * q + 2] + __ldg(bias + col + 4 * q + 2), v[4 * q + 3] + __ldg(bias + col + 4 * q + 3));
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
  if (cudaMalloc(&c->H, rows * kNHid * sizeof(uint16_t)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->H_rows = rows;
  return true;
}

// ---------------------------------------------------------------------------------
// Algorithm 1 packing: BF16 normalised block vectors
// ---------------------------------------------------------------------------------
__global__ void snapshot_pack_kernel(const float* f0, const float* f1, const float* f2,
                                     const float* f3, int nx, int ny, int NBx, int NBy,
                                     long long nblk, const float* scale, uint16_t* out) {
  // One thread per float4 of a grid row; consecutive threads read consecutive x
  // (coalesced) and write 8-byte pieces of the block vectors.
  const int xq_n = nx >> 2;
  const long long total = nblk / NBx * 256LL * xq_n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int xq = (int)(t % xq_n);
    long long r = t / xq_n;
    const int y = (int)(r & 7), f = (int)((r >> 3) & 3), z = (int)((r >> 5) & 7);
    const long long slab = r >> 8;               // (bz, by)
    const long long by = slab % NBy, bz = slab / NBy;
    const float* src = f == 0 ? f0 : (f == 1 ? f1 : (f == 2 ? f2 : f3));
    const float sc = scale[f];
    // y = x * (1/s): one correctly rounded reciprocal per field, then a product
    const float inv = sc > 0.f ? __frcp_rn(sc) : 0.f;
    const float4 a = *reinterpret_cast<const float4*>(
        src + ((size_t)(8 * bz + z) * ny + (size_t)(8 * by + y)) * nx + 4 * (size_t)xq);
    const float u0 = __fmul_rn(a.x, inv), u1 = __fmul_rn(a.y, inv);
    const float u2 = __fmul_rn(a.z, inv), u3 = __fmul_rn(a.w, inv);
    const long long b = slab * NBx + (xq >> 1);
    *reinterpret_cast<uint2*>(out + b * kNIn + z * 256 + f * 64 + y * 8 + 4 * (xq & 1)) =
        make_uint2(gemm::pack_bf16(u0, u1), gemm::pack_bf16(u2, u3));
  }
}

// strain rows of W4t (vector index z*256 + j, j < 64) packed as W4e [512][512]
__global__ void strain_rows_kernel(const uint16_t* __restrict__ W4t, uint16_t* __restrict__ W4e) {
  const int r = blockIdx.x, k = threadIdx.x;
  const int src = (r >> 6) * 256 + (r & 63);
  for (int q = k; q < kNHid; q += blockDim.x) W4e[(size_t)r * kNHid + q] = W4t[(size_t)src * kNHid + q];
}

__global__ void update_scale_kernel(const float* p, const unsigned* a, float* o) {
  const int i = threadIdx.x;
  float v = p ? p[i] : 0.f;
  if (a) v = fmaxf(v, __uint_as_float(a[i]));
  o[i] = v;
}

}  // namespace

// =================================================================================
namespace gemm {

CUresult make_tmap(CUtensorMap* map, const void* base, bool fp16, long long rows, int K,
                   long long ld, int box_rows, bool swizzle128) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        fn == nullptr || q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return CUDA_ERROR_NOT_FOUND;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
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

Codec* codec_new(int n_lat) {
  Codec* c = new Codec();
  c->n_lat = n_lat;
  const size_t nl = (size_t)n_lat;
  const size_t sz[8] = {(size_t)kNIn * kNHid, kNHid, kNHid * nl, nl, nl * kNHid, kNHid,
                        (size_t)kNHid * kNIn, kNIn};
  bool ok = true;
  for (int i = 0; i < 8 && ok; ++i) {
    c->wn[i] = sz[i];
    ok = cudaMalloc(&c->w[i], sz[i] * sizeof(float)) == cudaSuccess;
    c->bytes += sz[i] * sizeof(float);
  }
  ok = ok && cudaMalloc(&c->W1t, (size_t)kNIn * kNHid * 2) == cudaSuccess &&
       cudaMalloc(&c->W2t, nl * kNHid * 2) == cudaSuccess &&
       cudaMalloc(&c->W3t, nl * kNHid * 2) == cudaSuccess &&
       cudaMalloc(&c->W4t, (size_t)kNIn * kNHid * 2) == cudaSuccess &&
       cudaMalloc(&c->W4e, (size_t)512 * kNHid * 2) == cudaSuccess &&
       cudaMalloc(&c->err, sizeof(int)) == cudaSuccess &&
       cudaMalloc(&c->sc_tmp, 4 * sizeof(float)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    codec_free(c);
    return nullptr;
  }
  cudaMemset(c->err, 0, sizeof(int));
  c->bytes += ((size_t)2 * kNIn * kNHid + 2 * nl * kNHid) * 2;
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
size_t codec_device_bytes(const Codec* c) {
  return c->bytes + c->H_rows * kNHid * 2 + c->X_rows * kNIn * 2 +
         (c->train ? train_state_bytes(c->train) : 0);
}
bool codec_ready(const Codec* c) { return c && c->ready; }

// refresh the tensor-core operand copies from the FP32 masters
cudaError_t codec_refresh(Codec* c, cudaStream_t s) {
  const int nl = c->n_lat;
  cudaError_t e;
  if ((e = transpose16(c->w[0], kNIn, kNHid, c->W1t, false, s)) != cudaSuccess) return e;
  if ((e = transpose16(c->w[2], kNHid, nl, c->W2t, false, s)) != cudaSuccess) return e;
  if ((e = transpose16(c->w[4], nl, kNHid, c->W3t, true, s)) != cudaSuccess) return e;
  if ((e = transpose16(c->w[6], kNHid, kNIn, c->W4t, false, s)) != cudaSuccess) return e;
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

cudaError_t snapshot_pack(const float* const f[4], int nx, int ny, int nz, const float* scale,
                          uint16_t* out, cudaStream_t s);

cudaError_t codec_encode_grid(Codec* c, const float* const f[4], int nx, int ny, int nz,
                              const float* scale_prev, const unsigned* amax, float* scale_out,
                              uint16_t* lat, int* overflow, cudaStream_t s) {
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 8;
  const long long nb = (long long)NBx * NBy * NBz;
  if (!ensure_X(c, (size_t)nb)) return cudaErrorMemoryAllocation;
  // s_f = max(prev, amax): the scales this state is normalised with (kept for decoding)
  float* sc = scale_out ? scale_out : c->sc_tmp;
  update_scale_kernel<<<1, 4, 0, s>>>(scale_prev, amax, sc);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // normalised BF16 block vectors (the packing of Algorithm 1), then the encoder GEMMs
  if ((e = snapshot_pack(f, nx, ny, nz, sc, c->X, s)) != cudaSuccess) return e;
  return codec_encode_vectors(c, c->X, nb, lat, overflow, s);
}

cudaError_t codec_encode_vectors(Codec* c, const uint16_t* vec, long long n, uint16_t* lat,
                                 int* overflow, cudaStream_t s) {
  if (!ensure_H(c, (size_t)n)) return cudaErrorMemoryAllocation;
  EpBiasGeluH ep{c->w[1], c->H, n};
  cudaError_t e = gemm::launch<256, true>(n, kNHid, kNIn, gemm::Mat{vec, n, kNIn},
                                          gemm::Mat{c->W1t, kNHid, kNIn}, ep, c->err, s);
  if (e != cudaSuccess) return e;
  const int nl = c->n_lat;
  EpLatent e2{c->w[3], lat, nl, n, overflow};
  const gemm::Mat a2{c->H, n, kNHid}, b2{c->W2t, nl, kNHid};
  if (nl == 64) return gemm::launch<64, true>(n, nl, kNHid, a2, b2, e2, c->err, s);
  return gemm::launch<32, true>(n, nl, kNHid, a2, b2, e2, c->err, s);
}

static cudaError_t decode_hidden(Codec* c, const uint16_t* lat, long long nb, cudaStream_t s) {
  if (!ensure_H(c, (size_t)nb)) return cudaErrorMemoryAllocation;
  const int nl = c->n_lat;
  EpBiasGeluH ep{c->w[5], c->H, nb};
  return gemm::launch<256, false>(nb, kNHid, nl, gemm::Mat{lat, nb, nl},
                                  gemm::Mat{c->W3t, kNHid, nl}, ep, c->err, s);
}

cudaError_t codec_decode_grid_e(Codec* c, const uint16_t* lat, int nx, int ny, int nz,
                                const float* scale_e, float* e_out, cudaStream_t s) {
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 8;
  const long long nb = (long long)NBx * NBy * NBz;
  cudaError_t e = decode_hidden(c, lat, nb, s);
  if (e != cudaSuccess) return e;
  EpDecGrid ep{c->w[7], scale_e, e_out, nx, ny, nz, NBx, NBy, nb};
  return gemm::launch<256, true>(nb, 512, kNHid, gemm::Mat{c->H, nb, kNHid},
                                 gemm::Mat{c->W4e, 512, kNHid}, ep, c->err, s);
}

cudaError_t codec_decode_vectors(Codec* c, const uint16_t* lat, long long nvec, float* out,
                                 cudaStream_t s) {
  cudaError_t e = decode_hidden(c, lat, nvec, s);
  if (e != cudaSuccess) return e;
  EpVec ep{c->w[7], out, kNIn, nvec};
  return gemm::launch<256, true>(nvec, kNIn, kNHid, gemm::Mat{c->H, nvec, kNHid},
                                 gemm::Mat{c->W4t, kNIn, kNHid}, ep, c->err, s);
}

cudaError_t snapshot_pack(const float* const f[4], int nx, int ny, int nz, const float* scale,
                          uint16_t* out, cudaStream_t s) {
  const int NBx = nx / 8, NBy = ny / 8, NBz = nz / 8;
  const long long nb = (long long)NBx * NBy * NBz;
  const long long threads = nb * 256 * 2;
  long long blocks = (threads + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  snapshot_pack_kernel<<<(unsigned)blocks, 256, 0, s>>>(
      f[0], f[1], f[2], f[3], nx, ny, NBx, NBy, nb, scale, out);
  return cudaGetLastError();
}

}  // namespace aew
