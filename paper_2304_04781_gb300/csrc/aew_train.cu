// Training of the per-block autoencoder (Sec. 3.3, Table 2): mean-squared
// reconstruction error on normalised block vectors, back-propagation through both
// GELU layers with a straight-through FP16 latent, and the LAMB optimiser
// (You et al. 2019) with one trust ratio per parameter tensor.
//
// Every product is a tcgen05 GEMM (aew_gemm.cuh) with BF16 operands and FP32
// accumulation (the decoder's first forward product uses FP16 operands, as in
// inference).  Activations are written both row-major and transposed by the producing
// epilogue, so every weight-gradient product (K = batch) reads K-contiguous operands.
// FP32 master weights; LAMB moments in FP32; norms and the loss in FP64.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <string>

#include "aew_codec.cuh"
#include "aew_codec_state.cuh"
#include "aew_gemm.cuh"

namespace aew {


namespace {

struct TrainState {
  int B = 0;       // batch capacity
  int nl = 64;
  int t = 0;       // LAMB step count
  size_t bytes = 0;
  // activations
  float *a1, *a3, *d1, *d2, *d3, *d4;
  uint16_t *h1, *h1T, *z16, *zbT, *h3, *h3T, *d4b, *d4T, *d3b, *d3T, *d2b, *d2T, *d1T, *YT;
  // gradients and moments (8 tensors)
  float* g[8];
  float* m[8];
  float* v[8];
  // backward weight copies (natural layout, BF16)
  uint16_t *W4b, *W3b, *W2b;
  double* red;  // [0] loss, [1 + 2t], [2 + 2t]: |w|^2, |u|^2 of tensor t
  void* allocs[64];
  int nalloc = 0;
};

template <class T>
bool talloc(TrainState* s, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  s->allocs[s->nalloc++] = q;
  s->bytes += n * sizeof(T);
  *p = static_cast<T*>(q);
  return true;
}

TrainState* train_new(Codec* c, int B) {
  TrainState* s = new TrainState();
  s->B = B;
  s->nl = c->n_lat;
  const size_t b = (size_t)B, nl = (size_t)c->n_lat, H = (size_t)c->n_hid, I = kNIn;
  bool ok = talloc(s, &s->a1, b * H) && talloc(s, &s->a3, b * H) && talloc(s, &s->d1, b * H) &&
            talloc(s, &s->d2, b * nl) && talloc(s, &s->d3, b * H) && talloc(s, &s->d4, b * I) &&
            talloc(s, &s->h1, b * H) && talloc(s, &s->h1T, b * H) && talloc(s, &s->z16, b * nl) &&
            talloc(s, &s->zbT, b * nl) && talloc(s, &s->h3, b * H) && talloc(s, &s->h3T, b * H) &&
            talloc(s, &s->d4b, b * I) && talloc(s, &s->d4T, b * I) && talloc(s, &s->d3b, b * H) &&
            talloc(s, &s->d3T, b * H) && talloc(s, &s->d2b, b * nl) && talloc(s, &s->d2T, b * nl) &&
            talloc(s, &s->d1T, b * H) && talloc(s, &s->YT, b * I) &&
            talloc(s, &s->W4b, H * I) && talloc(s, &s->W3b, nl * H) && talloc(s, &s->W2b, H * nl) &&
            talloc(s, &s->red, 32);
  for (int i = 0; i < 8 && ok; ++i)
    ok = talloc(s, &s->g[i], c->wn[i]) && talloc(s, &s->m[i], c->wn[i]) &&
         talloc(s, &s->v[i], c->wn[i]);
  if (!ok) {
    for (int i = 0; i < s->nalloc; ++i) cudaFree(s->allocs[i]);
    delete s;
    return nullptr;
  }
  for (int i = 0; i < 8; ++i) {
    cudaMemset(s->m[i], 0, c->wn[i] * sizeof(float));
    cudaMemset(s->v[i], 0, c->wn[i] * sizeof(float));
  }
  return s;
}

// ---------------------------------------------------------------------------------
// Epilogues
// ---------------------------------------------------------------------------------
// 32 16-bit values of one row, as two 32-byte stores (dst 32-byte aligned: every row
// length here is a multiple of 16 values and every column group starts at a multiple of
// 32), so each store fills whole sectors
__device__ __forceinline__ void store_row16(uint16_t* dst, const uint32_t (&pk)[16]) {
  gemm::st_global_32B(dst, pk[0], pk[1], pk[2], pk[3], pk[4], pk[5], pk[6], pk[7]);
  gemm::st_global_32B(dst + 16, pk[8], pk[9], pk[10], pk[11], pk[12], pk[13], pk[14], pk[15]);
}

// 32 FP32 values of one row as four 32-byte stores (dst 32-byte aligned: every row length
// here is a multiple of 8 values and every column group starts at a multiple of 32)
__device__ __forceinline__ void store_row32f(float* dst, const float (&x)[32]) {
#pragma unroll
  for (int j = 0; j < 32; j += 8)
    gemm::st_global_32B(dst + j, __float_as_uint(x[j]), __float_as_uint(x[j + 1]),
                        __float_as_uint(x[j + 2]), __float_as_uint(x[j + 3]),
                        __float_as_uint(x[j + 4]), __float_as_uint(x[j + 5]),
                        __float_as_uint(x[j + 6]), __float_as_uint(x[j + 7]));
}

// the training kernels' activation and its derivative: GELU by erff (act 0) or ELU
// (act 1: e^a - 1 below 0, a above; derivative e^a below 0, 1 above)
__device__ __forceinline__ float act_f(int act, float a) {
  return act == 1 ? (a > 0.f ? a : expm1f(a)) : gemm::gelu_f(a);
}
__device__ __forceinline__ float act_prime_f(int act, float a) {
  return act == 1 ? (a > 0.f ? 1.f : expf(a)) : gemm::gelu_prime_f(a);
}

// a = acc + bias -> pre (FP32), h = bf16(act(a)) row-major and transposed
struct EpFwdGelu {
  const float* bias;
  float* pre;
  uint16_t* h;
  uint16_t* hT;
  int N;
  long long M;
  int act;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M) return;
    uint32_t pk[16];
    float* pd = pre + row * N + col;   // 32-byte aligned: N and col multiples of 32
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
      float a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = v[j + q] + __ldg(bias + col + j + q);
      gemm::st_global_32B(pd + j, __float_as_uint(a[0]), __float_as_uint(a[1]),
                          __float_as_uint(a[2]), __float_as_uint(a[3]), __float_as_uint(a[4]),
                          __float_as_uint(a[5]), __float_as_uint(a[6]), __float_as_uint(a[7]));
#pragma unroll
      for (int q = 0; q < 8; q += 4) {
        const float g0 = act_f(act, a[q]), g1 = act_f(act, a[q + 1]);
        const float g2 = act_f(act, a[q + 2]), g3 = act_f(act, a[q + 3]);
        pk[(j + q) / 2] = gemm::pack_bf16(g0, g1);
        pk[(j + q) / 2 + 1] = gemm::pack_bf16(g2, g3);
        hT[(size_t)(col + j + q + 0) * M + row] = gemm::bf16_bits(g0);
        hT[(size_t)(col + j + q + 1) * M + row] = gemm::bf16_bits(g1);
        hT[(size_t)(col + j + q + 2) * M + row] = gemm::bf16_bits(g2);
        hT[(size_t)(col + j + q + 3) * M + row] = gemm::bf16_bits(g3);
      }
    }
    store_row16(h + row * N + col, pk);
  }
};

// latent: z = fp16(acc + b2) row-major; bf16(z) transposed for dW3
struct EpFwdLatent {
  const float* bias;
  uint16_t* z16;
  uint16_t* zbT;
  int nl;
  long long M;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M || col >= nl) return;
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 32; j += 2) {
      const __half2 hv = __floats2half2_rn(v[j] + __ldg(bias + col + j), v[j + 1] + __ldg(bias + col + j + 1));
      pk[j / 2] = *reinterpret_cast<const uint32_t*>(&hv);
      zbT[(size_t)(col + j) * M + row] = gemm::bf16_bits(__low2float(hv));
      zbT[(size_t)(col + j + 1) * M + row] = gemm::bf16_bits(__high2float(hv));
    }
    store_row16(z16 + row * nl + col, pk);
  }
};

// reconstruction: a4 = acc + b4; diff = a4 - y; d4 = 2 diff / (B*2048)
struct EpMse {
  const float* bias;
  const uint16_t* Y;
  const float* w;    // [M][4] weight of each vector's fields (null: all ones)
  float* d4;
  uint16_t* d4b;
  uint16_t* d4T;
  double* loss;
  float scale;
  long long M;
  // called by all 32 lanes of a warp together (rows m0 + 32 q + lane): the loss is
  // reduced across the warp before its one atomic
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    double acc = 0.0;
    if (row < M) {
      // the 32 columns lie in one field's 64-column group: one weight
      const float wf = w ? __ldg(w + row * 4 + ((col >> 6) & 3)) : 1.f;
      uint32_t pk[16];
      float dd[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float a = v[j] + __ldg(bias + col + j);
        const float diff = a - gemm::bf16_val(__ldg(Y + row * kNIn + col + j));
        acc += (double)wf * (double)diff * (double)diff;
        dd[j] = scale * wf * diff;
        d4T[(size_t)(col + j) * M + row] = gemm::bf16_bits(dd[j]);
      }
#pragma unroll
      for (int j = 0; j < 32; j += 2) pk[j / 2] = gemm::pack_bf16(dd[j], dd[j + 1]);
      store_row32f(d4 + row * kNIn + col, dd);
      store_row16(d4b + row * kNIn + col, pk);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
  }
};

// backward through an activation: d = acc * act'(pre) (or d = acc), stored FP32,
// BF16 row-major (optional) and BF16 transposed
struct EpBack {
  const float* pre;  // null: straight-through
  float* d;
  uint16_t* db;
  uint16_t* dT;
  int N;
  long long M;
  int act;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M || col >= N) return;
    float dd[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      dd[j] = pre ? v[j] * act_prime_f(act, pre[row * N + col + j]) : v[j];
      dT[(size_t)(col + j) * M + row] = gemm::bf16_bits(dd[j]);
    }
    store_row32f(d + row * N + col, dd);
    if (db) {
      uint32_t pk[16];
#pragma unroll
      for (int j = 0; j < 32; j += 2) pk[j / 2] = gemm::pack_bf16(dd[j], dd[j + 1]);
      store_row16(db + row * N + col, pk);
    }
  }
};

// weight gradient: G[row][col..] = acc (FP32)
struct EpStore {
  float* G;
  int N;
  long long M;
  __device__ __forceinline__ void operator()(long long row, int col, const float (&v)[32]) const {
    if (row >= M || col >= N) return;
    store_row32f(G + row * N + col, v);
  }
};

// ---------------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------------
__global__ void transpose16_kernel(const uint16_t* __restrict__ src, int rows, int cols,
                                   uint16_t* __restrict__ dst) {
  __shared__ uint16_t tile[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * cols + c] : (uint16_t)0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[(size_t)c * rows + r] = tile[threadIdx.x][i];
  }
}

// bias gradients: the column sums of up to four [rows][cols] FP32 matrices in one
// launch.  A block takes 32 columns of one matrix: lane = column (coalesced rows), the 8
// warps split the rows; each thread keeps four FP32 partial sums (a batch of 512 rows
// gives each 16 terms), combined in FP64 in a fixed order.
struct ColSums {
  const float* d[4];
  float* out[4];
  int cols[4];
  int tiles[5];   // prefix of 32-column tiles per matrix
  int n;
};
__global__ void colsum_multi_kernel(ColSums cs, int rows) {
  __shared__ double part[8][33];
  int m = 0;
  while (m + 1 < cs.n && (int)blockIdx.x >= cs.tiles[m + 1]) ++m;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int c = (blockIdx.x - cs.tiles[m]) * 32 + lane;
  const int cols = cs.cols[m];
  // four independent FP32 partial sums per thread (a warp's rows r = wq + 8 t), then FP64
  float a4[4] = {0.f, 0.f, 0.f, 0.f};
  if (c < cols) {
    int t = 0;
    for (int r = wq; r < rows; r += 8, ++t) a4[t & 3] += cs.d[m][(size_t)r * cols + c];
  }
  part[wq][lane] = ((double)a4[0] + (double)a4[1]) + ((double)a4[2] + (double)a4[3]);
  __syncthreads();
  if (wq == 0 && c < cols) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += part[q][lane];
    cs.out[m][c] = (float)t;
  }
}

// BF16 copies of up to three FP32 tensors in one launch (blockIdx.y = tensor)
struct ToBf16 {
  const float* w[3];
  uint16_t* o[3];
  size_t n[3];
};
__global__ void to_bf16_multi_kernel(ToBf16 t) {
  // four elements per thread (every size is a multiple of 4)
  const float4* w = reinterpret_cast<const float4*>(t.w[blockIdx.y]);
  uint2* o = reinterpret_cast<uint2*>(t.o[blockIdx.y]);
  const size_t n4 = t.n[blockIdx.y] / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    const float4 v = w[i];
    o[i] = make_uint2(gemm::pack_bf16(v.x, v.y), gemm::pack_bf16(v.z, v.w));
  }
}

__global__ void loss_kernel(const double* red, double inv_n, float* out, double* acc) {
  const double l = red[0] * inv_n;
  if (out) out[0] = (float)l;
  if (acc) acc[0] += l;
}

// ---------------------------------------------------------------------------------
// Epoch driver pieces: seeded shuffle, minibatch gather, loss weights
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom number
  // generators", OOPSLA 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}
// A seeded bijection of [0, n): a balanced four-round Feistel network on 2 hb bits
// (2^(2 hb) >= n), walked until it lands inside [0, n) (a bijection on the larger
// domain restricted by cycle walking stays a bijection).
__device__ __forceinline__ long long shuffle_index(long long i, long long n, int hb, uint64_t key) {
  const uint64_t mask = (1ull << hb) - 1;
  uint64_t x = (uint64_t)i;
  do {
    uint64_t L = x >> hb, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const uint64_t F = mix64(key ^ (R * 0x100000001b3ull) ^ ((uint64_t)r << 56)) & mask;
      const uint64_t nL = R;
      R = L ^ F;
      L = nL;
    }
    x = (L << hb) | R;
  } while (x >= (uint64_t)n);
  return (long long)x;
}

// minibatch b of an epoch: rows i0 .. i0 + B of the shuffled order, one warp per row
__global__ void gather_kernel(const uint16_t* __restrict__ Y, const float* __restrict__ wts,
                              long long n, int hb, uint64_t key, long long i0, int B,
                              uint16_t* __restrict__ out, float* __restrict__ wout) {
  const int lane = threadIdx.x & 31;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < B;
       r += (gridDim.x * blockDim.x) >> 5) {
    const long long src = shuffle_index(i0 + r, n, hb, key);
    const uint4* a = reinterpret_cast<const uint4*>(Y + (size_t)src * kNIn);
    uint4* o = reinterpret_cast<uint4*>(out + (size_t)r * kNIn);
#pragma unroll
    for (int q = 0; q < kNIn / 8 / 32; ++q) o[q * 32 + lane] = a[q * 32 + lane];
    if (wts && lane < 4) wout[(size_t)r * 4 + lane] = wts[(size_t)src * 4 + lane];
  }
}

// a_v of the loss weights from the data set's maxima (space codec: block maxima [n][4],
// strain in column 0; time codec: vector maxima [n]): the power-of-two scale s (pw = 1)
// or s^2 (pw = 2); per-block FP64 partial sums for the mean
__global__ void weight_terms_kernel(const float* __restrict__ mx, int stride, long long n, int pw,
                                    double* __restrict__ a, double* __restrict__ part) {
  __shared__ double sh[256];
  double sum = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const double sc = (double)gemm::block_scale(mx[(size_t)v * stride]);
    const double t = pw == 1 ? sc : sc * sc;
    a[v] = t;
    sum += t;
  }
  sh[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// w[v][f] = a_v / mean(a) for the fields f < nf (the others 0)
__global__ void weight_write_kernel(const double* __restrict__ a, const double* __restrict__ part,
                                    int nblk, long long n, int nf, float* __restrict__ w) {
  double tot = 0.0;
  for (int b = 0; b < nblk; ++b) tot += part[b];
  const double inv = tot > 0 ? (double)n / tot : 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x) {
    const float x = (float)(a[v] * inv);
#pragma unroll
    for (int f = 0; f < 4; ++f) w[(size_t)v * 4 + f] = f < nf ? x : 0.f;
  }
}

// strain columns only (space codec): w[v] = (1, 0, 0, 0)
__global__ void weight_strain_kernel(long long n, float* __restrict__ w) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
       v += (long long)gridDim.x * blockDim.x)
    reinterpret_cast<float4*>(w)[v] = make_float4(1.f, 0.f, 0.f, 0.f);
}

// LAMB over all eight parameter tensors in two launches.  Blocks are dealt to the
// tensors in proportion to their sizes (prefix blk[]); a block reduces its norms in
// shared memory and adds them with one FP64 atomic per tensor and norm.
struct LambArgs {
  float* w[8];
  float* g[8];
  float* m[8];
  float* v[8];
  size_t n[8];
  int blk[9];
};
__device__ __forceinline__ int lamb_tensor(const LambArgs& a) {
  int t = 0;
  while (t < 7 && (int)blockIdx.x >= a.blk[t + 1]) ++t;
  return t;
}
__device__ __forceinline__ void block_add2(double x, double y, double* dst) {
  __shared__ double sx[8], sy[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sx[threadIdx.x >> 5] = x;
    sy[threadIdx.x >> 5] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      a += sx[q];
      b += sy[q];
    }
    atomicAdd(dst, a);
    atomicAdd(dst + 1, b);
  }
}

// pass 1: moments, u (written over g), norms |w|^2 and |u|^2 into norms[2 t], [2 t + 1]
__global__ void lamb1_multi_kernel(LambArgs a, float b1, float b2, float c1, float c2, float eps,
                                   double* norms) {
  const int t = lamb_tensor(a);
  const size_t n4 = a.n[t] / 4;
  const int nb = a.blk[t + 1] - a.blk[t];
  float4* w = reinterpret_cast<float4*>(a.w[t]);
  float4* g = reinterpret_cast<float4*>(a.g[t]);
  float4* m = reinterpret_cast<float4*>(a.m[t]);
  float4* v = reinterpret_cast<float4*>(a.v[t]);
  float sw = 0.f, su = 0.f;   // a thread's few terms in FP32; blocks and tensors in FP64
  for (size_t i = (size_t)(blockIdx.x - a.blk[t]) * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)nb * blockDim.x) {
    const float4 gi = g[i], mi0 = m[i], vi0 = v[i], wi = w[i];
    float gg[4] = {gi.x, gi.y, gi.z, gi.w}, mm[4] = {mi0.x, mi0.y, mi0.z, mi0.w};
    float vv[4] = {vi0.x, vi0.y, vi0.z, vi0.w}, ww[4] = {wi.x, wi.y, wi.z, wi.w}, uu[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      mm[q] = b1 * mm[q] + (1.f - b1) * gg[q];
      vv[q] = b2 * vv[q] + (1.f - b2) * gg[q] * gg[q];
      uu[q] = (mm[q] / c1) / (sqrtf(vv[q] / c2) + eps);
      sw = fmaf(ww[q], ww[q], sw);
      su = fmaf(uu[q], uu[q], su);
    }
    m[i] = make_float4(mm[0], mm[1], mm[2], mm[3]);
    v[i] = make_float4(vv[0], vv[1], vv[2], vv[3]);
    g[i] = make_float4(uu[0], uu[1], uu[2], uu[3]);
  }
  block_add2((double)sw, (double)su, norms + 2 * t);
}

// pass 2: w -= lr * (|w| / |u|) * u
__global__ void lamb2_multi_kernel(LambArgs a, float lr, const double* norms) {
  const int t = lamb_tensor(a);
  const size_t n4 = a.n[t] / 4;
  const int nb = a.blk[t + 1] - a.blk[t];
  const double wn = sqrt(norms[2 * t]), un = sqrt(norms[2 * t + 1]);
  const float r = (wn > 0.0 && un > 0.0) ? (float)(wn / un) : 1.f;
  float4* w = reinterpret_cast<float4*>(a.w[t]);
  const float4* u = reinterpret_cast<const float4*>(a.g[t]);
  for (size_t i = (size_t)(blockIdx.x - a.blk[t]) * blockDim.x + threadIdx.x; i < n4;
       i += (size_t)nb * blockDim.x) {
    float4 x = w[i];
    const float4 y = u[i];
    x.x -= lr * r * y.x;
    x.y -= lr * r * y.y;
    x.z -= lr * r * y.z;
    x.w -= lr * r * y.w;
    w[i] = x;
  }
}

int nblk(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 1216) b = 1216;
  return b < 1 ? 1 : (int)b;
}

gemm::Mat ld(const uint16_t* p, long long ldim, long long rows, int K) {
  (void)K;
  return gemm::Mat{p, rows, ldim};
}

#define TCK(x)                              \
  do {                                      \
    cudaError_t _e = (x);                   \
    if (_e != cudaSuccess) return _e;       \
  } while (0)

// a GEMM whose N is the latent width (32, 64, 256 or 512): the narrowest fitting tile
template <bool BF16, class EP>
cudaError_t launch_nl(long long M, int N, int K, const gemm::Mat& A, const gemm::Mat& B,
                      const EP& ep, int* err, cudaStream_t st) {
  if (N <= 32) return gemm::launch<32, BF16>(M, N, K, A, B, ep, err, st);
  if (N <= 64) return gemm::launch<64, BF16>(M, N, K, A, B, ep, err, st);
  return gemm::launch<256, BF16>(M, N, K, A, B, ep, err, st);
}

// a training GEMM (M rows of the batch or of a weight): the widest tile that still gives
// every SM a tile, since one batch's products are too small to fill the GPU with
// 128 x 256 tiles (AEW_TRAIN_BN = 64, 128 or 256 forces a width: tuning override)
template <bool BF16, class EP>
cudaError_t launch_t(long long M, int N, int K, const gemm::Mat& A, const gemm::Mat& B,
                     const EP& ep, int* err, cudaStream_t st) {
  static const int forced = [] {
    const char* env = getenv("AEW_TRAIN_BN");   // tuning override
    return env ? atoi(env) : 0;
  }();
  const long long mt = (M + 127) / 128;
  const int sms = gemm::sm_count();
  int bn = forced;
  if (bn != 64 && bn != 128 && bn != 256) {
    if (N < 128 || mt * ((N + 255) / 256) >= sms) bn = 256;
    else if (mt * ((N + 127) / 128) >= sms || N < 256) bn = 128;
    else bn = 64;
  }
  if (N <= 64) return launch_nl<BF16>(M, N, K, A, B, ep, err, st);
  if (bn == 64) return gemm::launch<64, BF16>(M, N, K, A, B, ep, err, st);
  if (bn == 128) return gemm::launch<128, BF16>(M, N, K, A, B, ep, err, st);
  return gemm::launch<256, BF16>(M, N, K, A, B, ep, err, st);
}

}  // namespace

void train_state_free(void* t) {
  TrainState* s = static_cast<TrainState*>(t);
  if (!s) return;
  for (int i = 0; i < s->nalloc; ++i) cudaFree(s->allocs[i]);
  delete s;
}
size_t train_state_bytes(const void* t) { return t ? static_cast<const TrainState*>(t)->bytes : 0; }

cudaError_t codec_train_step(Codec* c, const uint16_t* Y, const float* wts, int B, float lr,
                             float* loss_dev, cudaStream_t st, std::string* err, double* loss_acc) {
  if (B % 8 != 0) {
    if (err) *err = "batch must be a multiple of 8";
    return cudaErrorInvalidValue;
  }
  TrainState* s = static_cast<TrainState*>(c->train);
  if (!s || s->B < B) {
    if (s) train_state_free(s);
    c->train = nullptr;
    s = train_new(c, B);
    if (!s) return cudaErrorMemoryAllocation;
    c->train = s;
  }
  const int nl = c->n_lat;
  const long long Bm = B;
  const int H = c->n_hid, I = kNIn;
  int* e = c->err;
  TCK(cudaMemsetAsync(s->red, 0, 32 * sizeof(double), st));
  // backward weight copies of the current masters
  {
    const ToBf16 tb{{c->w[6], c->w[4], c->w[2]}, {s->W4b, s->W3b, s->W2b},
                    {(size_t)H * I, (size_t)nl * H, (size_t)H * nl}};
    to_bf16_multi_kernel<<<dim3(nblk((size_t)H * I / 4), 3), 256, 0, st>>>(tb);
    TCK(cudaGetLastError());
  }
  {
    dim3 grid((I + 31) / 32, (B + 31) / 32), block(32, 8);
    transpose16_kernel<<<grid, block, 0, st>>>(Y, B, I, s->YT);
    TCK(cudaGetLastError());
  }
  // ---- forward
  TCK((launch_t<true>(Bm, H, I, ld(Y, I, Bm, I), ld(c->W1t, I, H, I),
                               EpFwdGelu{c->w[1], s->a1, s->h1, s->h1T, H, Bm, c->act}, e, st)));
  TCK((launch_t<true>(Bm, nl, H, ld(s->h1, H, Bm, H), ld(c->W2t, H, nl, H),
                       EpFwdLatent{c->w[3], s->z16, s->zbT, nl, Bm}, e, st)));
  TCK((launch_t<false>(Bm, H, nl, ld(s->z16, nl, Bm, nl), ld(c->W3t, nl, H, nl),
                                EpFwdGelu{c->w[5], s->a3, s->h3, s->h3T, H, Bm, c->act}, e, st)));
  TCK((launch_t<true>(Bm, I, H, ld(s->h3, H, Bm, H), ld(c->W4t, H, I, H),
                               EpMse{c->w[7], Y, wts, s->d4, s->d4b, s->d4T, s->red,
                                     2.0f / (float)((double)B * I), Bm},
                               e, st)));
  // ---- backward
  TCK((launch_t<true>((long long)H, I, B, ld(s->h3T, B, H, B), ld(s->d4T, B, I, B),
                               EpStore{s->g[6], I, H}, e, st)));
  TCK((launch_t<true>(Bm, H, I, ld(s->d4b, I, Bm, I), ld(s->W4b, I, H, I),
                               EpBack{s->a3, s->d3, s->d3b, s->d3T, H, Bm, c->act}, e, st)));
  TCK((launch_t<true>((long long)nl, H, B, ld(s->zbT, B, nl, B), ld(s->d3T, B, H, B),
                               EpStore{s->g[4], H, nl}, e, st)));
  TCK((launch_t<true>(Bm, nl, H, ld(s->d3b, H, Bm, H), ld(s->W3b, H, nl, H),
                       EpBack{nullptr, s->d2, s->d2b, s->d2T, nl, Bm, c->act}, e, st)));
  TCK((launch_t<true>((long long)H, nl, B, ld(s->h1T, B, H, B), ld(s->d2T, B, nl, B),
                       EpStore{s->g[2], nl, H}, e, st)));
  TCK((launch_t<true>(Bm, H, nl, ld(s->d2b, nl, Bm, nl), ld(s->W2b, nl, H, nl),
                               EpBack{s->a1, s->d1, nullptr, s->d1T, H, Bm, c->act}, e, st)));
  TCK((launch_t<true>((long long)I, H, B, ld(s->YT, B, I, B), ld(s->d1T, B, H, B),
                               EpStore{s->g[0], H, I}, e, st)));
  // bias gradients
  {
    ColSums cs{{s->d1, s->d2, s->d3, s->d4}, {s->g[1], s->g[3], s->g[5], s->g[7]}, {H, nl, H, I},
               {0, 0, 0, 0, 0}, 4};
    for (int q = 0; q < 4; ++q) cs.tiles[q + 1] = cs.tiles[q] + (cs.cols[q] + 31) / 32;
    colsum_multi_kernel<<<cs.tiles[4], 256, 0, st>>>(cs, B);
    TCK(cudaGetLastError());
  }
  if (loss_dev || loss_acc) {
    loss_kernel<<<1, 1, 0, st>>>(s->red, 1.0 / ((double)B * I), loss_dev, loss_acc);
    TCK(cudaGetLastError());
  }
  // ---- LAMB
  s->t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-6f;
  const float c1 = (float)(1.0 - std::pow(0.9, s->t)), c2 = (float)(1.0 - std::pow(0.999, s->t));
  LambArgs la{};
  size_t total = 0;
  for (int i = 0; i < 8; ++i) {
    la.w[i] = c->w[i];
    la.g[i] = s->g[i];
    la.m[i] = s->m[i];
    la.v[i] = s->v[i];
    la.n[i] = c->wn[i];
    if (c->wn[i] % 4) return cudaErrorInvalidValue;   // float4 passes
    total += c->wn[i];
  }
  constexpr int kLambBlocks = 152 * 4;
  la.blk[0] = 0;
  for (int i = 0; i < 8; ++i) {
    const int b = (int)std::max<size_t>(1, (size_t)((double)kLambBlocks * c->wn[i] / total + 0.5));
    la.blk[i + 1] = la.blk[i] + b;
  }
  lamb1_multi_kernel<<<la.blk[8], 256, 0, st>>>(la, b1, b2, c1, c2, eps, s->red + 1);
  TCK(cudaGetLastError());
  lamb2_multi_kernel<<<la.blk[8], 256, 0, st>>>(la, lr, s->red + 1);
  TCK(cudaGetLastError());
  return codec_refresh(c, st);
}

cudaError_t codec_train(Codec* c, const uint16_t* Y, const float* maxima, long long n,
                        const TrainCfg& cfg, double* epoch_loss, cudaStream_t st,
                        std::string* err) {
  const int B = cfg.batch;
  if (B < 8 || B % 8 != 0 || n < B || cfg.epochs < 0) {
    if (err) *err = "batch must be a multiple of 8 and at most the number of vectors";
    return cudaErrorInvalidValue;
  }
  if (cfg.loss != kLossState && cfg.loss != kLossStrain && !maxima) {
    if (err) *err = "amplitude-weighted losses need the vectors' maxima";
    return cudaErrorInvalidValue;
  }
  if (cfg.loss != kLossState && cfg.loss != kLossStrain && c->norm == 1) {
    if (err) *err = "min-max normalisation trains with the plain losses only";
    return cudaErrorInvalidValue;
  }
  // loss weights [n][4] (none for the plain error, or the strain columns of the time codec)
  const bool need_w = !(cfg.loss == kLossState || (cfg.loss == kLossStrain && c->time));
  float* W = nullptr;
  double* a = nullptr;
  double* part = nullptr;
  uint16_t* mb = nullptr;
  float* mw = nullptr;
  double* lacc = nullptr;
  constexpr int kWB = 512;
  cudaError_t e = cudaMalloc(&mb, (size_t)B * kNIn * sizeof(uint16_t));
  if (e == cudaSuccess) e = cudaMalloc(&lacc, sizeof(double));
  if (e == cudaSuccess && need_w) {
    e = cudaMalloc(&W, (size_t)n * 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&mw, (size_t)B * 4 * sizeof(float));
    if (e == cudaSuccess && cfg.loss == kLossStrain) {
      weight_strain_kernel<<<nblk((size_t)n), 256, 0, st>>>(n, W);
      e = cudaGetLastError();
    } else if (e == cudaSuccess) {
      e = cudaMalloc(&a, (size_t)n * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&part, kWB * sizeof(double));
      const int pw = cfg.loss == kLossStrainAmplitude ? 1 : 2;
      if (e == cudaSuccess) {
        weight_terms_kernel<<<kWB, 256, 0, st>>>(maxima, c->time ? 1 : 4, n, pw, a, part);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) {
        weight_write_kernel<<<nblk((size_t)n), 256, 0, st>>>(a, part, kWB, n, c->time ? 4 : 1, W);
        e = cudaGetLastError();
      }
    }
  }
  int hb = 1;
  while ((1ll << (2 * hb)) < n) ++hb;
  const long long nb = n / B;
  for (int ep = 0; ep < cfg.epochs && e == cudaSuccess; ++ep) {
    const float lr = (float)(cfg.lr0 * std::pow(0.5, ep / (cfg.halve_every > 0 ? cfg.halve_every : 1 << 30)));
    const uint64_t key = cfg.seed * 0x9e3779b97f4a7c15ull + (uint64_t)ep * 0xd1b54a32d192ed03ull + 1;
    e = cudaMemsetAsync(lacc, 0, sizeof(double), st);
    for (long long b = 0; b < nb && e == cudaSuccess; ++b) {
      gather_kernel<<<(B + 7) / 8, 256, 0, st>>>(Y, W, n, hb, key, b * B, B, mb, mw);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = codec_train_step(c, mb, W ? mw : nullptr, B, lr, nullptr, st, err, lacc);
    }
    if (e == cudaSuccess && epoch_loss) {
      double l = 0.0;
      e = cudaMemcpyAsync(&l, lacc, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      epoch_loss[ep] = nb > 0 ? l / (double)nb : 0.0;
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  cudaFree(mb);
  cudaFree(mw);
  cudaFree(W);
  cudaFree(a);
  cudaFree(part);
  cudaFree(lacc);
  return e;
}

}  // namespace aew
