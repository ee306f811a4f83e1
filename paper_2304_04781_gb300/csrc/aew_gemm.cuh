// Generic tcgen05 GEMM building block for the codec and its training:
//   D[M][N] = sum_k A(m, k) B(n, k)      (FP32 accumulate in TMEM)
// with pluggable operand loaders (global memory -> canonical K-major shared-memory
// tiles) and epilogues (TMEM -> registers -> fused bias / activation / store).
//
// CTA tile: 128 rows (one TMEM lane per row) x BN columns, K in chunks of 64, two
// shared-memory stages so that the loads of chunk c+1 overlap the MMAs of chunk c.
// One thread issues the MMAs (4 K-steps of 16 per chunk) and commits them to the
// stage's mbarrier; all waits are bounded in time and set an error flag on timeout.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "aew_tc.cuh"

namespace aew {
namespace gemm {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kStages = 2;
constexpr int kThreads = 256;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

// byte offset of element (r, k) of a kBK-wide tile in the canonical layout
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

template <int BN>
constexpr size_t smem_bytes() {
  return (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 128 + 1024;
}

// ---------------------------------------------------------------------------------
// Loader: 16-bit matrix with K contiguous, row r at base + row_off(r).
// ---------------------------------------------------------------------------------
struct RowsLinear {
  long long ld;
  __device__ __forceinline__ long long operator()(long long r) const { return r * ld; }
};

template <class RowFn>
struct LdK16 {
  const uint16_t* p;
  RowFn rows;
  long long R;  // valid rows
  int K;        // valid K (multiple of 8)
  template <int NROWS>
  __device__ __forceinline__ void load(uint8_t* tile, long long r0, int k0, int tid) const {
    const int warp = tid >> 5, lane = tid & 31;
    constexpr int NG = NROWS / 8;                 // row groups of 8
    constexpr int IT = (NG + 7) / 8;              // per warp
    uint4 v[IT][2];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int g = warp + 8 * it;
      const long long gr = r0 + g * 8 + (lane & 7);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + ((lane >> 3) + 4 * h) * 8;
        v[it][h] = make_uint4(0u, 0u, 0u, 0u);
        if (g < NG && gr < R && k < K)
          v[it][h] = __ldg(reinterpret_cast<const uint4*>(p + rows(gr) + k));
      }
    }
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int g = warp + 8 * it;
      if (g < NG) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kc = (lane >> 3) + 4 * h;
          *reinterpret_cast<uint4*>(tile + g * 1024 + kc * 128 + (lane & 7) * 16) = v[it][h];
        }
      }
    }
  }
};

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}
__device__ __forceinline__ uint16_t bf16_bits(float a) {
  __nv_bfloat16 t = __float2bfloat16_rn(a);
  return *reinterpret_cast<uint16_t*>(&t);
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}
__device__ __forceinline__ float gelu_f(float a) {
  return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_prime_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) +
         a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// ---------------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------------
template <int BN, bool BF16, class AL, class BL, class EP>
__global__ void __launch_bounds__(kThreads) gemm_kernel(long long M, int N, int K, AL al, BL bl,
                                                        EP ep, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int A_BYTES = kBM * kBK * 2;
  constexpr int B_BYTES = BN * kBK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  constexpr int NSUB = BN > 256 ? BN / 256 : 1;
  constexpr int NMMA = BN > 256 ? 256 : BN;
  constexpr uint32_t IDESC = tc::idesc_f16(kBM, NMMA, BF16);
  static_assert(BN % 32 == 0 && BN <= 512, "BN");

  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kStages * STAGE);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kStages);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.y * kBM;
  const int n0 = blockIdx.x * BN;

  if (warp == 0) {
    tc::tmem_alloc(tc::smem_u32(tslot), TCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 32) {
    for (int s = 0; s < kStages; ++s) tc::mbar_init(tc::smem_u32(&mbar[s]), 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  const int nK = (K + kBK - 1) / kBK;
  bool ok = true;
  for (int c = 0; c < nK; ++c) {
    const int s = c % kStages;
    uint8_t* sa = smem + s * STAGE;
    uint8_t* sb = sa + A_BYTES;
    if (c >= kStages) ok = tc::mbar_wait(tc::smem_u32(&mbar[s]), ((c / kStages) - 1) & 1, kWaitNs);
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    al.template load<kBM>(sa, m0, c * kBK, tid);
    bl.template load<BN>(sb, n0, c * kBK, tid);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(sa), b0 = tc::smem_u32(sb);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
        for (int h = 0; h < NSUB; ++h) {
          const uint64_t ad = tc::sdesc(a0 + kk * 256, 128, 1024);
          const uint64_t bd = tc::sdesc(b0 + h * (256 / 8) * 1024 + kk * 256, 128, 1024);
          tc::mma_f16(tmem + h * 256, ad, bd, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(tc::smem_u32(&mbar[s]));
    }
  }
  if (ok && nK > 0) {
    const int cl = nK - 1;
    ok = tc::mbar_wait(tc::smem_u32(&mbar[cl % kStages]), (cl / kStages) & 1, kWaitNs);
  }
  ok = !__syncthreads_or(!ok);
  tc::fence_after_sync();
  if (ok) {
    const int q = warp & 3, hh = warp >> 2;
    const long long row = m0 + q * 32 + lane;
    constexpr int CPW = BN >= 64 ? BN / 2 : BN;
    if (BN >= 64 || hh == 0) {
#pragma unroll 1
      for (int cc = 0; cc < CPW; cc += 32) {
        const int col = (BN >= 64 ? hh * (BN / 2) : 0) + cc;
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, v);
        ep(row, n0 + col, v);
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

template <int BN, bool BF16, class AL, class BL, class EP>
cudaError_t launch(long long M, int N, int K, const AL& al, const BL& bl, const EP& ep, int* err,
                   cudaStream_t s) {
  auto kern = gemm_kernel<BN, BF16, AL, BL, EP>;
  const size_t smem = smem_bytes<BN>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const dim3 grid((N + BN - 1) / BN, (unsigned)((M + kBM - 1) / kBM));
  kern<<<grid, kThreads, smem, s>>>(M, N, K, al, bl, ep, err);
  return cudaGetLastError();
}

}  // namespace gemm
}  // namespace aew
