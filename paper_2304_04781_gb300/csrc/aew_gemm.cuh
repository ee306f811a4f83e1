// Generic tcgen05 GEMM building block for the codec and its training:
//   D[M][N] = sum_k A(m, k) B(n, k)      (FP32 accumulate in TMEM)
// A and B are 16-bit (BF16 or FP16) matrices with K contiguous in global memory,
// D goes through a pluggable epilogue (TMEM -> registers -> fused bias / activation /
// store).
//
// CTA tile: 128 rows (one TMEM lane per row) x BN columns, K in chunks of 64 through a
// ring of `ns` shared-memory stages.  Warp-specialised:
//   warps 0-3  producers: cp.async (16-byte, zero-filling) of the A and B chunks into
//              the canonical K-major layout, then the epilogue;
//   warp 4     TMEM allocation and, on one lane, the MMA issue loop;
// synchronised by mbarriers: full[s] (128 producer arrivals once chunk data has landed
// and been made visible to the async proxy) and empty[s] (tcgen05.commit once the MMAs
// reading stage s are done).  Every wait is bounded in time; on timeout the kernel
// drains its own copies, sets an error flag and returns.
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
constexpr int kProducers = 128;
constexpr int kThreads = 160;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s
constexpr int kSmemBudget = 200 * 1024;

template <int BN>
__host__ __device__ constexpr int stage_bytes() {
  return kBM * kBK * 2 + BN * kBK * 2;
}
template <int BN>
__host__ __device__ constexpr int max_stages() {
  return kSmemBudget / stage_bytes<BN>() > 8 ? 8 : kSmemBudget / stage_bytes<BN>();
}
inline size_t smem_bytes_for(int stage_b, int ns) { return (size_t)ns * stage_b + 256 + 1024; }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// ---------------------------------------------------------------------------------
// Operand: 16-bit matrix with K contiguous, row r at base + row_off(r).
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
  // issue the cp.async copies of one NROWS x 64 chunk (t = producer thread 0..127)
  template <int NROWS>
  __device__ __forceinline__ void issue(uint8_t* tile, long long r0, int k0, int t) const {
    const int warp = t >> 5, lane = t & 31;
    constexpr int NG = NROWS / 8;
    const uint32_t base = tc::smem_u32(tile) + (lane & 7) * 16;
#pragma unroll
    for (int g = warp; g < NG; g += 4) {
      const long long gr = r0 + g * 8 + (lane & 7);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kc = (lane >> 3) + 4 * h;
        const int k = k0 + kc * 8;
        const bool ok = gr < R && k < K;
        const uint16_t* src = ok ? p + rows(gr) + k : p;
        cp_async16(base + g * 1024 + kc * 128, src, ok ? 16u : 0u);
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
__global__ void __launch_bounds__(kThreads) gemm_kernel(long long M, int N, int K, int ns, AL al,
                                                        BL bl, EP ep, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int A_BYTES = kBM * kBK * 2;
  constexpr int STAGE = stage_bytes<BN>();
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  constexpr int NSUB = BN > 256 ? BN / 256 : 1;
  constexpr int NMMA = BN > 256 ? 256 : BN;
  constexpr uint32_t IDESC = tc::idesc_f16(kBM, NMMA, BF16);
  static_assert(BN % 32 == 0 && BN <= 512, "BN");

  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ns * STAGE);
  uint64_t* empty = full + ns;
  uint64_t* done = empty + ns;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long m0 = (long long)blockIdx.y * kBM;
  const int n0 = blockIdx.x * BN;
  const int nK = (K + kBK - 1) / kBK;

  if (warp == 4) {
    tc::tmem_alloc(tc::smem_u32(tslot), TCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < ns; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), kProducers);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(done), 1);
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp < 4) {
    // ------------------------------------------------------------- producers
    const int D = ns >= 3 ? 2 : ns - 1;   // chunks kept in flight beyond the newest
    int c = 0;
    for (; c < nK; ++c) {
      const int s = c % ns;
      if (c >= ns && !tc::mbar_wait(tc::smem_u32(&empty[s]), ((c / ns) - 1) & 1, kWaitNs)) {
        atomicExch(abort_flag, 1);
        break;
      }
      if (*reinterpret_cast<volatile int*>(abort_flag)) break;
      uint8_t* sa = smem + s * STAGE;
      al.template issue<kBM>(sa, m0, c * kBK, tid);
      bl.template issue<BN>(sa + A_BYTES, n0, c * kBK, tid);
      cp_async_commit();
      if (c >= D) {
        if (D == 2) cp_async_wait<2>();
        else if (D == 1) cp_async_wait<1>();
        else cp_async_wait<0>();
        tc::fence_proxy_async();
        mbar_arrive(tc::smem_u32(&full[(c - D) % ns]));
      }
    }
    cp_async_wait<0>();
    tc::fence_proxy_async();
    if (c == nK) {
      for (int q = (nK - D > 0 ? nK - D : 0); q < nK; ++q) mbar_arrive(tc::smem_u32(&full[q % ns]));
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------- MMA issuer
    bool ok = true;
    for (int c = 0; c < nK; ++c) {
      const int s = c % ns;
      if (!tc::mbar_wait(tc::smem_u32(&full[s]), (c / ns) & 1, kWaitNs)) {
        atomicExch(abort_flag, 1);
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
        for (int h = 0; h < NSUB; ++h) {
          const uint64_t ad = tc::sdesc(a0 + kk * 256, 128, 1024);
          const uint64_t bd = tc::sdesc(b0 + h * (256 / 8) * 1024 + kk * 256, 128, 1024);
          tc::mma_f16(tmem + h * 256, ad, bd, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
        }
      }
      tc::mma_commit(tc::smem_u32(&empty[s]));
    }
    if (ok) tc::mma_commit(tc::smem_u32(done));
  }

  // ------------------------------------------------------------- epilogue
  if (warp < 4) {
    bool ok = tc::mbar_wait(tc::smem_u32(done), 0, kWaitNs) && nK > 0;
    tc::fence_after_sync();
    if (ok && !*reinterpret_cast<volatile int*>(abort_flag)) {
      const long long row = m0 + warp * 32 + lane;
#pragma unroll 1
      for (int col = 0; col < BN; col += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
        ep(row, n0 + col, v);
      }
    } else if (lane == 0) {
      atomicExch(err, 1);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 4) tc::tmem_dealloc(tmem, TCOLS);
}

template <int BN, bool BF16, class AL, class BL, class EP>
cudaError_t launch(long long M, int N, int K, const AL& al, const BL& bl, const EP& ep, int* err,
                   cudaStream_t s) {
  auto kern = gemm_kernel<BN, BF16, AL, BL, EP>;
  const int nK = (K + kBK - 1) / kBK;
  int ns = max_stages<BN>();
  if (ns > nK) ns = nK < 1 ? 1 : nK;
  const size_t smem = smem_bytes_for(stage_bytes<BN>(), ns);
  static size_t configured = 0;
  if (configured < smem) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes_for(stage_bytes<BN>(), max_stages<BN>()));
    if (e != cudaSuccess) return e;
    configured = smem_bytes_for(stage_bytes<BN>(), max_stages<BN>());
  }
  const dim3 grid((N + BN - 1) / BN, (unsigned)((M + kBM - 1) / kBM));
  kern<<<grid, kThreads, smem, s>>>(M, N, K, ns, al, bl, ep, err);
  return cudaGetLastError();
}

}  // namespace gemm
}  // namespace aew
