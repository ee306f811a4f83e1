// Generic tcgen05 GEMM building block for the codec and its training:
//   D[M][N] = sum_k A(m, k) B(n, k)      (FP32 accumulate in TMEM)
// A and B are 16-bit (BF16 or FP16) row-major matrices with K contiguous, described by
// TMA tensor maps; D goes through a pluggable epilogue (TMEM -> registers -> fused
// bias / activation / store).
//
// Persistent CTAs (one per SM) walk 128 x BN output tiles; K runs in chunks of 64
// through a ring of `ns` shared-memory stages.  Eighteen warps:
//   warp 16, one lane TMA producer: per chunk one cp.async.bulk.tensor per operand
//                      (128-byte-swizzled tile; or, with SW = false, eight 16-byte-wide
//                      boxes into the unswizzled canonical layout), completion counted
//                      in bytes on the stage's `full` mbarrier;
//   warp 17           TMEM allocation (two BN-column accumulators) and, on one lane,
//                      the MMA issuer: 4 x tcgen05.mma (K = 16) per chunk,
//                      tcgen05.commit to the stage's `empty` mbarrier, and per tile to
//                      the accumulator's `accf` mbarrier;
//   warps 0-15        epilogue (four warps per TMEM lane quarter, each taking every
//                      fourth 32-column group), which drains accumulator a while the
//                      MMAs fill the other one, then arrives on `acce[a]`.
// Every wait is bounded in time; on timeout the kernel records an error and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "aew_tc.cuh"

namespace aew {
namespace gemm {

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kEpiWarps = 16;                // warps 0-15: epilogue
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTmaWarp = 16;
constexpr int kMmaWarp = 17;
constexpr int kThreads = 576;
constexpr uint64_t kWaitNs = 200000000ull;   // 200 ms (a healthy wait takes microseconds)
constexpr int kSmemBudget = 200 * 1024;

template <int BN>
__host__ __device__ constexpr int stage_bytes() {
  return kBM * kBK * 2 + BN * kBK * 2;   // [A][B]
}
template <int BN>
__host__ __device__ constexpr int max_stages() {
  return kSmemBudget / stage_bytes<BN>() > 8 ? 8 : kSmemBudget / stage_bytes<BN>();
}
inline size_t smem_bytes_for(int stage_b, int ns) { return (size_t)ns * stage_b + 256 + 1024; }

// ---------------------------------------------------------------------------------
// TMA
// ---------------------------------------------------------------------------------
// Tensor map of a row-major 16-bit matrix [rows][K] (row stride ld elements); box =
// (64 K x box_rows) with 128-byte swizzle, or (8 K x box_rows) unswizzled.
CUresult make_tmap(CUtensorMap* map, const void* base, bool fp16, long long rows, int K,
                   long long ld, int box_rows, bool swizzle128);
// cuTensorMapEncodeTiled of the CUDA driver API (looked up once; null if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// shared-memory descriptor of a K-major tile with 128-byte swizzle: rows of 128 bytes,
// 8-row groups 1024 bytes apart; K steps of 16 elements advance the start by 32 bytes
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                 // fixed 0b001
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Power-of-two block scale s = 2^max(e, -100) of a block maximum m 2^e (m in [0.5, 1)),
// 0 for m = 0; the clamp keeps 1/s finite in FP32 for blocks of subnormal values.
constexpr int kExpMin = -100;
__device__ __forceinline__ int block_exp(float mx) {
  int e = 0;
  frexpf(mx, &e);
  return e < kExpMin ? kExpMin : e;
}
__device__ __forceinline__ float block_scale(float mx) {
  return mx > 0.f ? ldexpf(1.f, block_exp(mx)) : 0.f;
}
__device__ __forceinline__ float block_inv_scale(float mx) {
  return mx > 0.f ? ldexpf(1.f, -block_exp(mx)) : 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}
// one 32-byte store (sm_100 family; p 32-byte aligned): a lane's half of a 32-column
// BF16 row group writes whole 32-byte sectors instead of two 16-byte halves
__device__ __forceinline__ void st_global_32B(void* p, uint32_t w0, uint32_t w1, uint32_t w2,
                                              uint32_t w3, uint32_t w4, uint32_t w5, uint32_t w6,
                                              uint32_t w7) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w0),
               "r"(w1), "r"(w2), "r"(w3), "r"(w4), "r"(w5), "r"(w6), "r"(w7)
               : "memory");
}
__device__ __forceinline__ uint16_t bf16_bits(float a) {
  __nv_bfloat16 t = __float2bfloat16_rn(a);
  return *reinterpret_cast<uint16_t*>(&t);
}
__device__ __forceinline__ float bf16_val(uint16_t b) {
  return __uint_as_float(((uint32_t)b) << 16);
}
// GELU(a) = a Phi(a), Phi(a) = (1 + erf(a / sqrt 2)) / 2, and its derivative
// Phi(a) + a phi(a), with erff: the training kernels' activation.
__device__ __forceinline__ float gelu_f(float a) {
  return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_prime_f(float a) {
  return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) +
         a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// The inference epilogues' GELU (encoder layer 1, decoder layer 1), where the activation
// is the hot arithmetic: Phi through the approximation of Abramowitz & Stegun, Handbook
// of Mathematical Functions, eq. 7.1.28 (after Hastings): erfc(z) = (1 + c1 z + c2 z^2 +
// ... + c6 z^6)^-16 for z >= 0, with |error| <= 3e-7, applied to z = |a| / sqrt 2, and
// Phi taken as erfc / 2 below 0 and 1 - erfc / 2 above, so the lower tail is never a
// difference of nearly equal numbers.  In FP32 the 16th power multiplies the rounding
// of its base by 16: Phi is within 1e-6, about a thousandth of the BF16 rounding the
// activations take next.  One reciprocal and twelve multiply-adds, far fewer
// instructions than erff.
__device__ __forceinline__ float normal_cdf_fast(float a) {
  const float z = fabsf(a) * 0.70710678118654752f;
  float d = fmaf(fmaf(fmaf(fmaf(fmaf(4.30638e-5f, z, 2.765672e-4f), z, 1.520143e-4f), z,
                          9.2705272e-3f), z, 4.22820123e-2f), z, 7.05230784e-2f);
  d = fmaf(d, z, 1.0f);
  d *= d;   // ^2
  d *= d;   // ^4
  d *= d;   // ^8
  d *= d;   // ^16
  float r;   // 1 / d to 1 ulp (0 once d overflows: erfc(z) below FP32's range)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  const float h = 0.5f * r;   // erfc(z) / 2
  return a >= 0.f ? 1.0f - h : h;
}
__device__ __forceinline__ float gelu_fast(float a) { return a * normal_cdf_fast(a); }

// sm_100-family paired FP32 instructions (add / sub / mul / fma on .f32x2): two FP32
// lanes of one 64-bit register, each lane rounded exactly as the scalar instruction
// rounds it, at one issue slot for the pair.
namespace f2 {
__device__ __forceinline__ uint64_t make(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ uint64_t splat(float v) { return make(v, v); }
__device__ __forceinline__ void split(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
}  // namespace f2

// gelu_fast on the pair (a0, a1) in place, with the paired instructions: the same
// operations in the same order as normal_cdf_fast and gelu_fast, so each result equals
// gelu_fast's bit for bit, in about 13 issue slots per value instead of about 20.  The
// hidden-layer epilogues are issue-bound on the activation where the product before
// them is short (decoder layer 1: K = 512 against 1024 activations per row).
__device__ __forceinline__ void gelu_fast_pair(float& a0, float& a1) {
  const uint64_t a = f2::make(a0, a1);
  const uint64_t z = f2::mul(f2::make(fabsf(a0), fabsf(a1)), f2::splat(0.70710678118654752f));
  uint64_t d = f2::fma(f2::splat(4.30638e-5f), z, f2::splat(2.765672e-4f));
  d = f2::fma(d, z, f2::splat(1.520143e-4f));
  d = f2::fma(d, z, f2::splat(9.2705272e-3f));
  d = f2::fma(d, z, f2::splat(4.22820123e-2f));
  d = f2::fma(d, z, f2::splat(7.05230784e-2f));
  d = f2::fma(d, z, f2::splat(1.0f));
  d = f2::mul(d, d);   // ^2
  d = f2::mul(d, d);   // ^4
  d = f2::mul(d, d);   // ^8
  d = f2::mul(d, d);   // ^16
  float d0, d1, r0, r1;
  f2::split(d, d0, d1);
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d0));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r1) : "f"(d1));
  const uint64_t h = f2::mul(f2::splat(0.5f), f2::make(r0, r1));   // erfc(z) / 2
  const uint64_t u = f2::sub(f2::splat(1.0f), h);
  float h0, h1, u0, u1;
  f2::split(h, h0, h1);
  f2::split(u, u0, u1);
  f2::split(f2::mul(a, f2::make(a0 >= 0.f ? u0 : h0, a1 >= 0.f ? u1 : h1)), a0, a1);
}

// ---------------------------------------------------------------------------------
// The kernel (persistent: each CTA walks tiles blockIdx.x, +gridDim.x, ...)
// ---------------------------------------------------------------------------------
template <int BN, bool BF16, bool SW, class EP>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                int M, int N, int K, int ns, EP ep, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int A_BYTES = kBM * kBK * 2;
  constexpr int B_BYTES = BN * kBK * 2;
  constexpr int STAGE = stage_bytes<BN>();                // [A][B]
  constexpr uint32_t TCOLS = 2 * BN < 32 ? 32 : 2 * BN;   // two accumulators
  constexpr uint32_t IDESC = tc::idesc_f16(kBM, BN, BF16);
  static_assert(BN % 32 == 0 && BN <= 256, "BN");

  uint64_t* full = reinterpret_cast<uint64_t*>(smem + ns * STAGE);
  uint64_t* empty = full + ns;
  uint64_t* accf = empty + ns;     // accumulator a ready for the epilogue
  uint64_t* acce = accf + 2;       // accumulator a drained by the epilogue
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  // a previous launch already failed: do nothing (the host reports the error)
  if (*reinterpret_cast<volatile int*>(err) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nK = (K + kBK - 1) / kBK;
  const int tn = (N + BN - 1) / BN;
  const int T = ((M + kBM - 1) / kBM) * tn;

  if (warp == kMmaWarp) {
    tc::tmem_alloc(tc::smem_u32(tslot), TCOLS);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    prefetch_tmap(&ta);
    prefetch_tmap(&tb);
    for (int s = 0; s < ns; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(tc::smem_u32(&accf[a]), 1);
      tc::mbar_init(tc::smem_u32(&acce[a]), kEpiThreads);
    }
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ----------------------------------------------------------- TMA producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < T && ok; t += gridDim.x) {
        const int m0 = (t / tn) * kBM, n0 = (t % tn) * BN;
        for (int c = 0; c < nK; ++c, ++it) {
          const int s = it % ns;
          if (it >= ns && !tc::mbar_wait(tc::smem_u32(&empty[s]), ((it / ns) - 1) & 1, kWaitNs)) {
            atomicExch(abort_flag, 1);
            ok = false;
            break;
          }
          const uint32_t fb = tc::smem_u32(&full[s]);
          const uint32_t sa = tc::smem_u32(smem + s * STAGE), sb = sa + A_BYTES;
          mbar_expect_tx(fb, A_BYTES + B_BYTES);   // bytes the two TMA loads deliver
          if (SW) {
            tma_load_2d(sa, &ta, c * kBK, m0, fb);
            tma_load_2d(sb, &tb, c * kBK, n0, fb);
          } else {
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              tma_load_2d(sa + g * (kBM * 16), &ta, c * kBK + 8 * g, m0, fb);
              tma_load_2d(sb + g * (BN * 16), &tb, c * kBK + 8 * g, n0, fb);
            }
          }
        }
      }
      // the MMAs' last arrivals on the stage barriers land before the teardown
      for (int j = it > ns ? it - ns : 0; j < it && ok; ++j)
        ok = tc::mbar_wait(tc::smem_u32(&empty[j % ns]), (j / ns) & 1, kWaitNs);
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ----------------------------------------------------------- MMA issuer
      int it = 0, tl = 0;
      for (int t = blockIdx.x; t < T; t += gridDim.x, ++tl) {
        const int a = tl & 1;
        if (tl >= 2 && !tc::mbar_wait(tc::smem_u32(&acce[a]), ((tl >> 1) - 1) & 1, kWaitNs)) {
          atomicExch(abort_flag, 1);
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(a * BN);
        bool ok = true;
        for (int c = 0; c < nK; ++c, ++it) {
          const int s = it % ns;
          if (!tc::mbar_wait(tc::smem_u32(&full[s]), (it / ns) & 1, kWaitNs)) {
            atomicExch(abort_flag, 1);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t st0 = tc::smem_u32(smem + s * STAGE);
          const uint32_t a0 = st0, b0 = st0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            uint64_t ad, bd;
            if (SW) {
              ad = sdesc_sw128(a0 + kk * 32);
              bd = sdesc_sw128(b0 + kk * 32);
            } else {
              ad = tc::sdesc(a0 + kk * 2 * (kBM * 16), kBM * 16, 128);
              bd = tc::sdesc(b0 + kk * 2 * (BN * 16), BN * 16, 128);
            }
            tc::mma_f16(acc, ad, bd, IDESC, (c > 0 || kk > 0) ? 1u : 0u);
          }
          tc::mma_commit(tc::smem_u32(&empty[s]));
        }
        if (!ok) break;
        tc::mma_commit(tc::smem_u32(&accf[a]));
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue warps
    // a warp reaches only its TMEM lane quarter (warp % 4); column groups g = cg, cg+4..
    const int q = warp & 3, cg = warp >> 2;
    constexpr int G = BN / 32;                   // 32-column groups per tile
    int tl = 0;
    for (int t = blockIdx.x; t < T; t += gridDim.x, ++tl) {
      const int a = tl & 1;
      const bool ok = tc::mbar_wait(tc::smem_u32(&accf[a]), (tl >> 1) & 1, kWaitNs);
      tc::fence_after_sync();
      if (!ok || *reinterpret_cast<volatile int*>(abort_flag)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      const int m0 = (t / tn) * kBM, n0 = (t % tn) * BN;
      const long long row = (long long)m0 + q * 32 + lane;
#pragma unroll 1
      for (int g = cg; g < G; g += kEpiWarps / 4) {
        const int col = g * 32;
        float v[32];
        tc::tmem_ld32(tmem + (uint32_t)(a * BN) + ((uint32_t)(q * 32) << 16) + (uint32_t)col, v);
        ep(row, n0 + col, v);
      }
      tc::fence_before_sync();
      // relaxed: it orders only the warp's completed TMEM reads (tcgen05.wait::ld) before
      // the MMAs that overwrite the accumulator, not the warp's global stores
      asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acce[a]))
                   : "memory");
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kMmaWarp) tc::tmem_dealloc(tmem, TCOLS);
}

// SM count of the current device, found once (thread-safe static initialisation).
inline int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// Operand description for launch(): row-major [rows][K] 16-bit matrix, row stride ld.
struct Mat {
  const void* p;
  long long rows;
  long long ld;
};

#ifndef AEW_GEMM_SWIZZLE
#define AEW_GEMM_SWIZZLE 1
#endif

template <int BN, bool BF16, class EP>
cudaError_t launch(long long M, int N, int K, const Mat& A, const Mat& B, const EP& ep, int* err,
                   cudaStream_t s, int max_ctas = 0, int max_ns = 0) {
  constexpr bool SW = AEW_GEMM_SWIZZLE != 0;
  auto kern = gemm_kernel<BN, BF16, SW, EP>;
  const int nK = (K + kBK - 1) / kBK;
  int ns = max_stages<BN>();
  if (ns > nK + 2) ns = nK + 2;   // a few chunks of the next tile may be in flight
  if (max_ns > 0 && ns > max_ns) ns = max_ns;   // fewer stages: room for a co-resident CTA
  if (ns < 2) ns = 2;
  const size_t smem = smem_bytes_for(stage_bytes<BN>(), ns);
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem_bytes_for(stage_bytes<BN>(), max_stages<BN>()));
  if (attr != cudaSuccess) return attr;
  const int sms = sm_count();
  CUtensorMap ta, tb;
  if (make_tmap(&ta, A.p, !BF16, A.rows, K, A.ld, kBM, SW) != CUDA_SUCCESS ||
      make_tmap(&tb, B.p, !BF16, B.rows, K, B.ld, BN, SW) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const long long tiles = ((M + kBM - 1) / kBM) * (long long)((N + BN - 1) / BN);
  const int cap = (max_ctas > 0 && max_ctas < sms) ? max_ctas : sms;
  const int grid = (int)(tiles < cap ? tiles : cap);
  kern<<<grid, kThreads, smem, s>>>(ta, tb, (int)M, N, K, ns, ep, err);
  return cudaGetLastError();
}

}  // namespace gemm
}  // namespace aew
