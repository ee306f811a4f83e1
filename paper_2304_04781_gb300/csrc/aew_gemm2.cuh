// Two-SM tcgen05 GEMM (cta_group::2) for the wide codec layer, the encoder's
// 2048 -> 512 product:  D[M][N] = sum_k A(m, k) B(n, k), FP32 accumulate in TMEM.
//
// A cluster of two CTAs on two SMs computes one 256 x 256 output tile with M = 256
// MMAs issued by the even CTA.  Each CTA stages its own 128 rows of A and one half
// (128 rows) of the tile's 256 rows of B; the tensor core reads the pair's operands
// from both shared memories and writes rows 0-127 of D into the even CTA's TMEM and
// rows 128-255 into the odd CTA's.  Per SM and K chunk of 64 that is 16 KB of A and
// 16 KB of B instead of the single-SM kernel's 16 + 32 KB for the same 128 x 256 x 64
// products, so the same shared memory holds six stages instead of four and each SM
// pulls a third fewer operand bytes.
//
// Per CTA, eighteen warps as in the single-SM kernel:
//   warp 16, one lane  TMA producer (both CTAs): waits for its own `empty` stage, loads
//                       its A rows and B half; the copies complete on the even CTA's
//                       `full` barrier, which the even CTA's producer arms with the
//                       pair's byte count;
//   warp 17            TMEM allocation for the pair (one warp in each CTA), and on the
//                       even CTA's lane 0 the MMA issuer; each commit arrives on the
//                       barrier of both CTAs (stage `empty`, accumulator `accf`);
//   warps 0-15         epilogue (both CTAs) on the CTA's own 128 rows; one arrival per
//                       warp on the even CTA's `acce` when an accumulator is drained.
// Every wait is bounded in time; a CTA that gives up records the error and runs on to
// the common teardown, so its partner's waits run out as well and both CTAs reach the
// final cluster barrier.
#pragma once

#include "aew_gemm.cuh"

namespace aew {
namespace gemm2 {

constexpr int kBM = 128;                        // rows per CTA; 256 per pair
constexpr int kBN = 256;                        // columns per pair tile
constexpr int kBK = 64;
constexpr int kABytes = kBM * kBK * 2;          // 16 KB
constexpr int kBBytes = (kBN / 2) * kBK * 2;    // 16 KB: this CTA's half of B
constexpr int kStage = kABytes + kBBytes;
constexpr int kStages = 6;
constexpr size_t kSmem = (size_t)kStages * kStage + 256 + 1024;
constexpr int kEpiWarps = 16;
constexpr int kTmaWarp = 16, kMmaWarp = 17;
constexpr int kThreads = 576;
constexpr uint32_t kCols = 2 * kBN;             // two accumulators

__device__ __forceinline__ uint32_t cta_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the address of the same shared-memory variable in cluster CTA `rank`
__device__ __forceinline__ uint32_t map_to(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc2(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish2() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc2(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma2(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                     uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// arrive once on the barrier at this offset in both CTAs when the issued MMAs complete
__device__ __forceinline__ void commit2_both(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 "
      "[%0], %1;" ::"r"(mbar), "h"((unsigned short)0x3)
      : "memory");
}
// TMA tile load into this CTA's shared memory, completing on a barrier of either CTA
// of the pair (cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int c0,
                                                 int c1, uint32_t mbar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar_cluster)
      : "memory");
}
// bounded wait (as tc::mbar_wait) with cluster-scope acquire: the arrivals come from
// the partner CTA or from MMAs that touched both CTAs' memories
__device__ __forceinline__ bool wait_cl(uint32_t mbar, uint32_t parity, uint64_t ns) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255u) == 0) {
      const uint64_t t = tc::globaltimer();
      if (t0 == 0) t0 = t;
      else if (t - t0 > ns) return false;
    }
  }
}
// An epilogue warp's "accumulator drained" signal.  Relaxed: the signal orders only the
// warp's TMEM reads, which tcgen05.wait::ld has already completed, before the MMAs that
// overwrite the accumulator; a release would also hold the warp until its global stores
// of the tile are performed at cluster scope, which nothing in the kernel reads.
__device__ __forceinline__ void arrive_remote(uint32_t mbar_cluster) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(mbar_cluster)
               : "memory");
}

template <bool BF16, class EP>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    gemm2_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                 int M, int N, int K, EP ep, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr uint32_t IDESC = tc::idesc_f16(2 * kBM, kBN, BF16);
  constexpr uint64_t W = gemm::kWaitNs;

  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint64_t* empty = full + kStages;
  uint64_t* accf = empty + kStages;   // accumulator a ready (both CTAs)
  uint64_t* acce = accf + 2;          // accumulator a drained (even CTA)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cta_rank();
  const bool lead = rank == 0;
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int nK = (K + kBK - 1) / kBK;
  const int tn = (N + kBN - 1) / kBN;
  const int T = ((M + 2 * kBM - 1) / (2 * kBM)) * tn;

  if (tid == 0) {
    gemm::prefetch_tmap(&ta);
    gemm::prefetch_tmap(&tb);
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(tc::smem_u32(&accf[a]), 1);
      tc::mbar_init(tc::smem_u32(&acce[a]), 2 * kEpiWarps);
    }
    tc::mbar_fence_init();
  }
  // both CTAs take part in the pair's TMEM allocation whatever happens next
  if (warp == kMmaWarp) {
    tmem_alloc2(tc::smem_u32(tslot), kCols);
    tmem_relinquish2();
  }
  tc::fence_before_sync();
  __syncthreads();
  cluster_sync();   // the partner's barriers are initialised from here on
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  // a previous launch already failed: skip the work (the host reports the error), but
  // still go through the teardown with the partner
  const bool dead = *reinterpret_cast<volatile int*>(err) != 0;

  if (warp == kTmaWarp) {
    if (lane == 0 && !dead) {
      // ----------------------------------------------------------- TMA producer
      int it = 0;
      bool ok = true;
      for (int t = pair; t < T && ok; t += npairs) {
        const int m0 = (t / tn) * (2 * kBM) + (int)rank * kBM;
        const int n0 = (t % tn) * kBN + (int)rank * (kBN / 2);
        for (int c = 0; c < nK; ++c, ++it) {
          const int s = it % kStages;
          if (it >= kStages &&
              !wait_cl(tc::smem_u32(&empty[s]), ((it / kStages) - 1) & 1, W)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          const uint32_t fl = tc::smem_u32(&full[s]);
          if (lead) gemm::mbar_expect_tx(fl, 2 * kStage);   // both CTAs' copies
          const uint32_t fb = map_to(fl, 0);
          const uint32_t sa = tc::smem_u32(smem + s * kStage);
          tma_load_2d_pair(sa, &ta, c * kBK, m0, fb);
          tma_load_2d_pair(sa + kABytes, &tb, c * kBK, n0, fb);
        }
      }
      // the MMAs' last arrivals on this CTA's stage barriers land before the teardown
      for (int j = it > kStages ? it - kStages : 0; j < it && ok; ++j)
        ok = wait_cl(tc::smem_u32(&empty[j % kStages]), (j / kStages) & 1, W);
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0 && lead && !dead) {
      // ----------------------------------------------------------- MMA issuer
      int it = 0, tl = 0;
      for (int t = pair; t < T; t += npairs, ++tl) {
        const int a = tl & 1;
        if (tl >= 2 && !wait_cl(tc::smem_u32(&acce[a]), ((tl >> 1) - 1) & 1, W)) {
          atomicExch(err, 1);
          break;
        }
        tc::fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(a * kBN);
        bool ok = true;
        for (int c = 0; c < nK; ++c, ++it) {
          const int s = it % kStages;
          if (!wait_cl(tc::smem_u32(&full[s]), (it / kStages) & 1, W)) {
            atomicExch(err, 1);
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t a0 = tc::smem_u32(smem + s * kStage), b0 = a0 + kABytes;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk)
            mma2(acc, gemm::sdesc_sw128(a0 + kk * 32), gemm::sdesc_sw128(b0 + kk * 32), IDESC,
                 (c > 0 || kk > 0) ? 1u : 0u);
          commit2_both(tc::smem_u32(&empty[s]));
        }
        if (!ok) break;
        commit2_both(tc::smem_u32(&accf[a]));
      }
    }
    __syncwarp();
  } else if (!dead) {
    // ------------------------------------------------------------- epilogue warps
    const int q = warp & 3, cg = warp >> 2;
    constexpr int G = kBN / 32;
    const uint32_t drained[2] = {map_to(tc::smem_u32(&acce[0]), 0),
                                 map_to(tc::smem_u32(&acce[1]), 0)};
    int tl = 0;
    for (int t = pair; t < T; t += npairs, ++tl) {
      const int a = tl & 1;
      if (!wait_cl(tc::smem_u32(&accf[a]), (tl >> 1) & 1, W)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      tc::fence_after_sync();
      const long long row = (long long)(t / tn) * (2 * kBM) + rank * kBM + q * 32 + lane;
      const int n0 = (t % tn) * kBN;
#pragma unroll 1
      for (int g = cg; g < G; g += kEpiWarps / 4) {
        float v[32];
        tc::tmem_ld32(tmem + (uint32_t)(a * kBN) + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 32), v);
        ep(row, n0 + g * 32, v);
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) arrive_remote(drained[a]);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  cluster_sync();   // no CTA leaves while its partner may still use the pair's TMEM
  tc::fence_after_sync();
  if (warp == kMmaWarp) tmem_dealloc2(tmem, kCols);
}

// D = A B^T through the pair kernel: at most max_ctas CTAs (rounded down to pairs).
template <bool BF16, class EP>
cudaError_t launch(long long M, int N, int K, const gemm::Mat& A, const gemm::Mat& B, const EP& ep,
                   int* err, cudaStream_t s, int max_ctas = 0) {
  auto kern = gemm2_kernel<BF16, EP>;
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (attr != cudaSuccess) return attr;
  const int sms = gemm::sm_count();
  CUtensorMap ta, tb;
  if (gemm::make_tmap(&ta, A.p, !BF16, A.rows, K, A.ld, kBM, true) != CUDA_SUCCESS ||
      gemm::make_tmap(&tb, B.p, !BF16, B.rows, K, B.ld, kBN / 2, true) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const long long tiles = ((M + 2 * kBM - 1) / (2 * kBM)) * (long long)((N + kBN - 1) / kBN);
  if (tiles == 0) return cudaSuccess;
  int cap = (max_ctas > 0 && max_ctas < sms) ? max_ctas : sms;
  cap /= 2;
  if (cap < 1) cap = 1;
  const int pairs = (int)(tiles < cap ? tiles : cap);
  kern<<<2 * pairs, kThreads, kSmem, s>>>(ta, tb, (int)M, N, K, ep, err);
  return cudaGetLastError();
}

}  // namespace gemm2
}  // namespace aew
