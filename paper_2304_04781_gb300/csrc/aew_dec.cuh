// Fused strain decoder (the adjoint's decode, Sec. 3.3 layers of Eq. (5)):
//   H = GELU(Z W3 + b3)         Z: FP16 latents [M][n_lat], W3t FP16 [512][n_lat]
//   E = H W4e^T (+ b4, x s_b)   W4e: the 512 strain rows of W4, BF16 [512][512]
// for tiles of 128 blocks, with H kept in shared memory between the two products
// instead of a round trip through HBM.
//
// Persistent CTAs (one per SM) walk the 128-block tiles.  Eighteen warps:
//   warp 16, one lane TMA producer.  Per tile: the latent tile (128 x 64, zero-filled
//                      past n_lat) and all of W3t (512 x 64) into the H buffer, which
//                      is free once the previous tile's second-layer MMAs have read it;
//                      then the 16 chunks of W4e (two output halves x 8 K chunks of
//                      256 x 64) through a 3-stage ring.
//   warp 17           TMEM (512 columns) and, on one lane, the MMA issuer: layer 1 as
//                      two N = 256 MMAs per K step into columns 0-511 (FP16 x FP16),
//                      then layer 2 for output half h into columns 256h..256h+255 (BF16
//                      x BF16): half 0's first four K chunks as soon as the epilogue has
//                      written hidden units 0-255 (whose accumulator columns 0-255 are
//                      then free), the rest once it has written 256-511.
//   warps 0-15        epilogue.  E1: layer-1 accumulator + b3, GELU, BF16, written into
//                      the H buffer in the 128-byte-swizzled K-major layout the MMA
//                      reads (8 K chunks of 128 rows x 128 bytes), hidden units 0-255
//                      first.  E2: layer-2 accumulator through the grid-scatter
//                      epilogue.
// H buffer, TMEM and ring are each reused tile after tile; mbarriers order every reuse,
// and every wait is bounded (a timed-out wait aborts the CTA and sets the error flag).
#pragma once

#include "aew_gemm.cuh"

namespace aew {
namespace dec {

constexpr int kRows = 128;                  // blocks per tile
constexpr int kHid = 512;
constexpr int kChunk = 16384;               // 128 rows x 64 x 2 bytes
constexpr int kHBytes = 8 * kChunk;         // H: 8 K chunks
constexpr int kW3Off = kChunk;              // W3t (512 x 64) behind the latent tile
constexpr int kRing = 3;
constexpr int kStage = 256 * 64 * 2;        // one W4e chunk: 256 output rows x 64 K
constexpr int kF1Bytes = kChunk + kHid * 64 * 2;
constexpr size_t kSmem = (size_t)kHBytes + (size_t)kRing * kStage + 256 + 1024;
constexpr int kThreads = 576;
constexpr int kEpi = 16;                    // epilogue warps
constexpr int kTmaWarp = 16, kMmaWarp = 17;

// byte offset of element k (0..63) of row r (0..127) in a 128-byte-swizzled K chunk
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  const int ch = k >> 3;
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4) + ((k & 7) << 1));
}

template <class EP>
__global__ void __launch_bounds__(kThreads, 1)
    dec2_kernel(const __grid_constant__ CUtensorMap tz, const __grid_constant__ CUtensorMap tw3,
                const __grid_constant__ CUtensorMap tw4, int M, const float* __restrict__ b3,
                EP ep, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint8_t* hb = smem;                       // H buffer (and layer-1 operands)
  uint8_t* ring = smem + kHBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + kRing * kStage);
  uint64_t* empty = full + kRing;
  uint64_t* f1 = empty + kRing;             // layer-1 operands landed
  uint64_t* acc1 = f1 + 1;                  // layer-1 accumulator complete
  uint64_t* hready = acc1 + 1;              // [2] H units 256j..256j+255 written
  uint64_t* hfree = hready + 2;             // layer-2 MMAs done reading H
  uint64_t* acc2 = hfree + 1;               // [2] output half complete
  uint64_t* tfree = acc2 + 2;               // [2] output half drained
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tfree + 2);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  if (*reinterpret_cast<volatile int*>(err) != 0) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int T = (M + kRows - 1) / kRows;
  constexpr uint32_t ID1 = tc::idesc_f16(kRows, 256, false);   // FP16 x FP16
  constexpr uint32_t ID2 = tc::idesc_f16(kRows, 256, true);    // BF16 x BF16
  constexpr uint64_t W = gemm::kWaitNs;

  if (warp == kMmaWarp) {
    tc::tmem_alloc(tc::smem_u32(tslot), 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    gemm::prefetch_tmap(&tz);
    gemm::prefetch_tmap(&tw3);
    gemm::prefetch_tmap(&tw4);
    for (int s = 0; s < kRing; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 1);
      tc::mbar_init(tc::smem_u32(&empty[s]), 1);
    }
    tc::mbar_init(tc::smem_u32(f1), 1);
    tc::mbar_init(tc::smem_u32(acc1), 1);
    for (int j = 0; j < 2; ++j) {
      tc::mbar_init(tc::smem_u32(&hready[j]), kEpi * 32);
      tc::mbar_init(tc::smem_u32(&acc2[j]), 1);
      tc::mbar_init(tc::smem_u32(&tfree[j]), kEpi * 32);
    }
    tc::mbar_init(tc::smem_u32(hfree), 1);
    *abort_flag = 0;
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == kTmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------------- TMA producer
      int it = 0, tl = 0;
      for (int t = blockIdx.x; t < T; t += gridDim.x, ++tl) {
        const int m0 = t * kRows;
        if (tl >= 1 && !tc::mbar_wait(tc::smem_u32(hfree), (tl - 1) & 1, W)) {
          atomicExch(abort_flag, 1);
          break;
        }
        const uint32_t fb = tc::smem_u32(f1), h0 = tc::smem_u32(hb);
        gemm::mbar_expect_tx(fb, kF1Bytes);
        gemm::tma_load_2d(h0, &tz, 0, m0, fb);
        gemm::tma_load_2d(h0 + kW3Off, &tw3, 0, 0, fb);
        gemm::tma_load_2d(h0 + kW3Off + 256 * 128, &tw3, 0, 256, fb);
        bool ok = true;
        for (int h = 0; h < 2 && ok; ++h)
          for (int kk = 0; kk < 8; ++kk, ++it) {
            const int s = it % kRing;
            if (it >= kRing &&
                !tc::mbar_wait(tc::smem_u32(&empty[s]), ((it / kRing) - 1) & 1, W)) {
              atomicExch(abort_flag, 1);
              ok = false;
              break;
            }
            const uint32_t b = tc::smem_u32(&full[s]);
            gemm::mbar_expect_tx(b, kStage);
            gemm::tma_load_2d(tc::smem_u32(ring + s * kStage), &tw4, kk * 64, h * 256, b);
          }
        if (!ok) break;
      }
      // the MMAs' last arrivals (ring stages, H released) land before the teardown
      bool ok = !*reinterpret_cast<volatile int*>(abort_flag);
      for (int j = it > kRing ? it - kRing : 0; j < it && ok; ++j)
        ok = tc::mbar_wait(tc::smem_u32(&empty[j % kRing]), (j / kRing) & 1, W);
      if (ok && tl > 0) ok = tc::mbar_wait(tc::smem_u32(hfree), (tl - 1) & 1, W);
      if (!ok) atomicExch(err, 1);
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ------------------------------------------------------------- MMA issuer
      int it = 0, tl = 0;
      const uint32_t h0 = tc::smem_u32(hb);
      for (int t = blockIdx.x; t < T; t += gridDim.x, ++tl) {
        const uint32_t ph = tl & 1;
        // layer 1: K = 64 in four steps of 16; outputs 256j..256j+255 into columns
        // 256j.., once the previous tile's output half j has left them.  One commit for
        // both: the epilogue overwrites the layer-1 operands with H, so it may start
        // only once every layer-1 MMA has read them.
        bool ok = tc::mbar_wait(tc::smem_u32(f1), ph, W);
        for (int j = 0; j < 2 && ok; ++j) {
          if (tl > 0 && !tc::mbar_wait(tc::smem_u32(&tfree[j]), (tl - 1) & 1, W)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_f16(tmem + (uint32_t)(j * 256), gemm::sdesc_sw128(h0 + k * 32),
                        gemm::sdesc_sw128(h0 + kW3Off + j * 256 * 128 + k * 32), ID1,
                        k > 0 ? 1u : 0u);
        }
        if (ok) tc::mma_commit(tc::smem_u32(acc1));
        if (!ok) {
          atomicExch(abort_flag, 1);
          break;
        }
        // layer 2: A = H from shared memory, B = W4e chunks from the ring.  K chunks 0-3
        // read hidden units 0-255 and 4-7 units 256-511, each half once the epilogue has
        // written it and so drained its accumulator columns (half 0 of the output
        // accumulates in columns 0-255, half 1 in 256-511).
        for (int h = 0; h < 2 && ok; ++h) {
          for (int kk = 0; kk < 8; ++kk, ++it) {
            if (h == 0 && (kk & 3) == 0) {
              if (!tc::mbar_wait(tc::smem_u32(&hready[kk >> 2]), ph, W)) {
                atomicExch(abort_flag, 1);
                ok = false;
                break;
              }
              tc::fence_after_sync();
            }
            const int s = it % kRing;
            if (!tc::mbar_wait(tc::smem_u32(&full[s]), (it / kRing) & 1, W)) {
              atomicExch(abort_flag, 1);
              ok = false;
              break;
            }
            tc::fence_after_sync();
            const uint32_t a0 = h0 + kk * kChunk, b0 = tc::smem_u32(ring + s * kStage);
#pragma unroll
            for (int k = 0; k < 4; ++k)
              tc::mma_f16(tmem + (uint32_t)(h * 256), gemm::sdesc_sw128(a0 + k * 32),
                          gemm::sdesc_sw128(b0 + k * 32), ID2, (kk > 0 || k > 0) ? 1u : 0u);
            tc::mma_commit(tc::smem_u32(&empty[s]));
          }
          if (ok) tc::mma_commit(tc::smem_u32(&acc2[h]));
        }
        if (!ok) break;
        tc::mma_commit(tc::smem_u32(hfree));
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------- epilogue warps
    const int q = warp & 3, cg = warp >> 2;   // TMEM lane quarter; column groups cg, cg+4, ..
    const int r = q * 32 + lane;              // row of the tile
    int tl = 0;
    for (int t = blockIdx.x; t < T; t += gridDim.x, ++tl) {
      const uint32_t ph = tl & 1;
      bool ok = tc::mbar_wait(tc::smem_u32(acc1), ph, W);
      tc::fence_after_sync();
      if (!ok || *reinterpret_cast<volatile int*>(abort_flag)) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
      // E1: H = bf16(gelu(acc + b3)), 32 columns at a time; hidden units 0-255 (K chunks
      // 0-3 of layer 2) first, each half released to the MMA issuer once written
      for (int half = 0; half < 2; ++half) {
#pragma unroll 1
        for (int g = cg + 8 * half; g < 8 * (half + 1); g += kEpi / 4) {
          // the bias loads go out ahead of the TMEM load, so that the two latencies overlap
          float4 bq[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) bq[j] = __ldg(reinterpret_cast<const float4*>(b3 + g * 32) + j);
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * 32), v);
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 32; j += 4) {
            const float4 b = bq[j / 4];
            float x0 = v[j] + b.x, x1 = v[j + 1] + b.y, x2 = v[j + 2] + b.z, x3 = v[j + 3] + b.w;
            gemm::gelu_fast_pair(x0, x1);
            gemm::gelu_fast_pair(x2, x3);
            pk[j / 2] = gemm::pack_bf16(x0, x1);
            pk[j / 2 + 1] = gemm::pack_bf16(x2, x3);
          }
          uint8_t* chunk = hb + (g >> 1) * kChunk;
          const int k0 = (g & 1) * 32;          // column within the 64-wide K chunk
#pragma unroll
          for (int c = 0; c < 4; ++c)
            *reinterpret_cast<uint4*>(chunk + sw128_off(r, k0 + 8 * c)) =
                make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
        }
        tc::fence_proxy_async();                // H visible to the tensor core
        tc::fence_before_sync();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&hready[half]))
                     : "memory");
      }
      // E2: output halves through the grid epilogue
      const typename EP::Row rc = ep.row((long long)t * kRows + r);
      for (int h = 0; h < 2 && ok; ++h) {
        ok = tc::mbar_wait(tc::smem_u32(&acc2[h]), ph, W);
        tc::fence_after_sync();
        if (!ok || *reinterpret_cast<volatile int*>(abort_flag)) {
          ok = false;
          break;
        }
#pragma unroll 1
        for (int g = cg; g < 8; g += kEpi / 4) {
          typename EP::Bias bb;
          ep.bias(h * 256 + g * 32, bb);   // ahead of the TMEM load, as in E1
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 256 + g * 32), v);
          ep(rc, h * 256 + g * 32, bb, v);
        }
        tc::fence_before_sync();
        // relaxed: it orders only the completed TMEM reads (tcgen05.wait::ld) before the
        // next tile's layer-1 MMAs into these columns, not the grid stores
        asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0];" ::"r"(
                         tc::smem_u32(&tfree[h]))
                     : "memory");
      }
      if (!ok) {
        if (lane == 0) atomicExch(err, 1);
        break;
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == kMmaWarp) tc::tmem_dealloc(tmem, 512);
}

}  // namespace dec
}  // namespace aew
