// Leapfrog stencil kernels for the velocity-strain acoustic system (Sec. 2, Eq. (1),
// rho = 1) and its discrete adjoint, with every input plane staged in shared memory by
// the Tensor Memory Accelerator.
//
// Tiling.  Each CTA owns a 128 (x) x TY (y) column of nodes and marches through a chunk
// of kc z-planes.  One thread computes 4 consecutive x nodes (float4 accesses; a warp
// covers one 512-byte row segment).  For every plane the CTA needs, one elected thread
// issues one cp.async.bulk.tensor.3d per input field into a ring of S shared-memory
// stages; completion is counted in bytes on the stage's mbarrier.  The boxes carry the
// halos the update needs (zero-filled by the TMA outside the grid):
//   forward   e, m (and dm, e^n for the incremental step)  136 x (TY+2)  x-1..x+128, y-1..y+TY
//             vx                                           136 x TY      x-1 face
//             vy                                           128 x (TY+1)  y-1 face
//             vz                                           128 x TY
//   adjoint   mu                                           136 x (TY+2)
//             lam_x / lam_y / lam_z                        as vx / vy / vz
//             m, e^n, FP32 window accumulator              128 x TY
// The plane below the chunk (for the z-face under its first plane) and the plane above
// it (for the z-faces of its last plane) are staged with only the fields they feed.
// With the next planes in flight, the SM's threads only wait when HBM falls behind.
//
// Faces shared with a neighbouring thread are recomputed with the identical expression
// instead of exchanged (x neighbours still come by warp shuffle), so the results are
// bitwise independent of the tiling.  Per plane a CTA synchronises once, after which
// the freed stage is refilled.  Every wait is bounded (200 ms); a timed-out wait sets
// the sticky error flag, and a kernel that finds the flag set returns at once.
//
// Algorithmic HBM traffic per node: forward 36 B (5 fields read, 4 written),
// incremental forward 44 B, adjoint 48 B + 16 B / W (FP64 flush every W steps).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "aew_gemm.cuh"
#include "aew_internal.cuh"
#include "aew_tc.cuh"

namespace aew {
namespace {

constexpr int TY = 8;                 // rows (warps) per CTA
constexpr int NTHR = 32 * TY;
constexpr int kHX = 4;                // x halo width (one float4)
constexpr int kWE = kTXW + 2 * kHX;   // 136: row width of boxes with an x halo
constexpr int kW4E = kWE / 4;         // 34 float4 per halo row
constexpr int kW4 = kTXW / 4;         // 32 float4 per plain row
// a BF16 e^n box of the incremental forward: an x halo of 8 (16 bytes, TMA's alignment
// unit) instead of 4, so the row is 144 wide and the FP32 layout's element (r, c) sits at
// r * 144 + c + 4
constexpr int kHX16 = 8;
constexpr int kWE16 = kTXW + 2 * kHX16;
constexpr uint64_t kWaitNs = 200000000ull;
// TMA ring depth: at least 3, since the first plane of a chunk needs the planes below and
// above it resident at once; 4 measured slower (one CTA fewer per SM).  A compile-time
// depth keeps the ring's slot and phase arithmetic to a few instructions per plane.
constexpr int kStages = 3;
// PACK: one plane of the CTA's 16 blocks, 4 fields x 8 rows x 8 BF16 each (a 512-byte
// row per block, rows 528 bytes apart so that the 16 lane pairs of a warp, one per
// block, write distinct banks), double-buffered.  MAXO: the block maxima of the output
// per warp row, [TY][16][4] floats.
constexpr int kPackRow = 512 + 16;
constexpr int kPackTile = (kTXW / 8) * kPackRow;
constexpr int kPackExtra = 2 * kPackTile;
constexpr int kMaxoExtra = TY * 16 * 4 * 4;

// bytes one box delivers (the mbarrier transaction count) ...
constexpr int kTxXY = kWE * (TY + 2) * 4;   // x halo both sides, y halo both sides
constexpr int kTxX = kWE * TY * 4;          // x halo only
constexpr int kTxYm = kTXW * (TY + 1) * 4;  // one row below
constexpr int kTxO = kTXW * TY * 4;         // own nodes only
constexpr int kTxXY16 = kWE16 * (TY + 2) * 2;   // BF16 e^n of the incremental forward
// ... and the shared-memory room it takes (128-byte aligned destinations)
constexpr int al128(int b) { return (b + 127) & ~127; }
constexpr int kBoxXY = al128(kTxXY);
constexpr int kBoxX = al128(kTxX);
constexpr int kBoxYm = al128(kTxYm);
constexpr int kBoxO = al128(kTxO);

// stage layouts (byte offsets)
struct FwdLayout {
  static constexpr int E = 0, M = kBoxXY, VX = 2 * kBoxXY, VY = VX + kBoxX, VZ = VY + kBoxYm;
  static constexpr int DM = VZ + kBoxO, EF = DM + kBoxXY;
  __host__ __device__ static constexpr int bytes(bool incr) { return incr ? EF + kBoxXY : VZ + kBoxO; }
};
struct AdjLayout {
  static constexpr int MU = 0, LX = kBoxXY, LY = LX + kBoxX, LZ = LY + kBoxYm, M = LZ + kBoxO;
  static constexpr int EN = M + kBoxO, W = EN + kBoxO, BYTES = W + kBoxO;
};

struct FwdMaps {
  CUtensorMap e, m, vx, vy, vz, dm, ef;
};
struct AdjMaps {
  CUtensorMap mu, lx, ly, lz, m, en, w;
};

__device__ __forceinline__ void tma3(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                     uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void st4(float* p, size_t i, float4 v) {
  *reinterpret_cast<float4*>(p + i) = v;
}
__device__ __forceinline__ float& comp(float4& v, int c) {
  return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 z4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
// the source's force on the z-faces of the 4 nodes (k, y, i0 .. i0 + 3): dts times the
// spread weight of each face inside the source box (a point source: the one face, 1)
__device__ __forceinline__ void add_source(float4& v, int k, int y, int i0, const FwdStep& a) {
  if (a.sk < 0) return;
  const int W = 2 * a.sr + 1;
  const int dk = k - a.sk + a.sr, dy = y - a.sj + a.sr;
  if ((unsigned)dk >= (unsigned)W || (unsigned)dy >= (unsigned)W) return;
  const float* w = a.src_w + ((size_t)dk * W + dy) * W;
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const int dx = i0 + d - a.si + a.sr;
    if ((unsigned)dx < (unsigned)W) comp(v, d) = fmaf(a.dts, __ldg(w + dx), comp(v, d));
  }
}
// The m e products are plain multiplies; the face updates below subtract them with
// __fsub_rn, which the compiler never merges with a multiply, so every face is
// fma(dth, round(m_hi e_hi) - round(m_lo e_lo), v) wherever it is computed: by its
// owner, or recomputed at a chunk's first plane or by the neighbouring lane.  (Left to
// the compiler, a subtraction could absorb one product into an FMA at one site and not
// at another, and the results then depended in the last bit on the z-chunk depth.)
__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float4 fma4(float4 a, float4 b, float4 c) {
  return make_float4(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y), fmaf(a.z, b.z, c.z),
                     fmaf(a.w, b.w, c.w));
}
// 1 / s for a block maximum m >= 0 given as float bits, equal to
// gemm::block_inv_scale(m) (s = 2^max(e, -100), m = f 2^e with f in [0.5, 1); 0 for
// m = 0) but from the exponent field: e = biased - 126 for normal m, and subnormal m
// falls under the clamp.  Maxima of 2^126 and above take the library path.
__device__ __forceinline__ float inv_scale_bits(uint32_t mb) {
  const int eb = (int)(mb >> 23);
  if (mb == 0u) return 0.f;
  if (eb >= 253) return gemm::block_inv_scale(__uint_as_float(mb));
  const int e = max(eb - 126, gemm::kExpMin);
  return __uint_as_float((uint32_t)(127 - e) << 23);
}
__device__ __forceinline__ float hmax4(float4 a) {
  return fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w)));
}
__device__ __forceinline__ uint32_t pack2bf(float a, float b) {
  __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&t);
}
// face update v' = v + dth (hi - lo), the difference rounded on its own (see above)
__device__ __forceinline__ float fupd(float dth, float hi, float lo, float v) {
  return fmaf(dth, __fsub_rn(hi, lo), v);
}
__device__ __forceinline__ float4 fupd4(float dth, float4 hi, float4 lo, float4 v) {
  return make_float4(fupd(dth, hi.x, lo.x, v.x), fupd(dth, hi.y, lo.y, v.y),
                     fupd(dth, hi.z, lo.z, v.z), fupd(dth, hi.w, lo.w, v.w));
}
// lam' = (lam + inj) + dth (mu - mu_hi)
__device__ __forceinline__ float lupd(float dth, float mu_hi, float mu, float l) {
  return fmaf(dth, mu - mu_hi, l);
}
__device__ __forceinline__ float4 lupd4(float dth, float4 hi, float4 lo, float4 l) {
  return make_float4(lupd(dth, hi.x, lo.x, l.x), lupd(dth, hi.y, lo.y, l.y),
                     lupd(dth, hi.z, lo.z, l.z), lupd(dth, hi.w, lo.w, l.w));
}

__device__ __forceinline__ bool sticky_error(const int* err) {
  return err && *reinterpret_cast<const volatile int*>(err) != 0;
}

// Ring bookkeeping shared by both kernels: the CTA stages planes p0 = kbeg - 1 .. pn =
// kend in order; plane p lives in stage (p - p0) % S and completes phase
// ((p - p0) / S) & 1 of that stage's barrier.
struct Ring {
  static constexpr int S = kStages;
  uint8_t* base;
  uint32_t bar0;   // shared address of barrier 0 (8 bytes each)
  int stage_bytes, p0;
  __device__ int slot(int p) const { return (p - p0) % S; }
  __device__ uint32_t parity(int p) const { return ((p - p0) / S) & 1; }
  __device__ uint8_t* at(int p) const { return base + (size_t)slot(p) * stage_bytes; }
  __device__ uint32_t sat(int p) const { return tc::smem_u32(at(p)); }
  __device__ uint32_t bar(int p) const { return bar0 + 8u * slot(p); }
  __device__ bool wait(int p) const { return tc::mbar_wait(bar(p), parity(p), kWaitNs); }
};

// ---------------------------------------------------------------------------------
// Forward-type step
// ---------------------------------------------------------------------------------
// fields staged per plane: full planes carry everything, the plane below the chunk
// e, m (dm, e^n) and vz, the plane above it e, m (dm, e^n); planes outside the grid
// only complete their barrier phase
template <bool INCR, bool EFB>
__device__ void fwd_issue(const FwdMaps& mp, const Ring& r, int p, int kbeg, int kend, int nz,
                          int x0, int y0) {
  const uint32_t bar = r.bar(p), d = r.sat(p);
  uint32_t bytes = 0;
  const bool inside = p >= 0 && p < nz;
  const bool full = p >= kbeg && p < kend;
  const bool below = p == kbeg - 1;
  if (inside) bytes = (INCR ? (EFB ? 3 * kTxXY + kTxXY16 : 4 * kTxXY) : 2 * kTxXY) +
                      (full ? kTxX + kTxYm + kTxO : 0) + (below ? kTxO : 0);
  gemm::mbar_expect_tx(bar, bytes);
  if (!inside) return;
  tma3(d + FwdLayout::E, &mp.e, x0 - kHX, y0 - 1, p, bar);
  tma3(d + FwdLayout::M, &mp.m, x0 - kHX, y0 - 1, p, bar);
  if (INCR) {
    tma3(d + FwdLayout::DM, &mp.dm, x0 - kHX, y0 - 1, p, bar);
    tma3(d + FwdLayout::EF, &mp.ef, x0 - (EFB ? kHX16 : kHX), y0 - 1, p, bar);
  }
  if (full) {
    tma3(d + FwdLayout::VX, &mp.vx, x0 - kHX, y0, p, bar);
    tma3(d + FwdLayout::VY, &mp.vy, x0, y0 - 1, p, bar);
  }
  if (full || below) tma3(d + FwdLayout::VZ, &mp.vz, x0, y0, p, bar);
}

// e^n of float4 number q (element f) of the FP32 halo layout, from the EF box: FP32, or
// BF16 in the wider box (see kHX16)
template <bool EFB>
__device__ __forceinline__ float4 ef_at(const uint8_t* s, int q) {
  if (!EFB) return reinterpret_cast<const float4*>(s + FwdLayout::EF)[q];
  const uint2 b = reinterpret_cast<const uint2*>(s + FwdLayout::EF)[(q / kW4E) * (kWE16 / 4) +
                                                                    q % kW4E + (kHX16 - kHX) / 4];
  return make_float4(__uint_as_float(b.x << 16), __uint_as_float(b.x & 0xffff0000u),
                     __uint_as_float(b.y << 16), __uint_as_float(b.y & 0xffff0000u));
}
template <bool EFB>
__device__ __forceinline__ float ef_sc(const uint8_t* s, int f) {
  if (!EFB) return reinterpret_cast<const float*>(s + FwdLayout::EF)[f];
  const uint16_t b =
      reinterpret_cast<const uint16_t*>(s + FwdLayout::EF)[(f / kWE) * kWE16 + f % kWE + kHX16 - kHX];
  return __uint_as_float((uint32_t)b << 16);
}

// m e (+ dm e^n) of float4 number q of a halo box in stage s
template <bool INCR, bool EFB>
__device__ __forceinline__ float4 me_at(const uint8_t* s, int q) {
  float4 r = mul4(reinterpret_cast<const float4*>(s + FwdLayout::M)[q],
                  reinterpret_cast<const float4*>(s + FwdLayout::E)[q]);
  if (INCR) r = fma4(reinterpret_cast<const float4*>(s + FwdLayout::DM)[q], ef_at<EFB>(s, q), r);
  return r;
}
template <bool INCR, bool EFB>
__device__ __forceinline__ float me_sc(const uint8_t* s, int f) {
  float r = reinterpret_cast<const float*>(s + FwdLayout::M)[f] *
            reinterpret_cast<const float*>(s + FwdLayout::E)[f];
  if (INCR) r = fmaf(reinterpret_cast<const float*>(s + FwdLayout::DM)[f], ef_sc<EFB>(s, f), r);
  return r;
}

// PACK: the input state's block vectors, normalised by the maxima in a.bmax_in (known
// before the step: the step that wrote the state stored them), go out in one pass.
// MAXO: the maxima of the output state, reduced inside the CTA (which owns whole
// blocks: 128 x 8 nodes per plane, chunks of whole 8-plane layers) and stored whole.
template <bool INCR, bool PACK, bool MAXO, bool TPACK, bool EFB>
__global__ void __launch_bounds__(NTHR, (INCR || PACK) ? 2 : 3)
    fwd_tma_kernel(const __grid_constant__ FwdMaps mp, const FwdStep a) {
  constexpr int S = kStages;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  if (sticky_error(a.err)) return;

  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = blockIdx.x * kTXW, y0 = blockIdx.y * TY;
  const int i0 = x0 + 4 * lane, y = y0 + ty;
  const int kbeg = blockIdx.z * a.kc;
  const int kend = min(kbeg + a.kc, nz);
  const bool act = (i0 < nx) && (y < ny);
  const size_t P = (size_t)nx * ny;
  const size_t row = (size_t)y * nx + i0;
  const float dth = a.dth;

  Ring r;
  r.base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                      ~static_cast<uintptr_t>(127));
  r.bar0 = tc::smem_u32(&bars[0]);
  r.stage_bytes = FwdLayout::bytes(INCR);
  r.p0 = kbeg - 1;
  const int pn = kend;
  int next = r.p0;   // next plane to issue (thread 0)
  if (tid == 0) {
    for (int s = 0; s < S; ++s) tc::mbar_init(r.bar0 + 8u * s, 1);
    tc::mbar_fence_init();
    tc::fence_proxy_async();
    for (; next <= pn && next < r.p0 + S; ++next)
      fwd_issue<INCR, EFB>(mp, r, next, kbeg, kend, nz, x0, y0);
  }
  __syncthreads();

  // indices (float4 units) of this thread's nodes in the boxes
  const int qE = (ty + 1) * kW4E + 1 + lane;   // halo boxes, own row
  const int qX = ty * kW4E + 1 + lane;         // vx box
  const int qY = (ty + 1) * kW4 + lane;        // vy box, own row
  const int qO = ty * kW4 + lane;              // own-only boxes

  bool failed = false;
  float4 vzl = z4();
  // z-face below the chunk, recomputed exactly as its owner computes it
  if (!r.wait(r.p0)) failed = true;
  if (!r.wait(kbeg)) failed = true;
  failed = __syncthreads_or(failed);   // every thread takes the same path from here
  if (kbeg >= 1 && !failed) {
    const uint8_t* sb = r.at(r.p0);
    const uint8_t* sc = r.at(kbeg);
    vzl = fupd4(dth, me_at<INCR, EFB>(sc, qE), me_at<INCR, EFB>(sb, qE),
                reinterpret_cast<const float4*>(sb + FwdLayout::VZ)[qO]);
    add_source(vzl, kbeg - 1, y, i0, a);
  }

  const int NBx = nx >> 3, NBy = ny >> 3;
  uint8_t* pk = r.base + (size_t)S * r.stage_bytes;              // PACK: staging tiles
  float* red = reinterpret_cast<float*>(pk + (PACK ? kPackExtra : 0));   // MAXO
  float pm[4] = {0.f, 0.f, 0.f, 0.f};   // MAXO: this thread's output maxima
  float tm = 0.f;                       // TPACK: this thread's max |e^{n+1}| in the z pair
  // PACK: inverse scales of this lane's block in the current layer, and the maxima of
  // the next layer, loaded one layer ahead (lane / 2 is the block: 8 nodes = 2 lanes)
  float isc[4] = {0.f, 0.f, 0.f, 0.f};
  uint4 mnext = make_uint4(0u, 0u, 0u, 0u);
  const unsigned* bml = nullptr;
  if (PACK) {
    bml = a.bmax_in + (((size_t)(y0 >> 3) * NBx + (i0 >> 3)) << 2);
    if (act) mnext = __ldg(reinterpret_cast<const uint4*>(bml + (size_t)(kbeg >> 3) * NBy * NBx * 4));
  }
  // PACK copy-out: this warp writes the plane rows of blocks ty and ty + 8 of the CTA,
  // 16 bytes per lane; their addresses at plane kbeg, advanced by whole layers below
  const bool cp0 = (x0 >> 3) + ty < NBx, cp1 = (x0 >> 3) + ty + 8 < NBx;
  const size_t layer_bytes = (size_t)NBy * NBx * 4096;
  uint8_t* cpd = nullptr;
  if (PACK)
    cpd = reinterpret_cast<uint8_t*>(a.xpack) +
          (((size_t)(kbeg >> 3) * NBy + (y0 >> 3)) * NBx + (x0 >> 3) + ty) * 4096 + lane * 16;
  int k = kbeg;
  for (; k < kend && !failed; ++k) {
    if (PACK && (k & 7) == 0) {
      isc[0] = inv_scale_bits(mnext.x);
      isc[1] = inv_scale_bits(mnext.y);
      isc[2] = inv_scale_bits(mnext.z);
      isc[3] = inv_scale_bits(mnext.w);
      if (act && k + 8 < kend)
        mnext = __ldg(reinterpret_cast<const uint4*>(bml + (size_t)((k >> 3) + 1) * NBy * NBx * 4));
    }
    // plane k was waited for as plane k + 1 of the previous iteration (or before the loop)
    if (!r.wait(k + 1)) failed = true;
    const uint8_t* sc = r.at(k);
    const uint8_t* sn = r.at(k + 1);
    const size_t i = (size_t)k * P + row;

    const float4 e_c = reinterpret_cast<const float4*>(sc + FwdLayout::E)[qE];
    const float4 me_c = me_at<INCR, EFB>(sc, qE);
    const float4 me_yp = me_at<INCR, EFB>(sc, qE + kW4E);
    const float4 me_ym = me_at<INCR, EFB>(sc, qE - kW4E);
    const float4 me_n = me_at<INCR, EFB>(sn, qE);
    const float4 vx_c = reinterpret_cast<const float4*>(sc + FwdLayout::VX)[qX];
    const float4 vy_c = reinterpret_cast<const float4*>(sc + FwdLayout::VY)[qY];
    const float4 vy_m = reinterpret_cast<const float4*>(sc + FwdLayout::VY)[qY - kW4];
    const float4 vz_c = reinterpret_cast<const float4*>(sc + FwdLayout::VZ)[qO];

    if (PACK) {   // normalised BF16 block vectors of the input state
      if (act) {
        // this plane's piece of block (lane / 2): [field][y][x] in the staging tile.
        // x / s is exact in FP32 (s a power of two), so one rounding to BF16.
        uint8_t* dst = pk + (k & 1) * kPackTile + (lane >> 1) * kPackRow + ty * 16 + (lane & 1) * 8;
        const float4 fv[4] = {e_c, vx_c, vy_c, vz_c};
#pragma unroll
        for (int f = 0; f < 4; ++f)
          *reinterpret_cast<uint2*>(dst + f * 128) =
              make_uint2(pack2bf(fv[f].x * isc[f], fv[f].y * isc[f]),
                         pack2bf(fv[f].z * isc[f], fv[f].w * isc[f]));
      }
    }

    // x-faces of the own nodes; the face x+3 -> x+4 takes m e from the next lane
    float mx1 = __shfl_down_sync(0xffffffffu, me_c.x, 1);
    if (lane == 31) mx1 = me_sc<INCR, EFB>(sc, (ty + 1) * kWE + kHX + kTXW);
    float4 vx1;
    vx1.x = fupd(dth, me_c.y, me_c.x, vx_c.x);
    vx1.y = fupd(dth, me_c.z, me_c.y, vx_c.y);
    vx1.z = fupd(dth, me_c.w, me_c.z, vx_c.z);
    vx1.w = fupd(dth, mx1, me_c.w, vx_c.w);
    if (i0 + 4 == nx) vx1.w = 0.f;   // unused last face
    float vxl = __shfl_up_sync(0xffffffffu, vx1.w, 1);
    if (lane == 0) {
      vxl = 0.f;
      if (i0 >= 1)
        vxl = fupd(dth, me_c.x, me_sc<INCR, EFB>(sc, (ty + 1) * kWE + kHX - 1),
                   reinterpret_cast<const float*>(sc + FwdLayout::VX)[ty * kWE + kHX - 1]);
    }
    // y-faces: own, and the one below recomputed as the row below computes it
    float4 vy1 = fupd4(dth, me_yp, me_c, vy_c);
    if (y == ny - 1) vy1 = z4();
    float4 vyl = z4();
    if (y >= 1) vyl = fupd4(dth, me_c, me_ym, vy_m);
    // z-faces
    float4 vz1 = fupd4(dth, me_n, me_c, vz_c);
    if (k == nz - 1) vz1 = z4();
    add_source(vz1, k, y, i0, a);
    // strain update on interior nodes
    float4 e1;
    e1.x = fmaf(dth, ((vx1.x - vxl) + (vy1.x - vyl.x)) + (vz1.x - vzl.x), e_c.x);
    e1.y = fmaf(dth, ((vx1.y - vx1.x) + (vy1.y - vyl.y)) + (vz1.y - vzl.y), e_c.y);
    e1.z = fmaf(dth, ((vx1.z - vx1.y) + (vy1.z - vyl.z)) + (vz1.z - vzl.z), e_c.z);
    e1.w = fmaf(dth, ((vx1.w - vx1.z) + (vy1.w - vyl.w)) + (vz1.w - vzl.w), e_c.w);
    if (k == 0 || k == nz - 1 || y == 0 || y == ny - 1) {
      e1 = z4();
    } else {
      if (i0 == 0) e1.x = 0.f;
      if (i0 + 4 == nx) e1.w = 0.f;
    }
    if (act && !failed) {
      st4(a.e1, i, e1);
      st4(a.vx1, i, vx1);
      st4(a.vy1, i, vy1);
      st4(a.vz1, i, vz1);
      if (k == a.krec && a.d_out) {
        const int4 rm = __ldg(reinterpret_cast<const int4*>(a.rec_map + (size_t)y * nx + i0));
        const int rr[4] = {rm.x, rm.y, rm.z, rm.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (rr[c] >= 0) {
            a.d_out[3 * rr[c] + 0] = comp(vx1, c);
            a.d_out[3 * rr[c] + 1] = comp(vy1, c);
            a.d_out[3 * rr[c] + 2] = comp(vz1, c);
          }
        }
      }
    }
    vzl = vz1;
    if (TPACK) {
      // raw BF16 strain into its window slot: this lane pair holds one 8-node row of
      // vector (z pair k/2, y block, x block i0/8)
      if (act && !failed) {
        const size_t v = ((size_t)(k >> 1) * NBy + (y0 >> 3)) * NBx + (i0 >> 3);
        *reinterpret_cast<uint2*>(a.tpack + v * 2048 + a.tslot * 128 + (k & 1) * 64 + ty * 8 +
                                  (i0 & 7)) = make_uint2(pack2bf(e1.x, e1.y), pack2bf(e1.z, e1.w));
        tm = fmaxf(tm, hmax4(e1));
      }
      if (k & 1) {   // z pair complete: this row's maxima of its 16 vectors
        const float v = fmaxf(tm, __shfl_xor_sync(0xffffffffu, tm, 1));
        if ((lane & 1) == 0) red[ty * 16 + (lane >> 1)] = v;
        tm = 0.f;
      }
    }
    if (MAXO) {
      if (act) {
        pm[0] = fmaxf(pm[0], hmax4(e1));
        pm[1] = fmaxf(pm[1], hmax4(vx1));
        pm[2] = fmaxf(pm[2], hmax4(vy1));
        pm[3] = fmaxf(pm[3], hmax4(vz1));
      }
      if ((k & 7) == 7) {   // layer complete: this row's maxima of its 16 blocks
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const float v = fmaxf(pm[f], __shfl_xor_sync(0xffffffffu, pm[f], 1));
          if ((lane & 1) == 0) red[(ty * 16 + (lane >> 1)) * 4 + f] = v;
          pm[f] = 0.f;
        }
      }
    }
    // every thread is done with plane k: refill its stage
    failed = __syncthreads_or(failed);
    if (tid == 0 && !failed)
      for (; next <= pn && next <= k + S; ++next)
        fwd_issue<INCR, EFB>(mp, r, next, kbeg, kend, nz, x0, y0);
    if (MAXO && (k & 7) == 7 && !failed && tid < 64) {
      // the rows' tables are visible after the barrier; they are rewritten eight
      // planes (and barriers) later
      const int j = tid >> 2, f = tid & 3;
      float mx = 0.f;
#pragma unroll
      for (int w = 0; w < TY; ++w) mx = fmaxf(mx, red[(w * 16 + j) * 4 + f]);
      const size_t blk0 = ((size_t)(k >> 3) * NBy + (y0 >> 3)) * NBx + (x0 >> 3);
      if ((x0 >> 3) + j < NBx) a.bmax_out[(blk0 + j) * 4 + f] = __float_as_uint(mx);
    }
    if (TPACK && (k & 1) && !failed && tid < 16) {
      // the rows' maxima are visible after the barrier; rewritten two planes later
      float mx = 0.f;
#pragma unroll
      for (int w = 0; w < TY; ++w) mx = fmaxf(mx, red[w * 16 + tid]);
      const size_t v = ((size_t)(k >> 1) * NBy + (y0 >> 3)) * NBx + (x0 >> 3) + tid;
      if ((x0 >> 3) + tid < NBx && mx > 0.f) atomicMax(a.vmax + v, __float_as_uint(mx));
    }
    if (PACK && !failed) {
      // plane k of the CTA's 16 blocks: one coalesced 512-byte row per block (the tile
      // is rewritten two planes later, after the next barrier)
      static_assert(kTXW / 8 == 2 * TY, "two block rows per warp");
      const uint8_t* src = pk + (k & 1) * kPackTile + ty * kPackRow + lane * 16;
      uint8_t* dst = cpd + (size_t)((k - kbeg) >> 3) * layer_bytes + (k & 7) * 512;
      if (cp0) *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
      if (cp1)
        *reinterpret_cast<uint4*>(dst + 8 * 4096) =
            *reinterpret_cast<const uint4*>(src + 8 * kPackRow);
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      // let the copies still in flight land before the shared memory is released
      for (int p = max(r.p0, next - S); p < next; ++p) r.wait(p);
    }
  }
}

// ---------------------------------------------------------------------------------
// Adjoint step
// ---------------------------------------------------------------------------------
struct AdjFlags {
  bool en, w;   // e^n present; FP32 window accumulator read
  bool enb;     // e^n given as BF16 (its box carries half the bytes)
};

__device__ void adj_issue(const AdjMaps& mp, const Ring& r, int p, int kbeg, int kend, int nz,
                          int x0, int y0, AdjFlags f) {
  const uint32_t bar = r.bar(p), d = r.sat(p);
  uint32_t bytes = 0;
  const bool inside = p >= 0 && p < nz;
  const bool full = p >= kbeg && p < kend;
  const bool below = p == kbeg - 1;
  if (inside)
    bytes = kTxXY +
            (full ? kTxX + kTxYm + kTxO * (2 + (f.w ? 1 : 0)) + (f.en ? (f.enb ? kTxO / 2 : kTxO) : 0)
                  : 0) +
            (below ? kTxO : 0);
  gemm::mbar_expect_tx(bar, bytes);
  if (!inside) return;
  tma3(d + AdjLayout::MU, &mp.mu, x0 - kHX, y0 - 1, p, bar);
  if (full) {
    tma3(d + AdjLayout::LX, &mp.lx, x0 - kHX, y0, p, bar);
    tma3(d + AdjLayout::LY, &mp.ly, x0, y0 - 1, p, bar);
    tma3(d + AdjLayout::M, &mp.m, x0, y0, p, bar);
    if (f.en) tma3(d + AdjLayout::EN, &mp.en, x0, y0, p, bar);
    if (f.w) tma3(d + AdjLayout::W, &mp.w, x0, y0, p, bar);
  }
  if (full || below) tma3(d + AdjLayout::LZ, &mp.lz, x0, y0, p, bar);
}

__device__ __forceinline__ float inj_one(const AdjStep& a, int comp3, int x, int y, int k) {
  if (k != a.krec || a.resid == nullptr) return 0.f;
  const int q = __ldg(a.rec_map + (size_t)y * a.nx + x);
  return q >= 0 ? __ldg(a.resid + 3 * q + comp3) : 0.f;
}
// add B^T r to the three face fields of a float4 of nodes on the receiver plane
__device__ __forceinline__ void inj4(const AdjStep& a, int y, int i0, float4& lx, float4& ly,
                                     float4& lz) {
  const int4 q = __ldg(reinterpret_cast<const int4*>(a.rec_map + (size_t)y * a.nx + i0));
  const int rr[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if (rr[c] >= 0) {
      comp(lx, c) += __ldg(a.resid + 3 * rr[c] + 0);
      comp(ly, c) += __ldg(a.resid + 3 * rr[c] + 1);
      comp(lz, c) += __ldg(a.resid + 3 * rr[c] + 2);
    }
  }
}

// V bit 0: write dt q to a.qout; bit 1: add a.dm2 * a.qin to the mu update (full Newton
// HVP: the first-order adjoint writes its dt q, the second-order adjoint reads it)
template <int V>
__global__ void __launch_bounds__(NTHR, 2)
    adj_tma_kernel(const __grid_constant__ AdjMaps mp, const AdjStep a) {
  constexpr int S = kStages;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[kStages];
  if (sticky_error(a.err)) return;

  const int lane = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + lane;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x0 = blockIdx.x * kTXW, y0 = blockIdx.y * TY;
  const int i0 = x0 + 4 * lane, y = y0 + ty;
  const int kbeg = blockIdx.z * a.kc;
  const int kend = min(kbeg + a.kc, nz);
  const bool act = (i0 < nx) && (y < ny);
  const size_t P = (size_t)nx * ny;
  const size_t row = (size_t)y * nx + i0;
  const float dth = a.dth;
  const bool has_r = a.resid != nullptr && a.krec >= 0;
  const int mode = a.acc_mode;
  const AdjFlags fl{a.en != nullptr || a.en16 != nullptr, !(mode & kAccFirst), a.en16 != nullptr};

  Ring r;
  r.base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                      ~static_cast<uintptr_t>(127));
  r.bar0 = tc::smem_u32(&bars[0]);
  r.stage_bytes = AdjLayout::BYTES;
  r.p0 = kbeg - 1;
  const int pn = kend;
  int next = r.p0;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) tc::mbar_init(r.bar0 + 8u * s, 1);
    tc::mbar_fence_init();
    tc::fence_proxy_async();
    for (; next <= pn && next < r.p0 + S; ++next) adj_issue(mp, r, next, kbeg, kend, nz, x0, y0, fl);
  }
  __syncthreads();

  const int qE = (ty + 1) * kW4E + 1 + lane;
  const int qX = ty * kW4E + 1 + lane;
  const int qY = (ty + 1) * kW4 + lane;
  const int qO = ty * kW4 + lane;

  bool failed = false;
  float4 lzl = z4();
  if (!r.wait(r.p0)) failed = true;
  if (!r.wait(kbeg)) failed = true;
  failed = __syncthreads_or(failed);
  if (kbeg >= 1 && !failed) {
    const uint8_t* sb = r.at(r.p0);
    const uint8_t* sc = r.at(kbeg);
    float4 lzm = reinterpret_cast<const float4*>(sb + AdjLayout::LZ)[qO];
    if (has_r && kbeg - 1 == a.krec && act) {
      float4 dx = z4(), dy = z4();
      inj4(a, y, i0, dx, dy, lzm);
    }
    lzl = lupd4(dth, reinterpret_cast<const float4*>(sc + AdjLayout::MU)[qE],
                reinterpret_cast<const float4*>(sb + AdjLayout::MU)[qE], lzm);
  }

  int k = kbeg;
  for (; k < kend && !failed; ++k) {
    const size_t i = (size_t)k * P + row;
    // the FP64 accumulator of a window's last step: in flight while the planes land
    double2 a64lo = make_double2(0.0, 0.0), a64hi = a64lo;
    if ((mode & kAccLast) && act) {
      const double2* p64 = reinterpret_cast<const double2*>(a.acc64 + i);
      a64lo = p64[0];
      a64hi = p64[1];
    }
    // second-order source dm2 * qin of the own nodes, in flight while the planes land
    float4 src2 = z4();
    if ((V & 2) && act) src2 = mul4(__ldg(reinterpret_cast<const float4*>(a.dm2 + i)),
                                     __ldg(reinterpret_cast<const float4*>(a.qin + i)));
    // plane k was waited for as plane k + 1 of the previous iteration (or before the loop)
    if (!r.wait(k + 1)) failed = true;
    const uint8_t* sc = r.at(k);
    const uint8_t* sn = r.at(k + 1);
    const float4* MU = reinterpret_cast<const float4*>(sc + AdjLayout::MU);
    const float4 mu_c = MU[qE];
    const float4 mu_yp = MU[qE + kW4E];
    const float4 mu_ym = MU[qE - kW4E];
    const float4 mu_n = reinterpret_cast<const float4*>(sn + AdjLayout::MU)[qE];
    float4 lx_c = reinterpret_cast<const float4*>(sc + AdjLayout::LX)[qX];
    float4 ly_c = reinterpret_cast<const float4*>(sc + AdjLayout::LY)[qY];
    float4 ly_m = reinterpret_cast<const float4*>(sc + AdjLayout::LY)[qY - kW4];
    float4 lz_c = reinterpret_cast<const float4*>(sc + AdjLayout::LZ)[qO];
    const float4 m4 = reinterpret_cast<const float4*>(sc + AdjLayout::M)[qO];
    float4 en4 = z4();
    if (fl.enb) {   // 4 BF16 values, element 0 in the low half
      const uint2 b = reinterpret_cast<const uint2*>(sc + AdjLayout::EN)[qO];
      en4 = make_float4(__uint_as_float(b.x << 16), __uint_as_float(b.x & 0xffff0000u),
                        __uint_as_float(b.y << 16), __uint_as_float(b.y & 0xffff0000u));
    } else if (fl.en) {
      en4 = reinterpret_cast<const float4*>(sc + AdjLayout::EN)[qO];
    }
    const float4 w_c = fl.w ? reinterpret_cast<const float4*>(sc + AdjLayout::W)[qO] : z4();

    const bool rplane = has_r && k == a.krec;
    if (rplane && act) inj4(a, y, i0, lx_c, ly_c, lz_c);

    float mx1 = __shfl_down_sync(0xffffffffu, mu_c.x, 1);
    if (lane == 31)
      mx1 = reinterpret_cast<const float*>(sc + AdjLayout::MU)[(ty + 1) * kWE + kHX + kTXW];
    float4 lx1;
    lx1.x = lupd(dth, mu_c.y, mu_c.x, lx_c.x);
    lx1.y = lupd(dth, mu_c.z, mu_c.y, lx_c.y);
    lx1.z = lupd(dth, mu_c.w, mu_c.z, lx_c.z);
    lx1.w = lupd(dth, mx1, mu_c.w, lx_c.w);
    if (i0 + 4 == nx) lx1.w = 0.f;
    float lxl = __shfl_up_sync(0xffffffffu, lx1.w, 1);
    if (lane == 0) {
      lxl = 0.f;
      if (act && i0 >= 1) {
        float l = reinterpret_cast<const float*>(sc + AdjLayout::LX)[ty * kWE + kHX - 1];
        if (rplane) l += inj_one(a, 0, i0 - 1, y, k);
        lxl = lupd(dth, mu_c.x,
                   reinterpret_cast<const float*>(sc + AdjLayout::MU)[(ty + 1) * kWE + kHX - 1], l);
      }
    }
    float4 ly1 = lupd4(dth, mu_yp, mu_c, ly_c);
    if (y == ny - 1) ly1 = z4();
    float4 lyl = z4();
    if (act && y >= 1) {
      if (rplane) {
        ly_m.x += inj_one(a, 1, i0 + 0, y - 1, k);
        ly_m.y += inj_one(a, 1, i0 + 1, y - 1, k);
        ly_m.z += inj_one(a, 1, i0 + 2, y - 1, k);
        ly_m.w += inj_one(a, 1, i0 + 3, y - 1, k);
      }
      lyl = lupd4(dth, mu_c, mu_ym, ly_m);
    }
    float4 lz1 = lupd4(dth, mu_n, mu_c, lz_c);
    if (k == nz - 1) lz1 = z4();
    // dt q = dt G^T lam' = -dt/h (div lam') on interior nodes
    float4 dq;
    dq.x = -dth * (((lx1.x - lxl) + (ly1.x - lyl.x)) + (lz1.x - lzl.x));
    dq.y = -dth * (((lx1.y - lx1.x) + (ly1.y - lyl.y)) + (lz1.y - lzl.y));
    dq.z = -dth * (((lx1.z - lx1.y) + (ly1.z - lyl.z)) + (lz1.z - lzl.z));
    dq.w = -dth * (((lx1.w - lx1.z) + (ly1.w - lyl.w)) + (lz1.w - lzl.w));
    if (k == 0 || k == nz - 1 || y == 0 || y == ny - 1) {
      dq = z4();
    } else {
      if (i0 == 0) dq.x = 0.f;
      if (i0 + 4 == nx) dq.w = 0.f;
    }
    // boundary nodes: mu_c, dq and (written as 0 there) qin are all 0
    const float4 mu1 = (V & 2) ? fma4(m4, dq, make_float4(mu_c.x + src2.x, mu_c.y + src2.y,
                                                         mu_c.z + src2.z, mu_c.w + src2.w))
                               : fma4(m4, dq, mu_c);
    if (act && !failed) {
      if (V & 1) st4(a.qout, i, dq);
      st4(a.mu1, i, mu1);
      st4(a.lx1, i, lx1);
      st4(a.ly1, i, ly1);
      st4(a.lz1, i, lz1);
      // dJ/dm += dt e^n q
      const float4 g = mul4(en4, dq);
      if (mode & kAccLast) {
        float4 s = g;
        if (fl.w) s = make_float4(w_c.x + g.x, w_c.y + g.y, w_c.z + g.z, w_c.w + g.w);
        a64lo.x += (double)s.x;
        a64lo.y += (double)s.y;
        a64hi.x += (double)s.z;
        a64hi.y += (double)s.w;
        double2* p64 = reinterpret_cast<double2*>(a.acc64 + i);
        p64[0] = a64lo;
        p64[1] = a64hi;
      } else if (mode & kAccFirst) {
        st4(a.acc32, i, g);
      } else {
        st4(a.acc32, i, make_float4(w_c.x + g.x, w_c.y + g.y, w_c.z + g.z, w_c.w + g.w));
      }
    }
    lzl = lz1;
    failed = __syncthreads_or(failed);
    if (tid == 0 && !failed)
      for (; next <= pn && next <= k + S; ++next) adj_issue(mp, r, next, kbeg, kend, nz, x0, y0, fl);
  }
  if (failed) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      for (int p = max(r.p0, next - S); p < next; ++p) r.wait(p);
    }
  }
}

// Failure-path probe: one thread waits, with the given bound, on an mbarrier that
// nothing arrives at, and records the time-out exactly as the stencil and codec kernels
// record theirs.
__global__ void wait_probe_kernel(int* err, uint64_t ns) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = tc::smem_u32(&bar);
  tc::mbar_init(b, 1);
  tc::mbar_fence_init();
  if (!tc::mbar_wait(b, 0, ns)) atomicExch(err, 1);
  // complete the phase so the barrier is not left pending when the CTA exits
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
// 3-D tensor map of an FP32 field [nz][ny][nx] with a (bx, by, 1) box; zero fill
// outside the grid
bool field_map(CUtensorMap* map, const float* base, int nx, int ny, int nz, int bx, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = gemm::tensor_map_encoder();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the same for a BF16 field (nx a multiple of 8: the row stride a multiple of 16 bytes;
// the boxes start at x multiples of 128)
bool field_map16(CUtensorMap* map, const uint16_t* base, int nx, int ny, int nz, int bx, int by) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = gemm::tensor_map_encoder();
  if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) || (nx % 8)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 2, (cuuint64_t)nx * ny * 2};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(base), dims, strides,
             box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

dim3 grid_of(int nx, int ny, int nz, int kc) {
  return dim3((nx + kTXW - 1) / kTXW, (ny + TY - 1) / TY, (nz + kc - 1) / kc);
}

template <bool INCR, bool PACK, bool MAXO, bool TPACK = false, bool EFB = false>
cudaError_t launch_fwd(const FwdMaps& mp, const FwdStep& a, cudaStream_t s) {
  const int extra = (PACK ? kPackExtra : 0) + ((MAXO || TPACK) ? kMaxoExtra : 0) + 128;
  const size_t smem = (size_t)kStages * FwdLayout::bytes(INCR) + extra;
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      fwd_tma_kernel<INCR, PACK, MAXO, TPACK, EFB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)smem);
  if (attr != cudaSuccess) return attr;
  fwd_tma_kernel<INCR, PACK, MAXO, TPACK, EFB>
      <<<grid_of(a.nx, a.ny, a.nz, a.kc), dim3(32, TY), smem, s>>>(mp, a);
  return cudaGetLastError();
}

template <int V>
cudaError_t launch_adj(const AdjMaps& mp, const AdjStep& a, cudaStream_t s) {
  const size_t smem = (size_t)kStages * AdjLayout::BYTES + 128;
  // once per instantiation (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(
      adj_tma_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  adj_tma_kernel<V><<<grid_of(a.nx, a.ny, a.nz, a.kc), dim3(32, TY), smem, s>>>(mp, a);
  return cudaGetLastError();
}

}  // namespace

int default_kc(int nx, int ny, int nz, bool adjoint) {
  // z planes per CTA: short chunks give many CTAs (several waves, good balance) at the
  // cost of staging one plane below and one above each chunk.  Measured at 256^3 on
  // GB300: 6 for the forward steps (plain 98.2 us against 100.2 with 8; the window-packing
  // step 107.1 against 109.6), 8 for the adjoint (129.8 us; 130.4 with 6, 131.0 with 12).
  // The space codec's packing step rounds it up to whole 8-plane block layers, the time
  // codec's to whole plane pairs.
  (void)nx;
  (void)ny;
  const int want = adjoint ? 8 : 6;
  int kc = nz < want ? nz : want;
  if (const char* env = getenv(adjoint ? "AEW_STENCIL_KC_ADJ" : "AEW_STENCIL_KC_FWD")) {
    const int v = atoi(env);   // tuning override
    if (v > 0) kc = v;
  }
  return kc < 1 ? 1 : kc;
}

// z planes per CTA of the packing step (whole 8-plane layers; default 16)
static int pack_kc() {
  static const int v = [] {
    const char* env = getenv("AEW_STENCIL_KC_PACK");   // tuning override
    return env ? atoi(env) : 16;
  }();
  return v > 0 ? v : 16;
}

cudaError_t launch_fwd_step(const FwdStep& a, bool incremental, cudaStream_t s) {
  if (!a.err) return cudaErrorInvalidValue;
  FwdMaps mp;
  memset(&mp, 0, sizeof(mp));
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  bool ok = field_map(&mp.e, a.e, nx, ny, nz, kWE, TY + 2) &&
            field_map(&mp.m, a.m, nx, ny, nz, kWE, TY + 2) &&
            field_map(&mp.vx, a.vx, nx, ny, nz, kWE, TY) &&
            field_map(&mp.vy, a.vy, nx, ny, nz, kTXW, TY + 1) &&
            field_map(&mp.vz, a.vz, nx, ny, nz, kTXW, TY);
  if (incremental && a.ef && a.ef16) return cudaErrorInvalidValue;
  if (ok && incremental)
    ok = field_map(&mp.dm, a.dm, nx, ny, nz, kWE, TY + 2) &&
         (a.ef16 ? field_map16(&mp.ef, a.ef16, nx, ny, nz, kWE16, TY + 2)
                 : field_map(&mp.ef, a.ef, nx, ny, nz, kWE, TY + 2));
  if (!ok) return cudaErrorInvalidValue;
  if (incremental && a.tpack) {
    if (nx % 8 || ny % 8 || nz % 2 || !a.vmax || a.tslot < 0 || a.tslot >= 16)
      return cudaErrorInvalidValue;
    FwdStep b = a;
    b.kc = (a.kc + 1) / 2 * 2;
    if (a.ef16) return launch_fwd<true, false, false, true, true>(mp, b, s);
    return launch_fwd<true, false, false, true>(mp, b, s);
  }
  if (incremental && a.ef16) return launch_fwd<true, false, false, false, true>(mp, a, s);
  if (incremental) return launch_fwd<true, false, false>(mp, a, s);
  if (a.tpack) {
    // window packing works on 2 x 8 x 8-node blocks: whole z pairs inside one CTA
    if (nx % 8 || ny % 8 || nz % 2 || !a.vmax || a.xpack || a.bmax_out || a.tslot < 0 ||
        a.tslot >= 16)
      return cudaErrorInvalidValue;
    FwdStep b = a;
    b.kc = (a.kc + 1) / 2 * 2;
    return launch_fwd<false, false, false, true>(mp, b, s);
  }
  if (a.xpack || a.bmax_out) {
    // block maxima and packing work on whole 8 x 8 x 8 blocks inside one CTA
    if (nx % 8 || ny % 8 || nz % 8) return cudaErrorInvalidValue;
    if (a.xpack && !a.bmax_in) return cudaErrorInvalidValue;
    FwdStep b = a;
    b.kc = ((a.xpack ? pack_kc() : a.kc) + 7) / 8 * 8;
    if (!a.xpack) return launch_fwd<false, false, true>(mp, b, s);
    if (!a.bmax_out) return launch_fwd<false, true, false>(mp, b, s);
    return launch_fwd<false, true, true>(mp, b, s);
  }
  return launch_fwd<false, false, false>(mp, a, s);
}

cudaError_t launch_wait_probe(int* err, unsigned long long wait_ns, cudaStream_t s) {
  if (!err) return cudaErrorInvalidValue;
  wait_probe_kernel<<<1, 1, 0, s>>>(err, wait_ns);
  return cudaGetLastError();
}

cudaError_t launch_adj_step(const AdjStep& a, cudaStream_t s) {
  if (!a.err) return cudaErrorInvalidValue;
  AdjMaps mp;
  memset(&mp, 0, sizeof(mp));
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  bool ok = field_map(&mp.mu, a.mu, nx, ny, nz, kWE, TY + 2) &&
            field_map(&mp.lx, a.lx, nx, ny, nz, kWE, TY) &&
            field_map(&mp.ly, a.ly, nx, ny, nz, kTXW, TY + 1) &&
            field_map(&mp.lz, a.lz, nx, ny, nz, kTXW, TY) &&
            field_map(&mp.m, a.m, nx, ny, nz, kTXW, TY);
  if (a.en && a.en16) return cudaErrorInvalidValue;
  if (ok && a.en) ok = field_map(&mp.en, a.en, nx, ny, nz, kTXW, TY);
  if (ok && a.en16) ok = field_map16(&mp.en, a.en16, nx, ny, nz, kTXW, TY);
  if (ok && !(a.acc_mode & kAccFirst)) ok = field_map(&mp.w, a.acc32, nx, ny, nz, kTXW, TY);
  if (!ok) return cudaErrorInvalidValue;
  if ((a.qin != nullptr) != (a.dm2 != nullptr)) return cudaErrorInvalidValue;
  const int V = (a.qout ? 1 : 0) | (a.qin ? 2 : 0);
  switch (V) {
    case 0: return launch_adj<0>(mp, a, s);
    case 1: return launch_adj<1>(mp, a, s);
    case 2: return launch_adj<2>(mp, a, s);
    default: return launch_adj<3>(mp, a, s);
  }
}

}  // namespace aew
