// Internal declarations shared by the translation units of the aewave library.
// Nothing here is part of the public C ABI (include/aewave.h).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace aew {

// x cells handled by one CTA row (32 lanes x float4)
constexpr int kTXW = 128;

// ------------------------------------------------------------------------------
// Forward-type leapfrog step (forward solve and incremental forward solve).
//   v' = v + dt/h (me[+1] - me) (+ dt s at the source z-face),
//   e' = interior ? e + dt/h (div of v') : 0,
// with me = m*e (forward) or m*e + dm*ef (incremental forward, no source).
// ------------------------------------------------------------------------------
struct FwdStep {
  const float* m;
  const float* e;
  const float* vx;
  const float* vy;
  const float* vz;
  float* e1;
  float* vx1;
  float* vy1;
  float* vz1;
  const float* dm;   // incremental only
  const float* ef;   // incremental only: forward strain e^n
  const uint16_t* ef16;  // or e^n as BF16 (a decoded window; nx a multiple of 8)
  int nx, ny, nz;
  int kc;            // z planes per CTA
  float dth;         // dt / h
  float dts;         // dt * s^n added to the source z-face(s)
  int si, sj, sk;    // source node (sk < 0: none)
  // the source's spread: faces |i - si|, |y - sj|, |k - sk| <= sr get dts times
  // src_w[(k - sk + sr)][(y - sj + sr)][(i - si + sr)] (a point source: sr = 0, {1})
  const float* src_w;
  int sr;
  int krec;          // receiver node plane (-1: none)
  const int* rec_map;  // [ny][nx] receiver index or -1
  float* d_out;        // receiver record row [nrec][3] (or null)
  // Optional packing of the INPUT state n into normalised BF16 block vectors
  // [nblocks][2048] (order z*256 + f*64 + y*8 + x; every field of every block divided by
  // its power-of-two scale), with the per-block, per-field maxima of |f| of that state
  // (float bits, bmax_in[nblocks][4]) as the step that produced it stored them.
  uint16_t* xpack;
  const unsigned int* bmax_in;
  // Optional: the per-block, per-field maxima of |f| of the OUTPUT state n + 1 (float
  // bits, bmax_out[nblocks][4], every entry written).  Must not alias bmax_in.
  unsigned int* bmax_out;
  // Both options need nx, ny, nz multiples of 8.
  // Optional (compression in time): the OUTPUT strain e^{n+1} as raw BF16 into slot
  // tslot of a window of strain vectors tpack[nvec][2048] (2 x 8 x 8-node blocks,
  // order t*128 + z*64 + y*8 + x, vector (bz*NBy + by)*NBx + bx), and the largest
  // |e^{n+1}| of each vector folded into vmax[nvec] (float bits, atomicMax).  Needs nx,
  // ny multiples of 8 and nz even.
  uint16_t* tpack;
  unsigned* vmax;
  int tslot;
  int* err;            // sticky device error flag (set on a timed-out wait)
};

// ------------------------------------------------------------------------------
// Adjoint step (reverse of one forward step) with gradient accumulation.
//   lam' = lam + B^T r - dt/h (mu[+1] - mu),
//   dtq  = interior ? -dt/h (div of lam') : 0          (= dt * G^T lam')
//   mu'  = interior ? mu + m * dtq : 0,
//   acc += e^n * dtq                                   (FP32 window, FP64 flush)
// ------------------------------------------------------------------------------
struct AdjStep {
  const float* m;
  const float* mu;
  const float* lx;
  const float* ly;
  const float* lz;
  float* mu1;
  float* lx1;
  float* ly1;
  float* lz1;
  const float* en;     // forward strain e^n (null: zero)
  const uint16_t* en16;  // or e^n as BF16 (a decoded window; nx a multiple of 8)
  float* acc32;        // FP32 window accumulator
  double* acc64;       // FP64 accumulator
  int acc_mode;        // bit0: first step of a window, bit1: last step of a window
  int nx, ny, nz;
  int kc;
  float dth;
  int krec;
  const int* rec_map;
  const float* resid;  // residual row r^{n+1} [nrec][3] (or null)
  // Full Newton HVP (both optional): qout receives this step's dt q (0 on boundary
  // nodes); with qin and dm2 the mu update gains the second-order adjoint's source:
  //   mu' = interior ? mu + m dtq + dm2 qin : 0   (qin = the first-order adjoint's dt q)
  float* qout;
  const float* qin;
  const float* dm2;
  int* err;            // sticky device error flag (set on a timed-out wait)
};

enum { kAccFirst = 1, kAccLast = 2 };

// TMA-staged steps (aew_stencil.cu); every field pointer must be 16-byte aligned
cudaError_t launch_fwd_step(const FwdStep& a, bool incremental, cudaStream_t s);
cudaError_t launch_adj_step(const AdjStep& a, cudaStream_t s);
// one bounded wait that nothing completes: sets *err after wait_ns (failure-path test)
cudaError_t launch_wait_probe(int* err, unsigned long long wait_ns, cudaStream_t s);
int default_kc(int nx, int ny, int nz, bool adjoint);

// ------------------------------------------------------------------------------
// Reductions and elementwise helpers (aew_reduce.cu)
// ------------------------------------------------------------------------------
struct FieldCheck {
  unsigned int nonfinite;
  unsigned int cmax_bits;   // max c as float bits (c >= 0 expected)
  unsigned int cneg;        // count of c <= 0
};
// m = c^2 and checks; writes *chk (device)
cudaError_t launch_prep_m(const float* c, float* m, size_t n, FieldCheck* chk, cudaStream_t s);
// dm = 2 c dc and checks of dc
cudaError_t launch_prep_dm(const float* c, const float* dc, float* dm, size_t n,
                           FieldCheck* chk, cudaStream_t s);
// r = d - d_obs (rows 1..nt; row 0 zero); FP64 partial sums of r^2 into part[nblk]
cudaError_t launch_residual(const float* d, const float* dobs, float* r, size_t n_row0,
                            size_t n, double* part, int nblk, cudaStream_t s);
// FP64 partial dot products of a and b into part[nblk]
cudaError_t launch_dot_partials(const float* a, const float* b, size_t n, double* part,
                                int nblk, cudaStream_t s);
// out[0] = scale * sum part[0..nblk)
cudaError_t launch_sum_partials(const double* part, int nblk, double scale, double* out,
                                cudaStream_t s);
// g = 2 c acc64 (FP32 output)
cudaError_t launch_finalize_grad(const float* c, const double* acc64, float* g, size_t n,
                                 cudaStream_t s);
// out = 2 c (a + b) + (dc / c) g  (full Newton HVP from its two accumulators and the
// gradient g of the same c)
cudaError_t launch_finalize_hvp_full(const float* c, const float* dc, const double* a,
                                     const double* b, const float* g, float* out, size_t n,
                                     cudaStream_t s);
constexpr int kRedBlocks = 1024;

}  // namespace aew
