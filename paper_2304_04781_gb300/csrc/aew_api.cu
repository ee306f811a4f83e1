// C-ABI of the aewave library: handle lifetime, the forward / adjoint / incremental
// time loops, the three history-storage modes and the checkpointing executor.
//
// Everything runs on the caller's stream; the host only sequences kernel launches.
// Operations (see include/aewave.h): forward solve d = B A(c) (Sec. 2), gradient of the
// misfit of Eq. (3), Gauss-Newton Hessian-vector product via the incremental forward
// and incremental adjoint problems (Sec. 4), with the forward history either stored,
// recomputed from binomial checkpoints (Sec. 1), or compressed to autoencoder latents
// once per gradient and decoded by every later adjoint-type solve (Sec. 3, Sec. 4).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aewave.h"
#include "aew_codec.cuh"
#include "aew_internal.cuh"
#include "aew_pca.h"
#include "aew_revolve.h"
#include "aew_solver.h"

using aew::Codec;

struct aew_handle {
  aew_config cfg{};
  std::vector<int> rec;
  int krec = -1;
  int device = 0;
  double dt = 0.0;
  float dth = 0.f;
  size_t C = 0;
  int kc = 1;       // z planes per CTA, forward-type steps
  int kc_adj = 1;   // z planes per CTA, adjoint steps
  size_t nrow = 0;   // nrec * 3
  std::string err;
  aew_stats_t stats{};

  float* c = nullptr;
  float* m = nullptr;
  float* dm = nullptr;
  float* st[2][4] = {};
  float* ad[2][4] = {};
  float* acc32 = nullptr;
  double* acc64 = nullptr;
  float* estore = nullptr;
  float* ckpt = nullptr;
  float* zst[4] = {};   // REVOLVE: the zero initial state
  uint16_t* lat = nullptr;
  unsigned* bmx = nullptr;   // AE: per step, block and field max |f| (float bits) [nt][nb][4]
  int* ovf = nullptr;
  float* d = nullptr;
  float* R = nullptr;
  float* dd = nullptr;
  int* rec_map = nullptr;
  double* part = nullptr;
  aew::FieldCheck* chk = nullptr;
  float* scratch8 = nullptr;     // 8 words: training loss, encode overflow flag
  unsigned* bm_tmp = nullptr;    // block maxima of a standalone encode / a snapshot (2 slices)
  // AE mode: side stream running the codec GEMMs concurrently with the stencil steps,
  // double-buffered packed inputs and decoded strains, and the events ordering them
  cudaStream_t side = nullptr;
  int overlap_ctas = 0;   // CTA cap of the codec GEMMs that run beside a stencil step
  cudaEvent_t ev_a[2] = {}, ev_b[2] = {}, ev_sync = nullptr, ev_sync2 = nullptr;
  uint16_t* xpk[2] = {};
  float* edb[2] = {};
  // AE mode with the time codec: per window and vector the max |e| (float bits)
  // [nwin][nvec], raw BF16 window vectors being filled / encoded, decoded windows of
  // 16 strain slices, and a window workspace of the standalone codec calls
  bool tcodec = false;
  unsigned* vmx = nullptr;
  uint16_t* xt[2] = {};
  float* edt[2] = {};
  uint16_t* wk_raw = nullptr;
  unsigned* wk_vmax = nullptr;
  // min-max normalisation (time codec): each window vector's offset and range (FP64
  // [nwin][nvec]) of the forward strain and (full Newton HVP) the incremental strain
  double* wmn = nullptr;
  double* wr = nullptr;
  double* wmn2 = nullptr;
  double* wr2 = nullptr;
  double* wk_mr = nullptr;   // standalone window calls: [2][nvec]
  // full Newton HVP: the last gradient (FP32, for its 2 dc dJ/dm term), the second-order
  // adjoint's states and accumulators, the first-order adjoint's dt q, and the
  // incremental strain history (FP32 for full storage; latents of the time codec)
  float* gc = nullptr;
  bool nw_ready = false;
  float* ad2[2][4] = {};
  float* acc32b = nullptr;
  double* acc64b = nullptr;
  float* qbuf = nullptr;
  float* desto = nullptr;
  uint16_t* lat2 = nullptr;
  unsigned* vmx2 = nullptr;
  float* edt2[2] = {};
  cudaEvent_t ev_c[2] = {}, ev_d[2] = {};
  // device timing of the last gradient and hessvec (read lazily by aew_stats)
  cudaEvent_t tg[2] = {}, th[2] = {};
  bool tg_set = false, th_set = false;
  std::vector<float> wav;
  bool have_grad = false;
  // Armijo gate of a gradient run by the Newton driver: stop after the forward solve
  // when the misfit exceeds it (+inf: never)
  double gate = INFINITY;
  // the source's spatial weights on the z-faces of a (2 src_r + 1)^3 box (point: {1})
  float* src_w = nullptr;
  int src_r = 0;
  Codec* codec = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
};

namespace {

thread_local std::string g_create_err;

int fail(aew_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(aew_handle* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, AEW_E_CUDA, m);
}

#define AEW_CK(expr)                                     \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(h, _e, #expr); \
  } while (0)

template <class T>
bool dalloc(aew_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return true;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->allocs.push_back(q);
  h->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return true;
}

double ricker(double t, double f0, double t0) {
  const double sig = 1.0 / (std::sqrt(2.0) * M_PI * f0);
  const double tau = t - t0;
  return (1.0 - tau * tau / (sig * sig)) * std::exp(-tau * tau / (2.0 * sig * sig));
}

cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

size_t nblocks_of(const aew_handle* h) {
  return (size_t)(h->cfg.nx / 8) * (h->cfg.ny / 8) * (h->cfg.nz / 8);
}

// time codec: vectors per window (2 x 8 x 8-node blocks) and windows covering e^0..e^{nt-1}
size_t nvec_of(const aew_handle* h) {
  return (size_t)(h->cfg.nx / 8) * (h->cfg.ny / 8) * (h->cfg.nz / 2);
}
int nwin_of(const aew_handle* h) { return (h->cfg.nt + aew::kTSteps - 1) / aew::kTSteps; }

// ---------------------------------------------------------------------------------
// Single steps
// ---------------------------------------------------------------------------------
// xpack / bmax_in: pack the input state n into normalised BF16 block vectors, by the
// block maxima that the step producing state n stored in bmax_in; bmax_out: store the
// block maxima of the output state n + 1 (AE forward and Algorithm 1 snapshots)
// tpack / tslot / vmax (time codec): store the output strain e^{n+1} as raw BF16 in slot
// tslot of the window buffer and fold its per-vector maxima into vmax
int fwd_step(aew_handle* h, int n, float* const in[4], float* const out[4], const float* wav,
             float* d_row, cudaStream_t s, uint16_t* xpack = nullptr,
             const unsigned* bmax_in = nullptr, unsigned* bmax_out = nullptr,
             uint16_t* tpack = nullptr, int tslot = 0, unsigned* vmax = nullptr) {
  aew::FwdStep a{};
  a.tpack = tpack;
  a.tslot = tslot;
  a.vmax = vmax;
  if (xpack) {
    a.xpack = xpack;
    a.bmax_in = bmax_in;
  }
  a.bmax_out = bmax_out;
  a.m = h->m;
  a.e = in[0];
  a.vx = in[1];
  a.vy = in[2];
  a.vz = in[3];
  a.e1 = out[0];
  a.vx1 = out[1];
  a.vy1 = out[2];
  a.vz1 = out[3];
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.kc = h->kc;
  a.dth = h->dth;
  a.dts = wav ? (float)(h->dt * (double)wav[n]) : 0.f;
  a.si = h->cfg.src[0];
  a.sj = h->cfg.src[1];
  a.sk = wav ? h->cfg.src[2] : -1;
  a.src_w = h->src_w;
  a.sr = h->src_r;
  a.krec = d_row ? h->krec : -1;
  a.rec_map = h->rec_map;
  a.d_out = d_row;
  a.err = aew::codec_err_flag(h->codec);
  AEW_CK(aew::launch_fwd_step(a, false, s));
  ++h->stats.kernel_launches;
  return AEW_OK;
}

int incr_step(aew_handle* h, float* const in[4], float* const out[4], const float* en,
              float* d_row, cudaStream_t s, uint16_t* tpack = nullptr, int tslot = 0,
              unsigned* vmax = nullptr, const uint16_t* en16 = nullptr) {
  aew::FwdStep a{};
  a.tpack = tpack;
  a.tslot = tslot;
  a.vmax = vmax;
  a.m = h->m;
  a.e = in[0];
  a.vx = in[1];
  a.vy = in[2];
  a.vz = in[3];
  a.e1 = out[0];
  a.vx1 = out[1];
  a.vy1 = out[2];
  a.vz1 = out[3];
  // with e^n = 0 (n = 0) the extra source G(dm e^n) vanishes: plain step, no source
  const bool incr = en != nullptr || en16 != nullptr;
  a.dm = incr ? h->dm : nullptr;
  a.ef = en;
  a.ef16 = en16;
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.kc = h->kc;
  a.dth = h->dth;
  a.dts = 0.f;
  a.sk = -1;
  a.krec = d_row ? h->krec : -1;
  a.rec_map = h->rec_map;
  a.d_out = d_row;
  a.err = aew::codec_err_flag(h->codec);
  AEW_CK(aew::launch_fwd_step(a, incr, s));
  ++h->stats.kernel_launches;
  return AEW_OK;
}

// reverse step n on explicit buffers: (mu, lam) in `in` -> `out`, accumulating
// e^n dt q into (acc32, acc64); qout / qin + dm2: the full Newton HVP's coupling
int adj_step_x(aew_handle* h, int n, float* const in[4], float* const out[4],
               const float* resid, const float* en, float* acc32, double* acc64, float* qout,
               const float* qin, const float* dm2, cudaStream_t s,
               const uint16_t* en16 = nullptr) {
  aew::AdjStep a{};
  a.m = h->m;
  a.mu = in[0];
  a.lx = in[1];
  a.ly = in[2];
  a.lz = in[3];
  a.mu1 = out[0];
  a.lx1 = out[1];
  a.ly1 = out[2];
  a.lz1 = out[3];
  a.en = en;
  a.en16 = en16;
  a.acc32 = acc32;
  a.acc64 = acc64;
  a.qout = qout;
  a.qin = qin;
  a.dm2 = dm2;
  const int W = h->cfg.accum_window;
  const int w = (h->cfg.nt - 1 - n) % W;
  a.acc_mode = (w == 0 ? aew::kAccFirst : 0) | ((w == W - 1 || n == 0) ? aew::kAccLast : 0);
  a.nx = h->cfg.nx;
  a.ny = h->cfg.ny;
  a.nz = h->cfg.nz;
  a.kc = h->kc_adj;
  a.dth = h->dth;
  a.krec = h->krec;
  a.rec_map = h->rec_map;
  a.resid = (resid && h->nrow) ? resid + (size_t)(n + 1) * h->nrow : nullptr;
  a.err = aew::codec_err_flag(h->codec);
  AEW_CK(aew::launch_adj_step(a, s));
  ++h->stats.kernel_launches;
  return AEW_OK;
}

// reverse step n: (lam, mu) in ad[cur] -> ad[cur ^ 1]
int adj_step(aew_handle* h, int n, int cur, const float* resid, const float* en,
             cudaStream_t s) {
  return adj_step_x(h, n, h->ad[cur], h->ad[cur ^ 1], resid, en, h->acc32, h->acc64, nullptr,
                    nullptr, nullptr, s);
}

int zero_state(aew_handle* h, float* const f[4], cudaStream_t s) {
  for (int i = 0; i < 4; ++i) AEW_CK(cudaMemsetAsync(f[i], 0, h->C * sizeof(float), s));
  return AEW_OK;
}

int copy_state(aew_handle* h, float* const dst[4], float* const src[4], cudaStream_t s) {
  for (int i = 0; i < 4; ++i)
    AEW_CK(cudaMemcpyAsync(dst[i], src[i], h->C * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return AEW_OK;
}

// m = c^2 with checks of c (synchronises the stream to read the checks)
int prepare_c(aew_handle* h, const float* c_dev, cudaStream_t s) {
  if (!c_dev) return fail(h, AEW_E_ARG, "c is NULL");
  AEW_CK(cudaMemsetAsync(h->chk, 0, sizeof(aew::FieldCheck), s));
  AEW_CK(cudaMemcpyAsync(h->c, c_dev, h->C * sizeof(float), cudaMemcpyDeviceToDevice, s));
  AEW_CK(aew::launch_prep_m(h->c, h->m, h->C, h->chk, s));
  ++h->stats.kernel_launches;
  aew::FieldCheck ck{};
  AEW_CK(cudaMemcpyAsync(&ck, h->chk, sizeof(ck), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  if (ck.nonfinite) return fail(h, AEW_E_NONFINITE, "c contains NaN or Inf");
  if (ck.cneg) return fail(h, AEW_E_CONFIG, "c must be positive everywhere");
  float cmax;
  std::memcpy(&cmax, &ck.cmax_bits, sizeof(float));
  if ((double)cmax * h->dt / h->cfg.h > 1.0 / std::sqrt(3.0)) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "max c = %.6g violates c dt / h <= 1/sqrt(3) (dt = %.6g)",
                  (double)cmax, h->dt);
    return fail(h, AEW_E_CFL, buf);
  }
  return AEW_OK;
}

// residual R = d - d_obs (rows 1..nt) and misfit J (device double part[kRedBlocks])
int residual_and_misfit(aew_handle* h, const float* d_obs, cudaStream_t s) {
  const size_t n = (size_t)(h->cfg.nt + 1) * h->nrow;
  if (n == 0) {
    AEW_CK(cudaMemsetAsync(h->part + aew::kRedBlocks, 0, sizeof(double), s));
    return AEW_OK;
  }
  AEW_CK(aew::launch_residual(h->d, d_obs, h->R, h->nrow, n, h->part, aew::kRedBlocks, s));
  AEW_CK(aew::launch_sum_partials(h->part, aew::kRedBlocks, 0.5, h->part + aew::kRedBlocks, s));
  h->stats.kernel_launches += 2;
  return AEW_OK;
}

// internal return value: the Armijo gate stopped a gradient after its forward solve
constexpr int kGated = 1;

// with a finite gate, read the misfit just computed and stop the gradient if it fails
int misfit_gate(aew_handle* h, cudaStream_t s) {
  if (!std::isfinite(h->gate)) return AEW_OK;
  double J = 0.0;
  AEW_CK(cudaMemcpyAsync(&J, h->part + aew::kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  h->stats.last_misfit = J;
  return J > h->gate ? kGated : AEW_OK;
}

int begin_adjoint(aew_handle* h, cudaStream_t s) {
  for (int i = 0; i < 4; ++i) AEW_CK(cudaMemsetAsync(h->ad[0][i], 0, h->C * sizeof(float), s));
  AEW_CK(cudaMemsetAsync(h->acc64, 0, h->C * sizeof(double), s));
  return AEW_OK;
}

const float* wav_or_default(aew_handle* h, const float* w) { return w ? w : h->wav.data(); }

float* drow(aew_handle* h, float* d, int n) {
  return h->nrow ? d + (size_t)n * h->nrow : nullptr;
}

// ---------------------------------------------------------------------------------
// AE helpers
// ---------------------------------------------------------------------------------
// encoder GEMMs of the packed, normalised state n (xpk[n % 2]) into latents[n]
int encode_packed(aew_handle* h, int n, cudaStream_t s) {
  const size_t nb = nblocks_of(h);
  cudaError_t e = aew::codec_encode_vectors(h->codec, h->xpk[n & 1], (long long)nb,
                                            h->lat + (size_t)n * nb * h->cfg.n_lat, h->ovf, s,
                                            h->overlap_ctas);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_vectors");
  h->stats.kernel_launches += 2;
  return AEW_OK;
}

// decoded strain of step n into buf
int decode_e(aew_handle* h, int n, float* buf, cudaStream_t s) {
  const size_t nb = nblocks_of(h);
  cudaError_t e = aew::codec_decode_grid_e(h->codec, h->lat + (size_t)n * nb * h->cfg.n_lat,
                                           h->cfg.nx, h->cfg.ny, h->cfg.nz,
                                           h->bmx + (size_t)n * nb * 4, buf, s, h->overlap_ctas);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_grid_e");
  h->stats.kernel_launches += 1;   // the fused two-layer decoder
  return AEW_OK;
}

// make stream `to` wait for all work enqueued so far on stream `from`
int join(aew_handle* h, cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  AEW_CK(cudaEventRecord(ev, from));
  AEW_CK(cudaStreamWaitEvent(to, ev, 0));
  return AEW_OK;
}

// Adjoint sweep in AE mode: the decode of step n-1 runs on the side stream while the
// adjoint step n runs on s.  edb[m % 2] holds the decoded strain of step m; its
// previous reader is adjoint step m + 2.  ev_b[m % 2]: decode m done; ev_a[m % 2]:
// adjoint step m done.
int ae_adjoint_sweep(aew_handle* h, const float* resid, cudaStream_t s) {
  const int nt = h->cfg.nt;
  int rc;
  if ((rc = begin_adjoint(h, s))) return rc;
  if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
  if (nt - 1 >= 1) {
    if ((rc = decode_e(h, nt - 1, h->edb[(nt - 1) & 1], h->side))) return rc;
    AEW_CK(cudaEventRecord(h->ev_b[(nt - 1) & 1], h->side));
  }
  int acur = 0;
  for (int n = nt - 1; n >= 0; --n) {
    if (n - 1 >= 1) {
      if (n + 1 <= nt - 1) AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(n + 1) & 1], 0));
      if ((rc = decode_e(h, n - 1, h->edb[(n - 1) & 1], h->side))) return rc;
      AEW_CK(cudaEventRecord(h->ev_b[(n - 1) & 1], h->side));
    }
    if (n >= 1) AEW_CK(cudaStreamWaitEvent(s, h->ev_b[n & 1], 0));
    if ((rc = adj_step(h, n, acur, resid, n >= 1 ? h->edb[n & 1] : nullptr, s))) return rc;
    AEW_CK(cudaEventRecord(h->ev_a[n & 1], s));
    acur ^= 1;
  }
  return join(h, h->side, s, h->ev_sync2);
}

// ---------------------------------------------------------------------------------
// Gradient drivers
// ---------------------------------------------------------------------------------
int gradient_full(aew_handle* h, const float* d_obs, const float* wav, cudaStream_t s) {
  const int nt = h->cfg.nt;
  float* vb[2][3] = {{h->st[0][1], h->st[0][2], h->st[0][3]},
                     {h->st[1][1], h->st[1][2], h->st[1][3]}};
  for (int i = 0; i < 3; ++i) AEW_CK(cudaMemsetAsync(vb[0][i], 0, h->C * sizeof(float), s));
  AEW_CK(cudaMemsetAsync(h->estore, 0, h->C * sizeof(float), s));
  AEW_CK(cudaMemsetAsync(h->d, 0, h->nrow * sizeof(float), s));
  for (int n = 0; n < nt; ++n) {
    const int a = n & 1;
    float* eout = (n + 1 < nt) ? h->estore + (size_t)(n + 1) * h->C : h->st[0][0];
    float* in[4] = {h->estore + (size_t)n * h->C, vb[a][0], vb[a][1], vb[a][2]};
    float* out[4] = {eout, vb[a ^ 1][0], vb[a ^ 1][1], vb[a ^ 1][2]};
    int rc = fwd_step(h, n, in, out, wav, drow(h, h->d, n + 1), s);
    if (rc) return rc;
  }
  int rc = residual_and_misfit(h, d_obs, s);
  if (rc) return rc;
  if ((rc = misfit_gate(h, s))) return rc;
  if ((rc = begin_adjoint(h, s))) return rc;
  int cur = 0;
  for (int n = nt - 1; n >= 0; --n) {
    const float* en = n > 0 ? h->estore + (size_t)n * h->C : nullptr;
    if ((rc = adj_step(h, n, cur, h->R, en, s))) return rc;
    cur ^= 1;
  }
  h->stats.forward_steps = nt;
  h->stats.adjoint_steps = nt;
  return AEW_OK;
}

// Execute a checkpointing plan.  mode gradient: the first pass records d and the
// 'final' action computes the misfit; otherwise (incremental adjoint of the GN-HVP) the
// residual is given.  The live state is a set of field pointers: a restore just points
// at the slot (or at the zero state), and a store is written by the last step of the
// preceding advance directly into the slot, so no state is ever copied.
int run_revolve(aew_handle* h, const float* d_obs, const float* resid, const float* wav,
                bool gradient, cudaStream_t s, long long* fwd_out) {
  const int nt = h->cfg.nt;
  const int ns = h->cfg.n_checkpoints;
  std::vector<aew::RevAction> plan;
  aew::revolve_plan(nt, ns, plan);
  int live_n = 0, acur = 0, rc;
  long long fwd = 0;
  auto slot = [&](int k, float** f) {
    for (int i = 0; i < 4; ++i) f[i] = h->ckpt + ((size_t)k * 4 + i) * h->C;
  };
  float* live[4];
  for (int i = 0; i < 4; ++i) live[i] = h->zst[i];
  int live_buf = -1;  // 0/1: ping-pong buffer, -1: zero state or a slot
  if (gradient) AEW_CK(cudaMemsetAsync(h->d, 0, h->nrow * sizeof(float), s));
  if ((rc = begin_adjoint(h, s))) return rc;
  std::vector<int> slot_step(ns > 0 ? ns : 1, -1);
  const float* R = resid;
  for (size_t a = 0; a < plan.size(); ++a) {
    const aew::RevAction& act = plan[a];
    switch (act.op) {
      case aew::kOpAdvance: {
        const bool to_slot = a + 1 < plan.size() && plan[a + 1].op == aew::kOpStore;
        for (int k = 0; k < act.arg; ++k) {
          float* out[4];
          int out_buf;
          if (to_slot && k == act.arg - 1) {
            slot(plan[a + 1].arg, out);
            out_buf = -1;
          } else {
            out_buf = live_buf == 0 ? 1 : 0;
            for (int i = 0; i < 4; ++i) out[i] = h->st[out_buf][i];
          }
          rc = fwd_step(h, live_n, live, out, wav, gradient ? drow(h, h->d, live_n + 1) : nullptr,
                        s);
          if (rc) return rc;
          for (int i = 0; i < 4; ++i) live[i] = out[i];
          live_buf = out_buf;
          ++live_n;
          ++fwd;
        }
        break;
      }
      case aew::kOpStore: {
        float* dst[4];
        slot(act.arg, dst);
        if (live[0] != dst[0]) {   // not produced in place by the previous advance
          if ((rc = copy_state(h, dst, live, s))) return rc;
          for (int i = 0; i < 4; ++i) live[i] = dst[i];
          live_buf = -1;
        }
        slot_step[act.arg] = live_n;
        break;
      }
      case aew::kOpRestore:
        if (act.arg < 0) {
          for (int i = 0; i < 4; ++i) live[i] = h->zst[i];
          live_n = 0;
        } else {
          slot(act.arg, live);
          live_n = slot_step[act.arg];
        }
        live_buf = -1;
        break;
      case aew::kOpFinal:
        if (gradient) {
          // last step into a scratch buffer: records d^{nt}, keeps state nt-1 live
          float* out[4];
          const int ob = live_buf == 0 ? 1 : 0;
          for (int i = 0; i < 4; ++i) out[i] = h->st[ob][i];
          rc = fwd_step(h, live_n, live, out, wav, drow(h, h->d, live_n + 1), s);
          if (rc) return rc;
          ++fwd;
          if ((rc = residual_and_misfit(h, d_obs, s))) return rc;
          R = h->R;
        }
        break;
      case aew::kOpReverse:
        if ((rc = adj_step(h, act.arg, acur, R, act.arg > 0 ? live[0] : nullptr, s))) return rc;
        acur ^= 1;
        break;
    }
  }
  *fwd_out = fwd;
  return AEW_OK;
}

// AE gradient: forward step n packs its input state n into xpk[n % 2]; the encoder of
// state n runs on the side stream while step n + 1 runs on s.  ev_a[n % 2]: step n
// done; ev_b[n % 2]: encoder of state n done (xpk[n % 2] free again for step n + 2).
int gradient_ae(aew_handle* h, const float* d_obs, const float* wav, cudaStream_t s) {
  const int nt = h->cfg.nt;
  int rc;
  if ((rc = zero_state(h, h->st[0], s))) return rc;
  // block maxima of every packed state are stored whole by its step; state 0 is zero
  AEW_CK(cudaMemsetAsync(h->bmx, 0, nblocks_of(h) * 4 * sizeof(unsigned), s));
  AEW_CK(cudaMemsetAsync(h->ovf, 0, sizeof(int), s));
  AEW_CK(cudaMemsetAsync(h->d, 0, h->nrow * sizeof(float), s));
  if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
  int cur = 0;
  for (int n = 0; n < nt; ++n) {
    if (n >= 3) AEW_CK(cudaStreamWaitEvent(s, h->ev_b[n & 1], 0));
    // step n packs state n by the maxima step n - 1 stored, and stores those of state
    // n + 1 (states 1 .. nt - 1 are encoded)
    const size_t nb4 = nblocks_of(h) * 4;
    rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], wav, drow(h, h->d, n + 1), s,
                  n >= 1 ? h->xpk[n & 1] : nullptr, h->bmx + n * nb4,
                  n + 1 < nt ? h->bmx + (n + 1) * nb4 : nullptr);
    if (rc) return rc;
    cur ^= 1;
    if (n >= 1) {
      AEW_CK(cudaEventRecord(h->ev_a[n & 1], s));
      AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[n & 1], 0));
      if ((rc = encode_packed(h, n, h->side))) return rc;
      AEW_CK(cudaEventRecord(h->ev_b[n & 1], h->side));
    }
  }
  if ((rc = join(h, h->side, s, h->ev_sync2))) return rc;
  if ((rc = residual_and_misfit(h, d_obs, s))) return rc;
  if ((rc = misfit_gate(h, s))) return rc;
  if ((rc = ae_adjoint_sweep(h, h->R, s))) return rc;
  h->stats.forward_steps = nt;
  h->stats.adjoint_steps = nt;
  return AEW_OK;
}

// ---------------------------------------------------------------------------------
// Compression in time: windows of 16 strain states per 2 x 8 x 8-node block
// ---------------------------------------------------------------------------------
// encoder of window tb (raw vectors in xt[tb % 2], maxima vmx[tb]) into its latents
int encode_window(aew_handle* h, int tb, cudaStream_t s) {
  const size_t nv = nvec_of(h);
  const bool mm = aew::codec_minmax(h->codec);
  cudaError_t e = aew::codec_encode_window(h->codec, h->xt[tb & 1], h->vmx + (size_t)tb * nv,
                                           (long long)nv, h->lat + (size_t)tb * nv * h->cfg.n_lat,
                                           h->ovf, s, h->overlap_ctas,
                                           mm ? h->wmn + (size_t)tb * nv : nullptr,
                                           mm ? h->wr + (size_t)tb * nv : nullptr);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_window");
  h->stats.kernel_launches += 2;
  return AEW_OK;
}

// decoder of window tb into its 16 strain slices edt[tb % 2]: BF16 for every sweep (their
// e^n boxes then carry half the bytes), FP32 for the profiling hook's FP32 kind
int decode_window(aew_handle* h, int tb, cudaStream_t s, bool bf16 = false) {
  const size_t nv = nvec_of(h);
  const bool mm = aew::codec_minmax(h->codec);
  cudaError_t e = aew::codec_decode_window(h->codec, h->lat + (size_t)tb * nv * h->cfg.n_lat,
                                           h->vmx + (size_t)tb * nv, h->cfg.nx, h->cfg.ny,
                                           h->cfg.nz, h->edt[tb & 1], s, h->overlap_ctas,
                                           mm ? h->wmn + (size_t)tb * nv : nullptr,
                                           mm ? h->wr + (size_t)tb * nv : nullptr, bf16);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_window");
  h->stats.kernel_launches += 2;
  return AEW_OK;
}

// decoded strain e^n (n >= 1) of the window being read
const float* window_e(aew_handle* h, int n) {
  return n >= 1 ? h->edt[(n / aew::kTSteps) & 1] + (size_t)(n % aew::kTSteps) * h->C : nullptr;
}
// the same, decoded as BF16
const uint16_t* window_e16(aew_handle* h, int n) {
  return n >= 1 ? reinterpret_cast<const uint16_t*>(h->edt[(n / aew::kTSteps) & 1]) +
                      (size_t)(n % aew::kTSteps) * h->C
                : nullptr;
}

// Adjoint sweep with the time codec: entering window tb (in reverse), the decoder of
// window tb - 1 runs on the side stream into the buffer window tb + 1 used, while the
// adjoint steps of window tb run on s.  ev_b[w % 2]: window w decoded; ev_a[w % 2]:
// window w's adjoint steps done.
int time_adjoint_sweep(aew_handle* h, const float* resid, cudaStream_t s) {
  const int nt = h->cfg.nt, W = nwin_of(h), T = aew::kTSteps;
  int rc;
  if ((rc = begin_adjoint(h, s))) return rc;
  if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
  if ((rc = decode_window(h, W - 1, h->side, true))) return rc;
  AEW_CK(cudaEventRecord(h->ev_b[(W - 1) & 1], h->side));
  int acur = 0;
  for (int n = nt - 1; n >= 0; --n) {
    const int tb = n / T;
    if (n == nt - 1 || n % T == T - 1) {
      if (tb >= 1) {
        if (tb + 1 <= W - 1) AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(tb + 1) & 1], 0));
        if ((rc = decode_window(h, tb - 1, h->side, true))) return rc;
        AEW_CK(cudaEventRecord(h->ev_b[(tb - 1) & 1], h->side));
      }
      AEW_CK(cudaStreamWaitEvent(s, h->ev_b[tb & 1], 0));
    }
    if ((rc = adj_step_x(h, n, h->ad[acur], h->ad[acur ^ 1], resid, nullptr, h->acc32, h->acc64,
                         nullptr, nullptr, nullptr, s, window_e16(h, n))))
      return rc;
    acur ^= 1;
    if (n % T == 0) AEW_CK(cudaEventRecord(h->ev_a[tb & 1], s));
  }
  return join(h, h->side, s, h->ev_sync2);
}

// AE gradient with the time codec: the step that writes state m = n + 1 stores it in
// slot m % 16 of window m / 16 (buffer xt[(m / 16) % 2]) with the vectors' maxima; a
// complete window is encoded on the side stream while the next window's steps run on
// s.  ev_a[w % 2]: window w complete; ev_b[w % 2]: window w encoded (its buffer is free
// for window w + 2).
int gradient_ae_time(aew_handle* h, const float* d_obs, const float* wav, cudaStream_t s) {
  const int nt = h->cfg.nt, W = nwin_of(h), T = aew::kTSteps;
  const size_t nv = nvec_of(h), wbytes = nv * aew::kNIn * sizeof(uint16_t);
  int rc;
  if ((rc = zero_state(h, h->st[0], s))) return rc;
  AEW_CK(cudaMemsetAsync(h->vmx, 0, (size_t)W * nv * sizeof(unsigned), s));
  AEW_CK(cudaMemsetAsync(h->xt[0], 0, wbytes, s));   // slot 0 of window 0 is e^0 = 0
  AEW_CK(cudaMemsetAsync(h->ovf, 0, sizeof(int), s));
  AEW_CK(cudaMemsetAsync(h->d, 0, h->nrow * sizeof(float), s));
  if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
  auto window_done = [&](int tb) -> int {
    AEW_CK(cudaEventRecord(h->ev_a[tb & 1], s));
    AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[tb & 1], 0));
    int r = encode_window(h, tb, h->side);
    if (r) return r;
    AEW_CK(cudaEventRecord(h->ev_b[tb & 1], h->side));
    return AEW_OK;
  };
  if (nt == 1 && (rc = window_done(0))) return rc;
  int cur = 0;
  for (int n = 0; n < nt; ++n) {
    const int m = n + 1;
    uint16_t* tp = nullptr;
    unsigned* vm = nullptr;
    const int tb = m / T, slot = m % T;
    if (m <= nt - 1) {
      if (slot == 0) {
        if (tb >= 2) AEW_CK(cudaStreamWaitEvent(s, h->ev_b[tb & 1], 0));
        if (T * tb + T > nt) AEW_CK(cudaMemsetAsync(h->xt[tb & 1], 0, wbytes, s));   // tail 0
      }
      tp = h->xt[tb & 1];
      vm = h->vmx + (size_t)tb * nv;
    }
    rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], wav, drow(h, h->d, n + 1), s, nullptr,
                  nullptr, nullptr, tp, slot, vm);
    if (rc) return rc;
    cur ^= 1;
    if (m <= nt - 1 && (slot == T - 1 || m == nt - 1) && (rc = window_done(tb))) return rc;
  }
  if ((rc = join(h, h->side, s, h->ev_sync2))) return rc;
  if ((rc = residual_and_misfit(h, d_obs, s))) return rc;
  if ((rc = misfit_gate(h, s))) return rc;
  if ((rc = time_adjoint_sweep(h, h->R, s))) return rc;
  h->stats.forward_steps = nt;
  h->stats.adjoint_steps = nt;
  return AEW_OK;
}

// ---------------------------------------------------------------------------------
// Full Newton HVP
// ---------------------------------------------------------------------------------
// buffers of the second-order adjoint and the incremental strain history (first call)
int ensure_newton(aew_handle* h) {
  if (h->nw_ready) return AEW_OK;
  const size_t C = h->C, nt = (size_t)h->cfg.nt;
  bool ok = dalloc(h, &h->acc32b, C) && dalloc(h, &h->acc64b, C) && dalloc(h, &h->qbuf, C);
  for (int b = 0; ok && b < 2; ++b)
    for (int i = 0; ok && i < 4; ++i) ok = dalloc(h, &h->ad2[b][i], C);
  if (ok && h->cfg.storage == AEW_FULL) ok = dalloc(h, &h->desto, nt * C);
  if (ok && h->cfg.storage == AEW_AE) {
    const size_t nv = nvec_of(h), W = (size_t)nwin_of(h);
    ok = dalloc(h, &h->lat2, W * nv * h->cfg.n_lat) && dalloc(h, &h->vmx2, W * nv) &&
         dalloc(h, &h->edt2[0], aew::kTSteps * C) && dalloc(h, &h->edt2[1], aew::kTSteps * C);
    if (ok && aew::codec_minmax(h->codec))
      ok = dalloc(h, &h->wmn2, W * nv) && dalloc(h, &h->wr2, W * nv);
    for (int i = 0; ok && i < 2; ++i)
      ok = cudaEventCreateWithFlags(&h->ev_c[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_d[i], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    return fail(h, AEW_E_NOMEM, "device allocation failed for the full Newton HVP buffers");
  }
  h->stats.device_bytes = h->bytes + aew::codec_device_bytes(h->codec);
  h->nw_ready = true;
  return AEW_OK;
}

// incremental forward keeping the incremental strain history: full storage writes it to
// desto; the time codec packs it into windows (xt) and encodes them (lat2, vmx2) on the
// side stream, while the forward strain's windows are decoded ahead as in
// incremental_forward.  ev_a/ev_b: e windows read / decoded; ev_c/ev_d: de windows
// complete / encoded.
int newton_incremental_forward(aew_handle* h, cudaStream_t s) {
  const int nt = h->cfg.nt;
  int rc;
  if ((rc = zero_state(h, h->ad[0], s))) return rc;
  if (h->nrow) AEW_CK(cudaMemsetAsync(h->dd, 0, h->nrow * sizeof(float), s));
  int cur = 0;
  if (h->cfg.storage == AEW_FULL) {
    AEW_CK(cudaMemsetAsync(h->desto, 0, h->C * sizeof(float), s));
    for (int n = 0; n < nt; ++n) {
      float* in[4] = {h->desto + (size_t)n * h->C, h->ad[cur][1], h->ad[cur][2], h->ad[cur][3]};
      float* eo = n + 1 < nt ? h->desto + (size_t)(n + 1) * h->C : h->ad[cur ^ 1][0];
      float* out[4] = {eo, h->ad[cur ^ 1][1], h->ad[cur ^ 1][2], h->ad[cur ^ 1][3]};
      const float* en = n > 0 ? h->estore + (size_t)n * h->C : nullptr;
      if ((rc = incr_step(h, in, out, en, drow(h, h->dd, n + 1), s))) return rc;
      cur ^= 1;
    }
    return AEW_OK;
  }
  const int W = nwin_of(h), T = aew::kTSteps;
  const size_t nv = nvec_of(h), wbytes = nv * aew::kNIn * sizeof(uint16_t);
  AEW_CK(cudaMemsetAsync(h->ovf, 0, sizeof(int), s));
  AEW_CK(cudaMemsetAsync(h->vmx2, 0, (size_t)W * nv * sizeof(unsigned), s));
  AEW_CK(cudaMemsetAsync(h->xt[0], 0, wbytes, s));   // de^0 = 0
  if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
  auto encode_de = [&](int tb) -> int {
    AEW_CK(cudaEventRecord(h->ev_c[tb & 1], s));
    AEW_CK(cudaStreamWaitEvent(h->side, h->ev_c[tb & 1], 0));
    const bool mm = aew::codec_minmax(h->codec);
    cudaError_t e = aew::codec_encode_window(h->codec, h->xt[tb & 1], h->vmx2 + (size_t)tb * nv,
                                             (long long)nv, h->lat2 + (size_t)tb * nv * h->cfg.n_lat,
                                             h->ovf, h->side, h->overlap_ctas,
                                             mm ? h->wmn2 + (size_t)tb * nv : nullptr,
                                             mm ? h->wr2 + (size_t)tb * nv : nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_window");
    h->stats.kernel_launches += 2;
    AEW_CK(cudaEventRecord(h->ev_d[tb & 1], h->side));
    return AEW_OK;
  };
  if ((rc = decode_window(h, 0, h->side, true))) return rc;
  AEW_CK(cudaEventRecord(h->ev_b[0], h->side));
  if (nt == 1 && (rc = encode_de(0))) return rc;
  for (int n = 0; n < nt; ++n) {
    const int tb = n / T;
    if (n % T == 0) {
      if (tb + 1 <= W - 1) {
        if (tb >= 1) AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(tb + 1) & 1], 0));
        if ((rc = decode_window(h, tb + 1, h->side, true))) return rc;
        AEW_CK(cudaEventRecord(h->ev_b[(tb + 1) & 1], h->side));
      }
      AEW_CK(cudaStreamWaitEvent(s, h->ev_b[tb & 1], 0));
    }
    const int m = n + 1, to = m / T, slot = m % T;
    uint16_t* tp = nullptr;
    unsigned* vm = nullptr;
    if (m <= nt - 1) {
      if (slot == 0) {
        if (to >= 2) AEW_CK(cudaStreamWaitEvent(s, h->ev_d[to & 1], 0));
        if (T * to + T > nt) AEW_CK(cudaMemsetAsync(h->xt[to & 1], 0, wbytes, s));
      }
      tp = h->xt[to & 1];
      vm = h->vmx2 + (size_t)to * nv;
    }
    if ((rc = incr_step(h, h->ad[cur], h->ad[cur ^ 1], nullptr, drow(h, h->dd, n + 1), s,
                        tp, slot, vm, window_e16(h, n))))
      return rc;
    cur ^= 1;
    if (n % T == T - 1 || n == nt - 1) AEW_CK(cudaEventRecord(h->ev_a[tb & 1], s));
    if (m <= nt - 1 && (slot == T - 1 || m == nt - 1) && (rc = encode_de(to))) return rc;
  }
  return join(h, h->side, s, h->ev_sync2);
}

// decoder of the incremental strain's window tb into edt2[tb % 2]
int decode_de_window(aew_handle* h, int tb, cudaStream_t s) {
  const size_t nv = nvec_of(h);
  const bool mm = aew::codec_minmax(h->codec);
  cudaError_t e = aew::codec_decode_window(h->codec, h->lat2 + (size_t)tb * nv * h->cfg.n_lat,
                                           h->vmx2 + (size_t)tb * nv, h->cfg.nx, h->cfg.ny,
                                           h->cfg.nz, h->edt2[tb & 1], s, h->overlap_ctas,
                                           mm ? h->wmn2 + (size_t)tb * nv : nullptr,
                                           mm ? h->wr2 + (size_t)tb * nv : nullptr, true);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_window");
  h->stats.kernel_launches += 2;
  return AEW_OK;
}

// the two adjoints in lockstep, n = nt-1 .. 0: first order (ad, residual R, accumulating
// de^n dt q into acc32/acc64, writing dt q), second order (ad2, residual B dv = dd,
// accumulating e^n dt dq into acc32b/acc64b, with the dm dt q source)
int newton_adjoint_sweep(aew_handle* h, cudaStream_t s) {
  const int nt = h->cfg.nt, T = aew::kTSteps;
  int rc;
  for (int i = 0; i < 4; ++i) {
    AEW_CK(cudaMemsetAsync(h->ad[0][i], 0, h->C * sizeof(float), s));
    AEW_CK(cudaMemsetAsync(h->ad2[0][i], 0, h->C * sizeof(float), s));
  }
  AEW_CK(cudaMemsetAsync(h->acc64, 0, h->C * sizeof(double), s));
  AEW_CK(cudaMemsetAsync(h->acc64b, 0, h->C * sizeof(double), s));
  const bool ae = h->cfg.storage == AEW_AE;
  const int W = nwin_of(h);
  auto decode_both = [&](int tb) -> int {
    int r = decode_window(h, tb, h->side, true);
    if (!r) r = decode_de_window(h, tb, h->side);
    return r;
  };
  if (ae) {
    if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
    if ((rc = decode_both(W - 1))) return rc;
    AEW_CK(cudaEventRecord(h->ev_b[(W - 1) & 1], h->side));
  }
  int cur = 0;
  for (int n = nt - 1; n >= 0; --n) {
    const float* en = nullptr;
    const float* den = nullptr;
    const uint16_t* en16 = nullptr;    // the time codec's decoded windows, BF16 (R34)
    const uint16_t* den16 = nullptr;
    if (ae) {
      const int tb = n / T;
      if (n == nt - 1 || n % T == T - 1) {
        if (tb >= 1) {
          if (tb + 1 <= W - 1) AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(tb + 1) & 1], 0));
          if ((rc = decode_both(tb - 1))) return rc;
          AEW_CK(cudaEventRecord(h->ev_b[(tb - 1) & 1], h->side));
        }
        AEW_CK(cudaStreamWaitEvent(s, h->ev_b[tb & 1], 0));
      }
      en16 = window_e16(h, n);
      den16 = n >= 1 ? reinterpret_cast<const uint16_t*>(h->edt2[tb & 1]) + (size_t)(n % T) * h->C
                     : nullptr;
    } else if (n > 0) {
      en = h->estore + (size_t)n * h->C;
      den = h->desto + (size_t)n * h->C;
    }
    if ((rc = adj_step_x(h, n, h->ad[cur], h->ad[cur ^ 1], h->R, den, h->acc32, h->acc64,
                         h->qbuf, nullptr, nullptr, s, den16)))
      return rc;
    if ((rc = adj_step_x(h, n, h->ad2[cur], h->ad2[cur ^ 1], h->dd, en, h->acc32b, h->acc64b,
                         nullptr, h->qbuf, h->dm, s, en16)))
      return rc;
    cur ^= 1;
    if (ae && n % T == 0) AEW_CK(cudaEventRecord(h->ev_a[(n / T) & 1], s));
  }
  if (ae) return join(h, h->side, s, h->ev_sync2);
  return AEW_OK;
}

// Algorithm 1 with the time codec: the complete windows tb = 0, every, 2 every, ... are
// packed by the forward steps that write their states (raw BF16 plus per-vector
// maxima), then normalised in place once their last state is in.
int snapshots_time(aew_handle* h, int every, uint16_t* out, long long max_vectors,
                   float* vmax_dev, long long* n_written, cudaStream_t s) {
  const int nt = h->cfg.nt, T = aew::kTSteps, W = nwin_of(h);
  const size_t nv = nvec_of(h);
  if (!vmax_dev && !h->wk_vmax && !dalloc(h, &h->wk_vmax, nv))
    return fail(h, AEW_E_NOMEM, "workspace");
  std::vector<long long> at((size_t)W, -1);
  long long w = 0;
  int last = -1;
  for (int tb = 0; tb < W; ++tb)
    if (tb % every == 0 && T * tb + T - 1 <= nt - 1 && w + (long long)nv <= max_vectors) {
      at[tb] = w;
      w += (long long)nv;
      last = tb;
    }
  *n_written = 0;
  if (last < 0) return AEW_OK;
  // the steps' vector maxima: into the caller's buffer (power-of-two scales), or scratch
  // (min-max: the caller's buffer receives offsets and ranges instead)
  const bool mm = aew::codec_minmax(h->codec);
  if (mm && !h->wk_vmax && !dalloc(h, &h->wk_vmax, nv)) return fail(h, AEW_E_NOMEM, "workspace");
  auto vm = [&](int tb) {
    return vmax_dev && !mm ? reinterpret_cast<unsigned*>(vmax_dev) + at[tb] : h->wk_vmax;
  };
  int rc;
  if ((rc = zero_state(h, h->st[0], s))) return rc;
  if (at[0] >= 0) {   // slot 0 of window 0 is e^0 = 0, written by no step
    AEW_CK(cudaMemsetAsync(out + (size_t)at[0] * aew::kNIn, 0, nv * aew::kNIn * sizeof(uint16_t), s));
    AEW_CK(cudaMemsetAsync(vm(0), 0, nv * sizeof(unsigned), s));
  }
  int cur = 0;
  for (int n = 0; n < T * last + T - 1; ++n) {
    const int m = n + 1, tb = m / T, slot = m % T;
    uint16_t* tp = nullptr;
    unsigned* vq = nullptr;
    if (at[tb] >= 0) {
      tp = out + (size_t)at[tb] * aew::kNIn;
      vq = vm(tb);
      if (slot == 0) AEW_CK(cudaMemsetAsync(vq, 0, nv * sizeof(unsigned), s));
    }
    if ((rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], h->wav.data(), nullptr, s, nullptr,
                       nullptr, nullptr, tp, slot, vq)))
      return rc;
    cur ^= 1;
    if (tp && slot == T - 1) {
      if (aew::codec_minmax(h->codec))   // offsets and ranges out as FP32 pairs
        AEW_CK(aew::window_minmax(tp, (long long)nv, aew::codec_beta(h->codec), tp, nullptr, nullptr, s,
                                  vmax_dev ? vmax_dev + 2 * (size_t)at[tb] : nullptr));
      else
        AEW_CK(aew::window_normalise(tp, vq, (long long)nv, tp, s));
      ++h->stats.kernel_launches;
    }
  }
  AEW_CK(cudaStreamSynchronize(s));
  *n_written = w;
  return AEW_OK;
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================
extern "C" {

int aew_create(const aew_config* cfg, aew_handle** out) {
  g_create_err.clear();
  if (!out) return AEW_E_ARG;
  *out = nullptr;
  if (!cfg) {
    g_create_err = "cfg is NULL";
    return AEW_E_ARG;
  }
  auto bad = [&](const char* m) {
    g_create_err = m;
    return AEW_E_CONFIG;
  };
  const aew_config& c = *cfg;
  if (c.nx < 4 || c.ny < 4 || c.nz < 4 || c.nx % 4 || c.ny % 4 || c.nz % 4)
    return bad("nx, ny, nz must be >= 4 and multiples of 4");
  if (!(c.h > 0) || !(c.cfl > 0) || !(c.cmax > 0)) return bad("h, cfl, cmax must be > 0");
  if (c.cfl > 1.0 / std::sqrt(3.0)) return bad("cfl must be <= 1/sqrt(3)");
  if (c.nt < 1) return bad("nt must be >= 1");
  if (c.src[0] < 0 || c.src[0] >= c.nx || c.src[1] < 0 || c.src[1] >= c.ny || c.src[2] < 0 ||
      c.src[2] >= c.nz)
    return bad("source node outside the grid");
  if (c.nrec < 0 || (c.nrec > 0 && !c.rec_ijk)) return bad("bad receiver list");
  if (c.storage != AEW_FULL && c.storage != AEW_REVOLVE && c.storage != AEW_AE)
    return bad("storage must be AEW_FULL, AEW_REVOLVE or AEW_AE");
  if (c.storage == AEW_REVOLVE && c.n_checkpoints < 0) return bad("n_checkpoints must be >= 0");
  if (c.accum_window < 1) return bad("accum_window must be >= 1");
  if (c.storage == AEW_AE && c.codec == AEW_CODEC_SPACE && (c.nx % 8 || c.ny % 8 || c.nz % 8))
    return bad("AE storage needs nx, ny, nz multiples of 8");
  if (c.codec != AEW_CODEC_SPACE && c.codec != AEW_CODEC_TIME)
    return bad("codec must be AEW_CODEC_SPACE or AEW_CODEC_TIME");
  if (c.codec == AEW_CODEC_SPACE && c.n_lat != 64 && c.n_lat != 32)
    return bad("n_lat must be 64 or 32 for the space codec");
  if (c.codec == AEW_CODEC_TIME && c.n_lat != 512 && c.n_lat != 256)
    return bad("n_lat must be 512 or 256 for the time codec");
  if (c.storage == AEW_AE && c.codec == AEW_CODEC_TIME && (c.nx % 8 || c.ny % 8 || c.nz % 2))
    return bad("AE storage with the time codec needs nx, ny multiples of 8 and nz even");
  if ((c.norm != AEW_NORM_POW2 && c.norm != AEW_NORM_MINMAX) ||
      (c.act != AEW_ACT_GELU && c.act != AEW_ACT_ELU))
    return bad("norm must be AEW_NORM_POW2 or AEW_NORM_MINMAX, act AEW_ACT_GELU or AEW_ACT_ELU");
  if ((c.norm != AEW_NORM_POW2 || c.act != AEW_ACT_GELU) && c.codec != AEW_CODEC_TIME)
    return bad("min-max normalisation and ELU are variants of the time codec");
  if (!(c.beta >= 0.0)) return bad("beta must be >= 0 (0: the default 1e-7)");
  if (!(c.src_sigma >= 0.0) || !std::isfinite(c.src_sigma)) return bad("src_sigma must be >= 0");
  const int src_r = c.src_sigma > 0.0 ? (int)std::ceil(3.0 * c.src_sigma / c.h) : 0;
  if (src_r > 0 && (c.src[0] - src_r < 1 || c.src[0] + src_r > c.nx - 2 || c.src[1] - src_r < 1 ||
                    c.src[1] + src_r > c.ny - 2 || c.src[2] - src_r < 1 ||
                    c.src[2] + src_r > c.nz - 2))
    return bad("the smoothed source's box (radius ceil(3 src_sigma / h)) must lie in nodes 1 .. n-2");

  aew_handle* h = new aew_handle();
  h->cfg = c;
  h->cfg.rec_ijk = nullptr;
  h->rec.assign(c.rec_ijk, c.rec_ijk + 3 * (size_t)c.nrec);
  for (int r = 0; r < c.nrec; ++r) {
    const int i = h->rec[3 * r], j = h->rec[3 * r + 1], k = h->rec[3 * r + 2];
    if (i < 0 || i >= c.nx || j < 0 || j >= c.ny || k < 0 || k >= c.nz) {
      delete h;
      return bad("receiver outside the grid");
    }
    if (r == 0) h->krec = k;
    if (k != h->krec) {
      delete h;
      return bad("all receivers must lie on one node plane k");
    }
  }
  cudaGetDevice(&h->device);
  h->dt = c.cfl * c.h / c.cmax;
  h->dth = (float)(h->dt / c.h);
  h->C = (size_t)c.nx * c.ny * c.nz;
  h->kc = aew::default_kc(c.nx, c.ny, c.nz, false);
  h->kc_adj = aew::default_kc(c.nx, c.ny, c.nz, true);
  h->nrow = (size_t)c.nrec * 3;
  h->wav.resize(c.nt);
  for (int n = 0; n < c.nt; ++n) h->wav[n] = (float)(-ricker(n * h->dt, c.f0, c.t0));

  // the source's spread over the z-faces: Gaussian weights by face-centre distance,
  // normalised to sum 1 (the point source: one face, weight 1)
  h->src_r = src_r;
  const int sw = 2 * src_r + 1;
  std::vector<float> src_w((size_t)sw * sw * sw, 1.f);
  if (src_r > 0) {
    std::vector<double> w(src_w.size());
    double tot = 0.0;
    for (int a = 0; a < sw; ++a)
      for (int b = 0; b < sw; ++b)
        for (int d = 0; d < sw; ++d) {
          const double r2 = ((double)(a - src_r) * (a - src_r) + (double)(b - src_r) * (b - src_r) +
                             (double)(d - src_r) * (d - src_r)) * c.h * c.h;
          const double v = std::exp(-r2 / (2.0 * c.src_sigma * c.src_sigma));
          w[((size_t)a * sw + b) * sw + d] = v;
          tot += v;
        }
    for (size_t q = 0; q < w.size(); ++q) src_w[q] = (float)(w[q] / tot);
  }

  const size_t C = h->C, nt = (size_t)c.nt;
  bool ok = dalloc(h, &h->src_w, src_w.size()) &&
            cudaMemcpy(h->src_w, src_w.data(), src_w.size() * sizeof(float),
                       cudaMemcpyHostToDevice) == cudaSuccess &&
            dalloc(h, &h->c, C) && dalloc(h, &h->m, C) && dalloc(h, &h->dm, C) &&
            dalloc(h, &h->acc32, C) && dalloc(h, &h->acc64, C) &&
            dalloc(h, &h->d, (nt + 1) * h->nrow) && dalloc(h, &h->R, (nt + 1) * h->nrow) &&
            dalloc(h, &h->dd, (nt + 1) * h->nrow) &&
            dalloc(h, &h->rec_map, (size_t)c.nx * c.ny) &&
            dalloc(h, &h->part, aew::kRedBlocks + 8) && dalloc(h, &h->chk, 1) &&
            dalloc(h, &h->scratch8, 8);
  for (int b = 0; ok && b < 2; ++b)
    for (int i = 0; ok && i < 4; ++i) ok = dalloc(h, &h->st[b][i], C) && dalloc(h, &h->ad[b][i], C);
  if (ok && c.storage == AEW_FULL) ok = dalloc(h, &h->estore, nt * C);
  if (ok && (c.storage == AEW_FULL || (c.storage == AEW_AE && c.codec == AEW_CODEC_TIME)))
    ok = dalloc(h, &h->gc, C);
  if (ok && c.storage == AEW_REVOLVE && c.n_checkpoints > 0)
    ok = dalloc(h, &h->ckpt, (size_t)c.n_checkpoints * 4 * C);
  for (int i = 0; ok && c.storage == AEW_REVOLVE && i < 4; ++i) {
    ok = dalloc(h, &h->zst[i], C) && cudaMemset(h->zst[i], 0, C * sizeof(float)) == cudaSuccess;
  }
  h->tcodec = c.codec == AEW_CODEC_TIME;
  if (ok && c.storage == AEW_AE && !h->tcodec) {
    const size_t nb = (size_t)(c.nx / 8) * (c.ny / 8) * (c.nz / 8);
    ok = dalloc(h, &h->lat, nt * nb * c.n_lat) && dalloc(h, &h->bmx, nt * nb * 4) &&
         dalloc(h, &h->ovf, 1) && dalloc(h, &h->xpk[0], nb * aew::kNIn) &&
         dalloc(h, &h->xpk[1], nb * aew::kNIn) && dalloc(h, &h->edb[0], C) &&
         dalloc(h, &h->edb[1], C);
  }
  if (ok && c.storage == AEW_AE && h->tcodec && c.norm == AEW_NORM_MINMAX) {
    const size_t nv = nvec_of(h), W = (size_t)nwin_of(h);
    ok = dalloc(h, &h->wmn, W * nv) && dalloc(h, &h->wr, W * nv);
  }
  if (ok && c.storage == AEW_AE && h->tcodec) {
    const size_t nv = nvec_of(h), W = (size_t)nwin_of(h);
    ok = dalloc(h, &h->lat, W * nv * c.n_lat) && dalloc(h, &h->vmx, W * nv) &&
         dalloc(h, &h->ovf, 1) && dalloc(h, &h->xt[0], nv * aew::kNIn) &&
         dalloc(h, &h->xt[1], nv * aew::kNIn) && dalloc(h, &h->edt[0], aew::kTSteps * C) &&
         dalloc(h, &h->edt[1], aew::kTSteps * C);
  }
  if (ok && c.storage == AEW_AE) {
    // The codec GEMMs run on a high-priority side stream with half the SMs, so their
    // CTAs are placed first and the concurrent stencil step keeps the other half
    // (measured best at 256^3 among caps of 76-152 CTAs and 2-4 GEMM stages).
    int lo = 0, hi = 0, sms = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) hi = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->overlap_ctas = sms > 1 ? sms / 2 : 0;
    if (const char* env = getenv("AEW_GEMM_CTAS_OVERLAP")) h->overlap_ctas = atoi(env);   // tuning override
    ok = ok && cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i)
      ok = cudaEventCreateWithFlags(&h->ev_a[i], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_b[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&h->ev_sync, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&h->ev_sync2, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    g_create_err = "device allocation failed (" + std::to_string(h->bytes) + " bytes held)";
    aew_destroy(h);
    return AEW_E_NOMEM;
  }
  std::vector<int> map((size_t)c.nx * c.ny, -1);
  for (int r = 0; r < c.nrec; ++r) map[(size_t)h->rec[3 * r + 1] * c.nx + h->rec[3 * r]] = r;
  if (cudaMemcpy(h->rec_map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    g_create_err = "copy of the receiver map failed";
    aew_destroy(h);
    return AEW_E_CUDA;
  }
  h->codec = aew::codec_new(c.n_lat, h->tcodec);
  if (!h->codec) {
    g_create_err = "codec allocation failed";
    aew_destroy(h);
    return AEW_E_NOMEM;
  }
  aew::codec_set_variant(h->codec, c.norm, c.act, c.beta > 0.0 ? c.beta : 1e-7);
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreate(&h->tg[i]) != cudaSuccess || cudaEventCreate(&h->th[i]) != cudaSuccess) {
      g_create_err = "event creation failed";
      aew_destroy(h);
      return AEW_E_CUDA;
    }
  h->stats.device_bytes = h->bytes + aew::codec_device_bytes(h->codec);
  h->stats.latent_bytes =
      c.storage != AEW_AE ? 0
      : h->tcodec         ? (size_t)nwin_of(h) * nvec_of(h) * c.n_lat * 2
                          : nt * (size_t)(c.nx / 8) * (c.ny / 8) * (c.nz / 8) * c.n_lat * 2;
  h->stats.history_bytes = c.storage == AEW_FULL      ? nt * C * 4
                           : c.storage == AEW_REVOLVE ? (size_t)c.n_checkpoints * 4 * C * 4
                                                      : h->stats.latent_bytes;
  *out = h;
  return AEW_OK;
}

void aew_destroy(aew_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < 2; ++i) {
    if (h->ev_a[i]) cudaEventDestroy(h->ev_a[i]);
    if (h->ev_b[i]) cudaEventDestroy(h->ev_b[i]);
  }
  for (int i = 0; i < 2; ++i) {
    if (h->tg[i]) cudaEventDestroy(h->tg[i]);
    if (h->th[i]) cudaEventDestroy(h->th[i]);
    if (h->ev_c[i]) cudaEventDestroy(h->ev_c[i]);
    if (h->ev_d[i]) cudaEventDestroy(h->ev_d[i]);
  }
  if (h->ev_sync) cudaEventDestroy(h->ev_sync);
  if (h->ev_sync2) cudaEventDestroy(h->ev_sync2);
  if (h->side) cudaStreamDestroy(h->side);
  for (void* p : h->allocs) cudaFree(p);
  if (h->codec) aew::codec_free(h->codec);
  delete h;
}

const char* aew_last_error(const aew_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

int aew_stats(const aew_handle* h, aew_stats_t* out) {
  if (!h || !out) return AEW_E_ARG;
  *out = h->stats;
  float ms = 0.f;
  if (h->tg_set && cudaEventQuery(h->tg[1]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, h->tg[0], h->tg[1]) == cudaSuccess)
    out->last_gradient_ms = ms;
  if (h->th_set && cudaEventQuery(h->th[1]) == cudaSuccess &&
      cudaEventElapsedTime(&ms, h->th[0], h->th[1]) == cudaSuccess)
    out->last_hessvec_ms = ms;
  cudaGetLastError();   // a query of an unfinished event is not an error of the handle
  return AEW_OK;
}

int aew_forward(aew_handle* h, const float* c_dev, const float* wavelet_host, float* d_dev,
                void* stream) {
  if (!h) return AEW_E_ARG;
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_c(h, c_dev, s);
  if (rc) return rc;
  h->have_grad = false;  // m changed: stored history no longer matches
  const float* wav = wav_or_default(h, wavelet_host);
  if ((rc = zero_state(h, h->st[0], s))) return rc;
  if (d_dev && h->nrow) AEW_CK(cudaMemsetAsync(d_dev, 0, h->nrow * sizeof(float), s));
  int cur = 0;
  for (int n = 0; n < h->cfg.nt; ++n) {
    rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], wav, d_dev ? drow(h, d_dev, n + 1) : nullptr,
                  s);
    if (rc) return rc;
    cur ^= 1;
  }
  return AEW_OK;
}

int aew_sync_check(aew_handle* h, void* stream) {
  if (!h) return AEW_E_ARG;
  h->err.clear();
  if (aew::codec_take_error(h->codec, S(stream)))
    return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
  return AEW_OK;
}

int aew_test_wait_timeout(aew_handle* h, unsigned long long wait_ns, void* stream) {
  if (!h || wait_ns == 0 || wait_ns > 1000000000ull) return AEW_E_ARG;
  h->err.clear();
  AEW_CK(aew::launch_wait_probe(aew::codec_err_flag(h->codec), wait_ns, S(stream)));
  ++h->stats.kernel_launches;
  return AEW_OK;
}

int aew_propagate(aew_handle* h, const float* c_dev, float* const state_dev[4], int n0,
                  int nsteps, const float* wavelet_host, float* d_dev, void* stream) {
  if (!h || !state_dev || nsteps < 0) return AEW_E_ARG;
  for (int i = 0; i < 4; ++i) {
    if (!state_dev[i]) return fail(h, AEW_E_ARG, "state pointer is NULL");
    if (reinterpret_cast<uintptr_t>(state_dev[i]) & 15)
      return fail(h, AEW_E_ARG, "state pointers must be 16-byte aligned");
  }
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_c(h, c_dev, s);
  if (rc) return rc;
  h->have_grad = false;
  if (d_dev && h->nrow) AEW_CK(cudaMemsetAsync(d_dev, 0, h->nrow * sizeof(float), s));
  float* tmp[4] = {h->st[0][0], h->st[0][1], h->st[0][2], h->st[0][3]};
  float* bufs[2][4] = {{state_dev[0], state_dev[1], state_dev[2], state_dev[3]},
                       {tmp[0], tmp[1], tmp[2], tmp[3]}};
  std::vector<float> w(wavelet_host ? (size_t)nsteps + (size_t)n0 : 0, 0.f);
  for (int k = 0; wavelet_host && k < nsteps; ++k) w[(size_t)n0 + k] = wavelet_host[k];
  int cur = 0;
  for (int k = 0; k < nsteps; ++k) {
    rc = fwd_step(h, n0 + k, bufs[cur], bufs[cur ^ 1], wavelet_host ? w.data() : nullptr,
                  d_dev ? drow(h, d_dev, k + 1) : nullptr, s);
    if (rc) return rc;
    cur ^= 1;
  }
  if (cur == 1) {
    if ((rc = copy_state(h, bufs[0], bufs[1], s))) return rc;
  }
  return AEW_OK;
}

// the gradient drivers with an optional Armijo gate (aew::gradient_gated)
static int gradient_impl(aew_handle* h, const float* c_dev, const float* d_obs_dev, float* g_dev,
                         double* misfit_host, double gate, bool* accepted, cudaStream_t s) {
  if (!h) return AEW_E_ARG;
  if (!d_obs_dev && h->nrow) return fail(h, AEW_E_ARG, "d_obs is NULL");
  if (!g_dev) return fail(h, AEW_E_ARG, "g is NULL");
  h->err.clear();
  if (accepted) *accepted = true;
  h->have_grad = false;
  if (h->cfg.storage == AEW_AE && !aew::codec_ready(h->codec))
    return fail(h, AEW_E_NOCODEC, "AE storage needs codec weights (aew_codec_set)");
  int rc = prepare_c(h, c_dev, s);
  if (rc) return rc;
  h->tg_set = false;
  AEW_CK(cudaEventRecord(h->tg[0], s));
  const float* wav = h->wav.data();
  h->gate = h->cfg.storage == AEW_REVOLVE ? INFINITY : gate;
  if (h->cfg.storage == AEW_FULL) {
    rc = gradient_full(h, d_obs_dev, wav, s);
  } else if (h->cfg.storage == AEW_REVOLVE) {
    long long fwd = 0;
    rc = run_revolve(h, d_obs_dev, nullptr, wav, true, s, &fwd);
    h->stats.forward_steps = fwd;
    h->stats.adjoint_steps = h->cfg.nt;
  } else if (h->tcodec) {
    rc = gradient_ae_time(h, d_obs_dev, wav, s);
  } else {
    rc = gradient_ae(h, d_obs_dev, wav, s);
  }
  h->gate = INFINITY;
  if (rc == kGated) {   // the misfit failed the gate: no adjoint solve, no gradient
    if (aew::codec_take_error(h->codec, s))
      return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
    if (misfit_host) *misfit_host = h->stats.last_misfit;
    if (accepted) *accepted = false;
    return AEW_OK;
  }
  if (rc) return rc;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
  AEW_CK(aew::launch_finalize_grad(h->c, h->acc64, g_dev, h->C, s));
  ++h->stats.kernel_launches;
  if (h->gc) AEW_CK(cudaMemcpyAsync(h->gc, g_dev, h->C * sizeof(float), cudaMemcpyDeviceToDevice, s));
  AEW_CK(cudaEventRecord(h->tg[1], s));
  h->tg_set = true;
  if (misfit_host || h->cfg.storage == AEW_AE) {
    double J = 0.0;
    int ovf = 0;
    AEW_CK(cudaMemcpyAsync(&J, h->part + aew::kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (h->cfg.storage == AEW_AE)
      AEW_CK(cudaMemcpyAsync(&ovf, h->ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
    AEW_CK(cudaStreamSynchronize(s));
    h->stats.last_misfit = J;
    h->stats.latent_overflow = ovf;
    if (misfit_host) *misfit_host = J;
    if (ovf) return fail(h, AEW_E_OVERFLOW, "a latent overflowed FP16 during encoding");
    if (accepted && J > gate) *accepted = false;   // revolve: tested after the adjoint
  }
  h->have_grad = true;
  return AEW_OK;
}

int aew_gradient(aew_handle* h, const float* c_dev, const float* d_obs_dev, float* g_dev,
                 double* misfit_host, void* stream) {
  return gradient_impl(h, c_dev, d_obs_dev, g_dev, misfit_host, INFINITY, nullptr, S(stream));
}

// incremental forward at the stored c: dd = J_F dc  (dm must be prepared)
static int incremental_forward(aew_handle* h, float* dd_out, cudaStream_t s, long long* fwd) {
  const int nt = h->cfg.nt;
  int rc;
  // incremental state in ad[] buffers (free until the incremental adjoint)
  if ((rc = zero_state(h, h->ad[0], s))) return rc;
  if (h->nrow) AEW_CK(cudaMemsetAsync(dd_out, 0, h->nrow * sizeof(float), s));
  int cur = 0, fcur = 0;
  *fwd = 0;
  if (h->cfg.storage == AEW_REVOLVE && (rc = zero_state(h, h->st[0], s))) return rc;
  const bool ae = h->cfg.storage == AEW_AE;
  if (ae && h->tcodec) {
    // decoder of window tb + 1 on the side stream while window tb's steps run on s;
    // ev_b[w % 2]: window w decoded, ev_a[w % 2]: window w's incremental steps done
    const int W = nwin_of(h), T = aew::kTSteps;
    if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
    if ((rc = decode_window(h, 0, h->side, true))) return rc;
    AEW_CK(cudaEventRecord(h->ev_b[0], h->side));
    for (int n = 0; n < nt; ++n) {
      const int tb = n / T;
      if (n % T == 0) {
        if (tb + 1 <= W - 1) {
          if (tb >= 1) AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(tb + 1) & 1], 0));
          if ((rc = decode_window(h, tb + 1, h->side, true))) return rc;
          AEW_CK(cudaEventRecord(h->ev_b[(tb + 1) & 1], h->side));
        }
        AEW_CK(cudaStreamWaitEvent(s, h->ev_b[tb & 1], 0));
      }
      if ((rc = incr_step(h, h->ad[cur], h->ad[cur ^ 1], nullptr, drow(h, dd_out, n + 1), s,
                          nullptr, 0, nullptr, window_e16(h, n))))
        return rc;
      if (n % T == T - 1 || n == nt - 1) AEW_CK(cudaEventRecord(h->ev_a[tb & 1], s));
      cur ^= 1;
      ++*fwd;
    }
    return join(h, h->side, s, h->ev_sync2);
  }
  if (ae) {
    // decode of step n+1 on the side stream while incremental step n runs on s;
    // edb[m % 2] is next read by incremental step m, previously by step m - 2
    if ((rc = join(h, s, h->side, h->ev_sync))) return rc;
    if (nt - 1 >= 1) {
      if ((rc = decode_e(h, 1, h->edb[1], h->side))) return rc;
      AEW_CK(cudaEventRecord(h->ev_b[1], h->side));
    }
  }
  for (int n = 0; n < nt; ++n) {
    const float* en = nullptr;
    if (ae) {
      if (n + 1 <= nt - 1 && n + 1 >= 2) {
        AEW_CK(cudaStreamWaitEvent(h->side, h->ev_a[(n + 1) & 1], 0));
        if ((rc = decode_e(h, n + 1, h->edb[(n + 1) & 1], h->side))) return rc;
        AEW_CK(cudaEventRecord(h->ev_b[(n + 1) & 1], h->side));
      }
      if (n >= 1) {
        AEW_CK(cudaStreamWaitEvent(s, h->ev_b[n & 1], 0));
        en = h->edb[n & 1];
      }
    } else if (n > 0 && h->cfg.storage == AEW_FULL) {
      en = h->estore + (size_t)n * h->C;
    }
    if (h->cfg.storage == AEW_REVOLVE) {
      if (n > 0) {  // lockstep forward recompute: state n from state n-1
        rc = fwd_step(h, n - 1, h->st[fcur], h->st[fcur ^ 1], h->wav.data(), nullptr, s);
        if (rc) return rc;
        fcur ^= 1;
        ++*fwd;
        en = h->st[fcur][0];
      }
    }
    if ((rc = incr_step(h, h->ad[cur], h->ad[cur ^ 1], en, drow(h, dd_out, n + 1), s))) return rc;
    if (ae) AEW_CK(cudaEventRecord(h->ev_a[n & 1], s));
    cur ^= 1;
    ++*fwd;
  }
  if (ae) return join(h, h->side, s, h->ev_sync2);
  return AEW_OK;
}

static int prepare_dc(aew_handle* h, const float* dc_dev, cudaStream_t s) {
  if (!dc_dev) return fail(h, AEW_E_ARG, "dc is NULL");
  if (!h->have_grad)
    return fail(h, AEW_E_NOGRADIENT, "no forward history: call aew_gradient first");
  AEW_CK(cudaMemsetAsync(h->chk, 0, sizeof(aew::FieldCheck), s));
  AEW_CK(aew::launch_prep_dm(h->c, dc_dev, h->dm, h->C, h->chk, s));
  ++h->stats.kernel_launches;
  aew::FieldCheck ck{};
  AEW_CK(cudaMemcpyAsync(&ck, h->chk, sizeof(ck), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  if (ck.nonfinite) return fail(h, AEW_E_NONFINITE, "dc contains NaN or Inf");
  return AEW_OK;
}

int aew_jvp(aew_handle* h, const float* dc_dev, float* dd_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!dd_dev && h->nrow) return fail(h, AEW_E_ARG, "dd is NULL");
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_dc(h, dc_dev, s);
  if (rc) return rc;
  long long fwd = 0;
  return incremental_forward(h, dd_dev, s, &fwd);
}

int aew_hessvec(aew_handle* h, const float* dc_dev, float* hdc_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!hdc_dev) return fail(h, AEW_E_ARG, "hdc is NULL");
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_dc(h, dc_dev, s);
  if (rc) return rc;
  h->th_set = false;
  AEW_CK(cudaEventRecord(h->th[0], s));
  long long fwd = 0;
  if ((rc = incremental_forward(h, h->dd, s, &fwd))) return rc;
  // incremental adjoint: the adjoint solve with residual dd (row 0 unused)
  const int nt = h->cfg.nt;
  if (h->cfg.storage == AEW_REVOLVE) {
    long long f2 = 0;
    if ((rc = run_revolve(h, nullptr, h->dd, h->wav.data(), false, s, &f2))) return rc;
    fwd += f2;
  } else if (h->cfg.storage == AEW_AE) {
    if ((rc = h->tcodec ? time_adjoint_sweep(h, h->dd, s) : ae_adjoint_sweep(h, h->dd, s)))
      return rc;
  } else {
    if ((rc = begin_adjoint(h, s))) return rc;
    int acur = 0;
    for (int n = nt - 1; n >= 0; --n) {
      const float* en = n > 0 ? h->estore + (size_t)n * h->C : nullptr;
      if ((rc = adj_step(h, n, acur, h->dd, en, s))) return rc;
      acur ^= 1;
    }
  }
  h->stats.hvp_forward_steps = fwd;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
  AEW_CK(aew::launch_finalize_grad(h->c, h->acc64, hdc_dev, h->C, s));
  ++h->stats.kernel_launches;
  AEW_CK(cudaEventRecord(h->th[1], s));
  h->th_set = true;
  return AEW_OK;
}

int aew_hessvec_full(aew_handle* h, const float* dc_dev, float* hdc_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!hdc_dev) return fail(h, AEW_E_ARG, "hdc is NULL");
  if (!h->gc)
    return fail(h, AEW_E_CONFIG, "the full Newton HVP needs full storage or the time codec");
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_dc(h, dc_dev, s);
  if (rc) return rc;
  if ((rc = ensure_newton(h))) return rc;
  h->th_set = false;
  AEW_CK(cudaEventRecord(h->th[0], s));
  if ((rc = newton_incremental_forward(h, s))) return rc;
  if ((rc = newton_adjoint_sweep(h, s))) return rc;
  h->stats.hvp_forward_steps = h->cfg.nt;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
  AEW_CK(aew::launch_finalize_hvp_full(h->c, dc_dev, h->acc64, h->acc64b, h->gc, hdc_dev, h->C, s));
  ++h->stats.kernel_launches;
  AEW_CK(cudaEventRecord(h->th[1], s));
  h->th_set = true;
  if (h->cfg.storage == AEW_AE) {
    int ovf = 0;
    AEW_CK(cudaMemcpyAsync(&ovf, h->ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
    AEW_CK(cudaStreamSynchronize(s));
    if (ovf) return fail(h, AEW_E_OVERFLOW, "a latent overflowed FP16 during encoding");
  }
  return AEW_OK;
}

int aew_test_gelu(const float* x_dev, float* y_dev, float* dy_dev, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !y_dev || !dy_dev))) return AEW_E_ARG;
  return aew::launch_activation_probe(x_dev, y_dev, dy_dev, n, S(stream)) == cudaSuccess
             ? AEW_OK
             : AEW_E_CUDA;
}

int aew_dot(const float* a_dev, const float* b_dev, size_t n, double* out_host, void* stream) {
  if (!a_dev || !b_dev || !out_host) return AEW_E_ARG;
  cudaStream_t s = S(stream);
  double* part = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&part), (aew::kRedBlocks + 1) * sizeof(double), s) !=
      cudaSuccess)
    return AEW_E_NOMEM;
  int rc = AEW_OK;
  if (aew::launch_dot_partials(a_dev, b_dev, n, part, aew::kRedBlocks, s) != cudaSuccess ||
      aew::launch_sum_partials(part, aew::kRedBlocks, 1.0, part + aew::kRedBlocks, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(out_host, part + aew::kRedBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess)
    rc = AEW_E_CUDA;
  cudaFreeAsync(part, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = AEW_E_CUDA;
  return rc;
}

int aew_revolve_plan(int nt, int s, int* ops, int* args, long long cap, long long* n_ops,
                     long long* fwd_steps) {
  if (nt < 1 || s < 0 || !n_ops || !fwd_steps) return AEW_E_ARG;
  std::vector<aew::RevAction> plan;
  const long long f = aew::revolve_plan(nt, s, plan);
  if (f < 0) return AEW_E_ARG;
  *n_ops = (long long)plan.size();
  *fwd_steps = f;
  for (long long i = 0; i < (long long)plan.size() && i < cap; ++i) {
    if (ops) ops[i] = plan[i].op;
    if (args) args[i] = plan[i].arg;
  }
  return AEW_OK;
}

// ------------------------------------------------------------------------------ codec
int aew_codec_set(aew_handle* h, const float* W1, const float* b1, const float* W2,
                  const float* b2, const float* W3, const float* b3, const float* W4,
                  const float* b4) {
  if (!h) return AEW_E_ARG;
  const float* w[8] = {W1, b1, W2, b2, W3, b3, W4, b4};
  for (const float* p : w)
    if (!p) return fail(h, AEW_E_ARG, "weight pointer is NULL");
  cudaError_t e = aew::codec_set_weights(h->codec, w);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_set_weights");
  return AEW_OK;
}

int aew_codec_get(const aew_handle* h, float* W1, float* b1, float* W2, float* b2, float* W3,
                  float* b3, float* W4, float* b4) {
  if (!h) return AEW_E_ARG;
  float* w[8] = {W1, b1, W2, b2, W3, b3, W4, b4};
  for (float* p : w)
    if (!p) return AEW_E_ARG;
  if (!aew::codec_ready(h->codec)) return AEW_E_NOCODEC;
  return aew::codec_get_weights(h->codec, w) == cudaSuccess ? AEW_OK : AEW_E_CUDA;
}

int aew_codec_encode(aew_handle* h, const float* const fields_dev[4], uint16_t* latents_dev,
                     float* block_max_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (h->tcodec) return fail(h, AEW_E_CONFIG, "aew_codec_encode needs the space codec");
  if (!fields_dev || !latents_dev) return fail(h, AEW_E_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(latents_dev) & 31)
    return fail(h, AEW_E_ARG, "latents_dev must be 32-byte aligned");
  if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 8)
    return fail(h, AEW_E_CONFIG, "codec needs nx, ny, nz multiples of 8");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaStream_t s = S(stream);
  const size_t nb = nblocks_of(h);
  if (!h->bm_tmp && !dalloc(h, &h->bm_tmp, 2 * nb * 4)) return fail(h, AEW_E_NOMEM, "workspace");
  int* ovf = reinterpret_cast<int*>(h->scratch8 + 4);
  AEW_CK(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  const float* f[4] = {fields_dev[0], fields_dev[1], fields_dev[2], fields_dev[3]};
  cudaError_t e = aew::codec_encode_grid(h->codec, f, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->bm_tmp,
                                         latents_dev, ovf, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_grid");
  if (block_max_dev)
    AEW_CK(cudaMemcpyAsync(block_max_dev, h->bm_tmp, nb * 4 * sizeof(float),
                           cudaMemcpyDeviceToDevice, s));
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  int o = 0;
  AEW_CK(cudaMemcpyAsync(&o, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  if (o) return fail(h, AEW_E_OVERFLOW, "a latent overflowed FP16");
  return AEW_OK;
}

int aew_codec_decode(aew_handle* h, const uint16_t* latents_dev, long long n, float* out_dev,
                     void* stream) {
  if (!h) return AEW_E_ARG;
  if (!latents_dev || !out_dev || n < 0) return fail(h, AEW_E_ARG, "bad argument");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  if (n == 0) return AEW_OK;
  cudaError_t e = aew::codec_decode_vectors(h->codec, latents_dev, n, out_dev, S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_vectors");
  if (aew::codec_take_error(h->codec, S(stream)))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  return AEW_OK;
}

int aew_codec_decode_e(aew_handle* h, const uint16_t* latents_dev, const float* block_max_dev,
                       float* e_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (h->tcodec) return fail(h, AEW_E_CONFIG, "aew_codec_decode_e needs the space codec");
  if (!latents_dev || !block_max_dev || !e_dev) return fail(h, AEW_E_ARG, "NULL argument");
  if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 8)
    return fail(h, AEW_E_CONFIG, "codec needs nx, ny, nz multiples of 8");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaError_t e = aew::codec_decode_grid_e(h->codec, latents_dev, h->cfg.nx, h->cfg.ny, h->cfg.nz,
                                           reinterpret_cast<const unsigned*>(block_max_dev), e_dev,
                                           S(stream));
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_grid_e");
  if (aew::codec_take_error(h->codec, S(stream)))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  return AEW_OK;
}

int aew_codec_encode_vectors(aew_handle* h, const uint16_t* vectors_dev, long long n,
                             uint16_t* latents_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!vectors_dev || !latents_dev || n < 0) return fail(h, AEW_E_ARG, "bad argument");
  if (reinterpret_cast<uintptr_t>(latents_dev) & 31)
    return fail(h, AEW_E_ARG, "latents_dev must be 32-byte aligned");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  if (n == 0) return AEW_OK;
  cudaStream_t s = S(stream);
  int* ovf = reinterpret_cast<int*>(h->scratch8 + 4);
  AEW_CK(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  cudaError_t e = aew::codec_encode_vectors(h->codec, vectors_dev, n, latents_dev, ovf, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_vectors");
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  int o = 0;
  AEW_CK(cudaMemcpyAsync(&o, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  if (o) return fail(h, AEW_E_OVERFLOW, "a latent overflowed FP16");
  return AEW_OK;
}

int aew_codec_encode_window(aew_handle* h, const float* e_dev, int nsteps, uint16_t* latents_dev,
                            void* scale_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!h->tcodec) return fail(h, AEW_E_CONFIG, "aew_codec_encode_window needs the time codec");
  if (!e_dev || !latents_dev || nsteps < 1 || nsteps > aew::kTSteps)
    return fail(h, AEW_E_ARG, "bad argument");
  if (reinterpret_cast<uintptr_t>(e_dev) & 15) return fail(h, AEW_E_ARG, "e_dev must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(latents_dev) & 31)
    return fail(h, AEW_E_ARG, "latents_dev must be 32-byte aligned");
  if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 2)
    return fail(h, AEW_E_CONFIG, "the time codec needs nx, ny multiples of 8 and nz even");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaStream_t s = S(stream);
  const size_t nv = nvec_of(h);
  const bool mm = aew::codec_minmax(h->codec);
  if ((!h->wk_raw && !dalloc(h, &h->wk_raw, nv * aew::kNIn)) ||
      (!h->wk_vmax && !dalloc(h, &h->wk_vmax, nv)) ||
      (mm && !h->wk_mr && !dalloc(h, &h->wk_mr, 2 * nv)))
    return fail(h, AEW_E_NOMEM, "workspace");
  int* ovf = reinterpret_cast<int*>(h->scratch8 + 4);
  AEW_CK(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  AEW_CK(aew::window_pack(e_dev, nsteps, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->wk_raw, h->wk_vmax, s));
  cudaError_t e = aew::codec_encode_window(h->codec, h->wk_raw, h->wk_vmax, (long long)nv,
                                           latents_dev, ovf, s, 0, mm ? h->wk_mr : nullptr,
                                           mm ? h->wk_mr + nv : nullptr);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_encode_window");
  h->stats.kernel_launches += mm ? 4 : 3;
  if (scale_dev)
    AEW_CK(cudaMemcpyAsync(scale_dev, mm ? static_cast<const void*>(h->wk_mr) : h->wk_vmax,
                           mm ? 2 * nv * sizeof(double) : nv * sizeof(float),
                           cudaMemcpyDeviceToDevice, s));
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  int o = 0;
  AEW_CK(cudaMemcpyAsync(&o, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
  AEW_CK(cudaStreamSynchronize(s));
  if (o) return fail(h, AEW_E_OVERFLOW, "a latent overflowed FP16");
  return AEW_OK;
}

int aew_codec_decode_window(aew_handle* h, const uint16_t* latents_dev, const void* scale_dev,
                            float* e_dev, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!h->tcodec) return fail(h, AEW_E_CONFIG, "aew_codec_decode_window needs the time codec");
  if (!latents_dev || !scale_dev || !e_dev) return fail(h, AEW_E_ARG, "NULL argument");
  if (reinterpret_cast<uintptr_t>(e_dev) & 15) return fail(h, AEW_E_ARG, "e_dev must be 16-byte aligned");
  if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 2)
    return fail(h, AEW_E_CONFIG, "the time codec needs nx, ny multiples of 8 and nz even");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaStream_t s = S(stream);
  const bool mm = aew::codec_minmax(h->codec);
  const size_t nv = nvec_of(h);
  const double* mr = static_cast<const double*>(scale_dev);
  cudaError_t e = aew::codec_decode_window(h->codec, latents_dev,
                                           static_cast<const unsigned*>(scale_dev), h->cfg.nx,
                                           h->cfg.ny, h->cfg.nz, e_dev, s, 0, mm ? mr : nullptr,
                                           mm ? mr + nv : nullptr);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_decode_window");
  h->stats.kernel_launches += 2;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  return AEW_OK;
}

int aew_codec_init_pca(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                       long long n, int loss, double* eigvals_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!vectors_dev || n < 1) return fail(h, AEW_E_ARG, "bad argument");
  if (reinterpret_cast<uintptr_t>(vectors_dev) & 15)
    return fail(h, AEW_E_ARG, "vectors_dev must be 16-byte aligned");
  const bool weighted = loss == AEW_LOSS_STRAIN_AMPLITUDE || loss == AEW_LOSS_STRAIN_ENERGY;
  if (loss != AEW_LOSS_STATE && !(h->tcodec && (loss == AEW_LOSS_STRAIN || weighted)))
    return fail(h, AEW_E_ARG, "PCA weights: AEW_LOSS_STATE, or a strain loss with the time codec");
  if (weighted && !maxima_dev) return fail(h, AEW_E_ARG, "weighted PCA needs the vectors' maxima");
  const int k = h->cfg.n_lat, nh = aew::codec_nhid(h->codec), I = aew::kNIn;
  if (2 * k > nh) return fail(h, AEW_E_CONFIG, "the hidden layer must hold 2 n_lat units");
  if (h->cfg.act != AEW_ACT_GELU)
    return fail(h, AEW_E_CONFIG, "the PCA code passes GELU(a) - GELU(-a) = a: GELU only");
  if (aew::codec_minmax(h->codec) && weighted)
    return fail(h, AEW_E_ARG, "min-max normalisation: unweighted PCA only");
  h->err.clear();
  cudaStream_t s = S(stream);
  double* G = nullptr;
  double* sm = nullptr;
  float* wv = nullptr;
  if (cudaMalloc(&G, (size_t)I * I * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&sm, (I + 1) * sizeof(double)) != cudaSuccess ||
      (weighted && cudaMalloc(&wv, (size_t)n * sizeof(float)) != cudaSuccess)) {
    cudaGetLastError();
    cudaFree(G);
    cudaFree(sm);
    cudaFree(wv);
    return fail(h, AEW_E_NOMEM, "moment buffers");
  }
  std::vector<double> Gh((size_t)I * I), sh(I + 1);
  cudaError_t e = cudaSuccess;
  if (weighted)   // w_v = s_v (amplitude) or s_v^2 (energy): the scales are powers of two
    e = aew::vector_weights(maxima_dev, n, loss == AEW_LOSS_STRAIN_AMPLITUDE ? 1 : 2, wv, s);
  if (e == cudaSuccess) e = aew::codec_moments(h->codec, vectors_dev, n, wv, G, sm, s);
  cudaFree(wv);
  if (e == cudaSuccess) e = cudaMemcpy(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(sh.data(), sm, sh.size() * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(G);
  cudaFree(sm);
  h->stats.kernel_launches += 2 + 2 * ((n + 32767) / 32768);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_moments");
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  const double sw = sh[I];
  if (!(sw > 0)) return fail(h, AEW_E_ARG, "the weights sum to zero");
  // weighted covariance (G / sw - mu mu^T), its eigenvectors, the rank-k pair code
  std::vector<double> mu(I), C((size_t)I * I), w(I), V((size_t)I * I);
  for (int i = 0; i < I; ++i) mu[i] = sh[i] / sw;
  for (int i = 0; i < I; ++i)
    for (int j = 0; j < I; ++j) C[(size_t)i * I + j] = Gh[(size_t)i * I + j] / sw - mu[i] * mu[j];
  if (!aew::sym_eig(I, C.data(), w.data(), V.data()))
    return fail(h, AEW_E_CUDA, "the symmetric eigensolver did not converge");
  const size_t szs[8] = {(size_t)I * nh, (size_t)nh, (size_t)nh * k, (size_t)k,
                         (size_t)k * nh, (size_t)nh, (size_t)nh * I, (size_t)I};
  std::vector<std::vector<float>> W(8);
  for (int i = 0; i < 8; ++i) W[i].resize(szs[i]);
  aew::pca_pair_weights(I, nh, k, mu.data(), V.data(), W[0].data(), W[1].data(), W[2].data(),
                        W[3].data(), W[4].data(), W[5].data(), W[6].data(), W[7].data());
  const float* wp[8];
  for (int i = 0; i < 8; ++i) wp[i] = W[i].data();
  e = aew::codec_set_weights(h->codec, wp);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_set_weights");
  aew::codec_reset_training(h->codec);
  if (eigvals_host) std::memcpy(eigvals_host, w.data(), I * sizeof(double));
  return AEW_OK;
}

int aew_profile_steps(aew_handle* h, const float* c_dev, int kind, int nsteps, double* ms_host,
                      void* stream) {
  if (!h) return AEW_E_ARG;
  if (kind < 0 || kind > 9 || nsteps < 1 || !ms_host) return fail(h, AEW_E_ARG, "bad argument");
  const bool tw = h->cfg.storage == AEW_AE && h->tcodec;
  if ((kind == 1 || kind == 4 || kind == 5 || kind == 7) && !tw)
    return fail(h, AEW_E_CONFIG, "this kernel needs AE storage with the time codec");
  if (kind == 9 && !(h->cfg.storage == AEW_AE && !h->tcodec))
    return fail(h, AEW_E_CONFIG, "this kernel needs AE storage with the space codec");
  if ((kind == 4 || kind == 5 || kind == 7 || kind == 9) && !aew::codec_ready(h->codec))
    return fail(h, AEW_E_NOCODEC, "codec weights not set");
  if ((kind == 6 || kind == 8) && h->cfg.nx % 8)
    return fail(h, AEW_E_CONFIG, "a BF16 strain field needs nx % 8 == 0");
  h->err.clear();
  cudaStream_t s = S(stream);
  int rc = prepare_c(h, c_dev, s);
  if (rc) return rc;
  h->have_grad = false;
  const int nt = h->cfg.nt, T = aew::kTSteps;
  cudaEvent_t e0, e1;
  AEW_CK(cudaEventCreate(&e0));
  AEW_CK(cudaEventCreate(&e1));
  AEW_CK(cudaEventRecord(e0, s));
  int cur = 0;
  for (int k = 0; k < nsteps && rc == AEW_OK; ++k) {
    const int n = k % nt;
    switch (kind) {
      case 0:
        rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], h->wav.data(), nullptr, s);
        break;
      case 1:
        rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], h->wav.data(), nullptr, s, nullptr,
                      nullptr, nullptr, h->xt[0], (n + 1) % T, h->vmx);
        break;
      case 2:
        rc = adj_step(h, nt - 1 - n, cur, h->R, h->st[0][0], s);
        break;
      case 3:
        rc = incr_step(h, h->ad[cur], h->ad[cur ^ 1], h->st[0][0], nullptr, s);
        break;
      case 4:
        rc = encode_window(h, 0, s);
        break;
      case 5:
        rc = decode_window(h, 0, s);
        break;
      case 6:   // the adjoint step reading its strain field as BF16 (time-codec sweeps)
        rc = adj_step_x(h, nt - 1 - n, h->ad[cur], h->ad[cur ^ 1], h->R, nullptr, h->acc32,
                        h->acc64, nullptr, nullptr, nullptr, s,
                        reinterpret_cast<const uint16_t*>(h->st[0][0]));
        break;
      case 7:
        rc = decode_window(h, 0, s, true);
        break;
      case 8:   // the incremental forward step reading its strain field as BF16
        rc = incr_step(h, h->ad[cur], h->ad[cur ^ 1], nullptr, nullptr, s, nullptr, 0, nullptr,
                       reinterpret_cast<const uint16_t*>(h->st[0][0]));
        break;
      case 9:   // the space codec's fused strain decoder, step 0's latents
        rc = decode_e(h, 0, h->st[1][0], s);
        break;
    }
    cur ^= 1;
  }
  AEW_CK(cudaEventRecord(e1, s));
  AEW_CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a kernel gave up waiting (bounded mbarrier wait)");
  *ms_host = ms / nsteps;
  return AEW_OK;
}

int aew_sym_eig(int n, const double* A_host, double* w_host, double* V_host) {
  if (n < 1 || !A_host || !w_host || !V_host) return AEW_E_ARG;
  return aew::sym_eig(n, A_host, w_host, V_host) ? AEW_OK : AEW_E_ARG;
}

int aew_snapshots(aew_handle* h, const float* c_dev, int every, uint16_t* out_dev,
                  long long max_vectors, float* block_max_dev, long long* n_written,
                  void* stream) {
  if (!h) return AEW_E_ARG;
  if (!out_dev || !n_written || every < 1 || max_vectors < 0)
    return fail(h, AEW_E_ARG, "bad argument");
  if (reinterpret_cast<uintptr_t>(out_dev) & 15)
    return fail(h, AEW_E_ARG, "out_dev must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(block_max_dev) & 15)
    return fail(h, AEW_E_ARG, "block_max_dev must be 16-byte aligned");
  h->err.clear();
  cudaStream_t s = S(stream);
  if (h->tcodec) {
    if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 2)
      return fail(h, AEW_E_CONFIG, "time-codec snapshots need nx, ny multiples of 8 and nz even");
    int rc = prepare_c(h, c_dev, s);
    if (rc) return rc;
    h->have_grad = false;
    return snapshots_time(h, every, out_dev, max_vectors, block_max_dev, n_written, s);
  }
  if (h->cfg.nx % 8 || h->cfg.ny % 8 || h->cfg.nz % 8)
    return fail(h, AEW_E_CONFIG, "snapshots need nx, ny, nz multiples of 8");
  int rc = prepare_c(h, c_dev, s);
  if (rc) return rc;
  h->have_grad = false;
  const size_t nb = nblocks_of(h);
  // without block_max_dev the maxima go to two alternating scratch slices (a step reads
  // one state's and writes the next one's)
  if (!block_max_dev && !h->bm_tmp && !dalloc(h, &h->bm_tmp, 2 * nb * 4))
    return fail(h, AEW_E_NOMEM, "workspace");
  if ((rc = zero_state(h, h->st[0], s))) return rc;
  int cur = 0;
  long long written = 0;
  const int nt = h->cfg.nt;
  // state n (1 <= n < nt, n % every == 0) is packed by the forward step that reads it:
  // step n, or one extra step past the end for the state nt - 1; its maxima come from
  // step n - 1, which wrote the state
  auto packs = [&](int n, long long w) {
    return n >= 1 && n < nt && n % every == 0 && w + (long long)nb <= max_vectors;
  };
  auto bm_at = [&](long long w) {
    return block_max_dev ? reinterpret_cast<unsigned*>(block_max_dev) + (size_t)w * 4
                         : h->bm_tmp + ((size_t)(w / (long long)nb) & 1) * nb * 4;
  };
  for (int n = 0; n < nt; ++n) {
    const bool pack = packs(n, written);
    if (n + 1 == nt && !pack) break;
    const long long wnext = written + (pack ? (long long)nb : 0);
    uint16_t* xp = pack ? out_dev + (size_t)written * aew::kNIn : nullptr;
    const unsigned* bin = pack ? bm_at(written) : nullptr;
    unsigned* bout = packs(n + 1, wnext) ? bm_at(wnext) : nullptr;
    if ((rc = fwd_step(h, n, h->st[cur], h->st[cur ^ 1], h->wav.data(), nullptr, s, xp, bin,
                       bout)))
      return rc;
    cur ^= 1;
    written = wnext;
  }
  AEW_CK(cudaStreamSynchronize(s));
  *n_written = written;
  return AEW_OK;
}

int aew_codec_train(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                    long long n, const aew_train_cfg* cfg, double* epoch_loss_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!vectors_dev || !cfg || n < 1) return fail(h, AEW_E_ARG, "bad argument");
  if (cfg->loss < AEW_LOSS_STATE || cfg->loss > AEW_LOSS_STRAIN_ENERGY)
    return fail(h, AEW_E_ARG, "unknown loss");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  if (reinterpret_cast<uintptr_t>(vectors_dev) & 15)
    return fail(h, AEW_E_ARG, "vectors_dev must be 16-byte aligned");
  h->err.clear();
  cudaStream_t s = S(stream);
  aew::TrainCfg tc{cfg->epochs, cfg->batch, cfg->halve_every, cfg->loss, cfg->lr0, cfg->seed};
  cudaError_t e = aew::codec_train(h->codec, vectors_dev, maxima_dev, n, tc, epoch_loss_host, s,
                                   &h->err);
  if (e == cudaErrorInvalidValue && !h->err.empty()) return AEW_E_ARG;
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_train");
  h->stats.kernel_launches += (long long)cfg->epochs * (n / (cfg->batch > 0 ? cfg->batch : 1)) * 30;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  return AEW_OK;
}

int aew_codec_eval(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                   long long n, double* err_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!vectors_dev || !maxima_dev || !err_host || n < 1) return fail(h, AEW_E_ARG, "bad argument");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaStream_t s = S(stream);
  cudaError_t e = aew::codec_eval(h->codec, vectors_dev, maxima_dev, n, err_host, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_eval");
  h->stats.kernel_launches += 3 * ((n + 16383) / 16384) + 2;
  if (aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  h->stats.decoded_err_normalised = err_host[0];
  h->stats.decoded_err_physical = err_host[5];
  return AEW_OK;
}

int aew_codec_train_step(aew_handle* h, const uint16_t* batch_dev, const float* weights_dev,
                         int batch, float lr, float* loss_host, void* stream) {
  if (!h) return AEW_E_ARG;
  if (!batch_dev || batch < 1) return fail(h, AEW_E_ARG, "bad batch");
  if (!aew::codec_ready(h->codec)) return fail(h, AEW_E_NOCODEC, "codec weights not set");
  h->err.clear();
  cudaStream_t s = S(stream);
  float* loss_dev = h->scratch8;
  cudaError_t e =
      aew::codec_train_step(h->codec, batch_dev, weights_dev, batch, lr, loss_dev, s, &h->err);
  if (e != cudaSuccess) return cuda_fail(h, e, "codec_train_step");
  if (loss_host && aew::codec_take_error(h->codec, s))
    return fail(h, AEW_E_TIMEOUT, "a codec kernel gave up waiting (bounded mbarrier wait)");
  if (loss_host) {
    AEW_CK(cudaMemcpyAsync(loss_host, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, s));
    AEW_CK(cudaStreamSynchronize(s));
  }
  return AEW_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Internal interface of the optimisation drivers (aew_solver.h)
// ---------------------------------------------------------------------------------
namespace aew {

GridInfo grid_of(const aew_handle* h) {
  return GridInfo{h->cfg.nx, h->cfg.ny, h->cfg.nz, h->cfg.h, h->C};
}

int set_error(aew_handle* h, int code, const std::string& msg) { return fail(h, code, msg); }

int gradient_gated(aew_handle* h, const float* c_dev, const float* d_obs_dev, float* g_dev,
                   double gate, double* misfit, bool* accepted, cudaStream_t s) {
  double J = 0.0;
  const int rc = gradient_impl(h, c_dev, d_obs_dev, g_dev, &J, gate, accepted, s);
  if (misfit) *misfit = J;
  return rc;
}

}  // namespace aew
