/*
 * aewave -- autoencoder-compressed adjoint gradients and Gauss-Newton Hessian-vector
 * products for the 3-D acoustic velocity-strain wave equation, on one GB300 (sm_103a).
 *
 * The operations follow the statement of the inverse problem in Sec. 2 of
 * "An Autoencoder Compression Approach for Accelerating Large-scale Inverse Problems"
 * (arXiv 2304.04781):
 *   forward  : c -> d = F(c) = B A(c)                 (parameter-to-observable map, Sec. 2)
 *   gradient : c, d_obs -> J, dJ/dc, J = 1/2 |F(c) - d_obs|^2   (Eq. (3), misfit term)
 *   hessvec  : dc -> J_F^T J_F dc                      (incremental forward + incremental
 *                                                       adjoint, Sec. 4)
 * with the forward history kept in one of three ways: full storage, binomial
 * recompute-checkpointing, or autoencoder latents -- of every state's 8x8x8-node
 * blocks (compression in space, Sec. 3.1) or of the strain of 2x8x8-node blocks over
 * 16 consecutive steps (compression in time, Sec. 3.2); architecture and training of
 * Sec. 3.3, data generation of Algorithm 1.
 *
 * Discretisation (the same in every mode): nodes [k][j][i] = (z, y, x), row-major with
 * x fastest, spacing h, rho = 1, m = c^2.  e lives on nodes and is 0 on boundary
 * nodes; vx lives on x-faces (i+1/2, j, k) stored at [k][j][i] (the last face,
 * i = nx-1, is unused and 0); vy, vz likewise.  One step n -> n+1:
 *     v^{n+1} = v^n + dt (G(m e^n) + s^n),   e^{n+1} = e^n + dt D v^{n+1},
 *     d^{n+1} = B v^{n+1},
 * G = forward differences, D = backward differences on interior nodes (D = -G^T),
 * dt = cfl * h / cmax, s^n a force on the z-face of the source node.
 *
 * Conventions for every call:
 *  - Array arguments named *_dev are DEVICE pointers owned by the caller (for example
 *    a torch tensor's data_ptr()), contiguous, FP32 unless stated.  Grid fields are
 *    [nz][ny][nx].  Receiver data are [nt+1][nrec][3] (row n = d^n, component x,y,z).
 *    Arguments named *_host are host pointers.  The library never frees caller memory.
 *  - The handle owns every internal buffer (states, stored history, latents,
 *    checkpoints, workspace) and frees them in aew_destroy.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream).
 *    Calls that return a host scalar (misfit, dot) synchronise that stream.
 *  - Return value: AEW_OK (0) or a negative AEW_E_* code; aew_last_error() then gives
 *    a message.  A failed call leaves the handle usable.
 *  - Device waits are bounded.  A kernel whose wait gives up sets the handle's sticky
 *    device error flag and returns; later kernels of the handle see the flag and return
 *    at once.  Calls that synchronise (aew_gradient, aew_hessvec, the codec calls) and
 *    aew_sync_check read and clear the flag and report AEW_E_TIMEOUT; the asynchronous
 *    solves (aew_forward, aew_propagate, aew_jvp) leave it for the next such call.
 *  - A handle is not thread-safe: one call at a time per handle.
 */
#ifndef AEWAVE_H
#define AEWAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aew_handle aew_handle;

/* Storage of the forward history used by the adjoint and incremental solves. */
enum {
  AEW_FULL = 0,     /* every strain e^n kept in HBM (FP32, nt * nx*ny*nz floats)       */
  AEW_REVOLVE = 1,  /* binomial recompute-checkpointing with n_checkpoints state slots  */
  AEW_AE = 2        /* the history encoded to FP16 latents by the autoencoder codec     */
};

/* Codec kind of AEW_AE storage. */
enum {
  AEW_CODEC_SPACE = 0,  /* per state: 8x8x8-node blocks x 4 fields (e, vx, vy, vz)        */
  AEW_CODEC_TIME = 1    /* per 16-step window: the strain of 2x8x8-node blocks            */
};

/* Normalisation and activation of the time codec: the default power-of-two vector
 * scale with GELU, or the paper's per-vector min-max normalisation to [0, 1] (offset and
 * range kept in FP64, the range floored at beta; Sec. 3.3) and its ELU. */
enum {
  AEW_NORM_POW2 = 0,
  AEW_NORM_MINMAX = 1
};
enum {
  AEW_ACT_GELU = 0,
  AEW_ACT_ELU = 1    /* e^a - 1 below 0, a above */
};

/* Error codes. */
enum {
  AEW_OK = 0,
  AEW_E_CONFIG = -1,      /* invalid configuration (sizes, spacing, receivers, ...)    */
  AEW_E_CFL = -2,         /* max c violates the stability bound c dt / h <= 1/sqrt(3)  */
  AEW_E_NONFINITE = -3,   /* NaN or Inf in an input field                              */
  AEW_E_NOCODEC = -4,     /* AE storage requested before codec weights were set        */
  AEW_E_NOGRADIENT = -5,  /* hessvec/jvp with no stored forward history for this c     */
  AEW_E_NOMEM = -6,       /* device allocation failed                                  */
  AEW_E_CUDA = -7,        /* a CUDA runtime call or kernel launch failed               */
  AEW_E_OVERFLOW = -8,    /* a latent overflowed FP16                                  */
  AEW_E_ARG = -9,         /* NULL pointer or out-of-range argument                     */
  AEW_E_IO = -10,         /* file could not be read or written                         */
  AEW_E_TIMEOUT = -11,    /* a bounded device-side wait gave up                        */
  AEW_E_NOCONVERGE = -12  /* an iterative solve missed its tolerance                   */
};

typedef struct {
  int nx, ny, nz;         /* nodes per axis, each >= 4 and a multiple of 4; for
                             AEW_AE with the space codec multiples of 8 (8x8x8-node
                             blocks), with the time codec nx, ny multiples of 8 and
                             nz even (2x8x8-node blocks)                              */
  double h;               /* grid spacing [m]                                         */
  double cfl;             /* dt = cfl * h / cmax                                      */
  double cmax;            /* wave speed used for dt [m/s]                             */
  int nt;                 /* number of time steps (>= 1)                              */
  int src[3];             /* source node (i, j, k); the force acts on its z-face      */
  double f0, t0;          /* default source: s^n = -R(n dt), Ricker wavelet of Sec. 4.1
                             with peak frequency f0 [Hz] centred at t0 [s]            */
  int nrec;               /* number of receivers (>= 0)                               */
  const int* rec_ijk;     /* host [nrec][3] receiver nodes (i, j, k); all receivers
                             must share one k (a node plane), copied at create time   */
  int storage;            /* AEW_FULL, AEW_REVOLVE or AEW_AE                          */
  int n_checkpoints;      /* AEW_REVOLVE: number of state slots (>= 0)                */
  int accum_window;       /* steps summed in FP32 before each FP64 flush of the
                             gradient accumulator (>= 1; 8 is a good default)         */
  int n_lat;              /* codec latent width: space codec 64 (32x compression of
                             the 4-field state) or 32 (64x); time codec 512 (4x of the
                             strain values, 32x of the FP32 state's bytes) or 256     */
  int codec;              /* AEW_CODEC_SPACE (0) or AEW_CODEC_TIME (1)                */
  int norm;               /* time codec: AEW_NORM_POW2 (0) or AEW_NORM_MINMAX (1)     */
  int act;                /* time codec: AEW_ACT_GELU (0) or AEW_ACT_ELU (1)          */
  double beta;            /* AEW_NORM_MINMAX: floor of the range (0 = the paper's 1e-7)*/
  double src_sigma;       /* source smoothing in space [m] (Sec. 4.1's box problem): 0 is
                             the point force; > 0 spreads it over the z-faces within
                             R = ceil(3 src_sigma / h) faces of the source face with
                             weights exp(-r^2 / (2 src_sigma^2)) normalised to sum 1
                             (r: distance between face centres); the box must lie in
                             nodes 1 .. n-2 of every axis                             */
} aew_config;

typedef struct {
  size_t device_bytes;          /* bytes of device memory held by the handle         */
  size_t latent_bytes;          /* of which latent store (AEW_AE)                    */
  size_t history_bytes;         /* of which stored e^n (AEW_FULL) or checkpoints     */
  long long forward_steps;      /* forward leapfrog steps run by the last gradient   */
  long long adjoint_steps;      /* adjoint steps run by the last gradient            */
  long long hvp_forward_steps;  /* forward-type steps run by the last hessvec        */
  double last_misfit;           /* J of the last gradient                            */
  int latent_overflow;          /* 1 if a latent overflowed FP16 in the last encode  */
  long long kernel_launches;    /* kernels launched by this handle since creation    */
  double decoded_err_normalised; /* strain rel-L2 error of decode(encode(y)) in
                                    normalised units, from the last aew_codec_eval    */
  double decoded_err_physical;  /* the same in physical units (x = y s)              */
  double last_gradient_ms;      /* device time of the last aew_gradient (0 until it
                                   has finished on its stream)                       */
  double last_hessvec_ms;       /* device time of the last aew_hessvec (likewise)    */
} aew_stats_t;

/* Loss of the codec training: Table 2's mean squared reconstruction error, or a
 * weighted variant (each squared error of vector v in field f times w[v][f]). */
enum {
  AEW_LOSS_STATE = 0,             /* every output alike (Table 2)                          */
  AEW_LOSS_STRAIN = 1,            /* strain outputs only (the adjoint reads nothing else)  */
  AEW_LOSS_STRAIN_AMPLITUDE = 2,  /* strain only, each vector weighted by its strain scale
                                     s, divided by the data set's mean of s              */
  AEW_LOSS_STRAIN_ENERGY = 3      /* strain only, weighted by s^2 / mean(s^2): the
                                     squared error in physical units                     */
};

typedef struct {
  int epochs;               /* passes over the data (Table 2: 20; 0 = none)             */
  int batch;                /* minibatch size (Table 2: 512), a multiple of 8, <= n     */
  double lr0;               /* initial learning rate (Table 2: 1e-3)                    */
  int halve_every;          /* lr = lr0 * 0.5^(epoch / halve_every) (Table 2: 5;
                               <= 0: constant)                                          */
  int loss;                 /* AEW_LOSS_*                                               */
  unsigned long long seed;  /* seed of the per-epoch shuffles                           */
} aew_train_cfg;

/* ---------------------------------------------------------------------------------
 * Handle lifetime
 * ------------------------------------------------------------------------------- */

/* Validate `cfg`, allocate every buffer the storage mode needs on the current
 * device, and return a handle in *out.  Returns AEW_E_CONFIG / AEW_E_NOMEM on
 * failure (*out is then NULL).  The handle records the device that was current. */
int aew_create(const aew_config* cfg, aew_handle** out);

/* Free every buffer of the handle (synchronising the device first).  NULL is a no-op. */
void aew_destroy(aew_handle* h);

/* Message describing the last error on this handle ("" if none); valid until the
 * next call on the handle.  With h == NULL: the last error of aew_create. */
const char* aew_last_error(const aew_handle* h);

/* Counters and memory of the handle (host struct filled in). */
int aew_stats(const aew_handle* h, aew_stats_t* out);

/* ---------------------------------------------------------------------------------
 * Codec: the autoencoder of Sec. 3.1-3.3 (dense layers sigma(yW+b), Eq. (5)).
 * Encoder 2048 -> n_hid (GELU) -> n_lat; decoder n_lat -> n_hid (GELU) -> 2048, with
 * n_hid = 512 for the space codec and n_hid = 2 n_lat for the time codec.
 * Space codec, block vector order: k = z*256 + f*64 + y*8 + x, f = 0:e, 1:vx, 2:vy,
 * 3:vz (x, y, z node offsets inside the 8x8x8 block); block b = (bz*NBy + by)*NBx + bx.
 * Each field of each block is divided by its power-of-two scale (aew_codec_encode).
 * Time codec, window vector order: k = t*128 + z*64 + y*8 + x (t the step inside the
 * 16-step window of states e^{16w} .. e^{16w+15}; z, y, x the node offsets inside the
 * 2x8x8 block); vector v = (bz*NBy + by)*NBx + bx with NBz = nz/2, NBy = ny/8,
 * NBx = nx/8; states past nt - 1 are 0.  The whole vector is divided by its
 * power-of-two scale s = 2^max(e, -100), m 2^e (m in [0.5, 1)) its largest |e|.
 * Either way encoder inputs lie in (-1, 1) whatever the amplitude.
 * Precision: BF16 operands (FP16 for the decoder's first layer, whose input is the
 * FP16 latent) with FP32 accumulation on tcgen05 tensor cores; FP32 biases and GELU.
 * ------------------------------------------------------------------------------- */

/* Set the codec weights from host FP32 arrays, row-major, layer y -> y W + b:
 * W1 [2048][n_hid], b1 [n_hid], W2 [n_hid][n_lat], b2 [n_lat],
 * W3 [n_lat][n_hid], b3 [n_hid], W4 [n_hid][2048], b4 [2048].  Copied; not retained. */
int aew_codec_set(aew_handle* h, const float* W1_host, const float* b1_host,
                  const float* W2_host, const float* b2_host,
                  const float* W3_host, const float* b3_host,
                  const float* W4_host, const float* b4_host);

/* Copy the current FP32 master weights out (same shapes as aew_codec_set). */
int aew_codec_get(const aew_handle* h, float* W1_host, float* b1_host,
                  float* W2_host, float* b2_host,
                  float* W3_host, float* b3_host,
                  float* W4_host, float* b4_host);

/* Space codec only (AEW_E_CONFIG otherwise).  Encode one state.
 * fields_dev = {e, vx, vy, vz} device [nz][ny][nx];
 * latents_dev: device FP16 [nblocks][n_lat] (written; 32-byte aligned, AEW_E_ARG
 * otherwise: each lane stores 32 bytes of a row at once).  Each field of each block is
 * normalised by its own power-of-two scale s = 2^e, where max |f| over the block is
 * m 2^e with m in [0.5, 1) (the per-vector normalisation of Sec. 3.3); block_max_dev
 * (may be NULL): device FP32 [nblocks][4] receiving the block maxima m 2^e from which
 * the scales follow. */
int aew_codec_encode(aew_handle* h, const float* const fields_dev[4], uint16_t* latents_dev,
                     float* block_max_dev, void* stream);

/* Encode normalised block vectors (e.g. training snapshots): vectors_dev = device
 * BF16 bit patterns [n][2048] in the block-vector order above; latents_dev: device
 * FP16 [n][n_lat] (written; 32-byte aligned, AEW_E_ARG otherwise). */
int aew_codec_encode_vectors(aew_handle* h, const uint16_t* vectors_dev, long long n,
                             uint16_t* latents_dev, void* stream);

/* Decode n latent vectors (FP16 [n][n_lat]).  out_dev: device FP32 [n][2048]
 * normalised block vectors (all four fields, not multiplied by any scale). */
int aew_codec_decode(aew_handle* h, const uint16_t* latents_dev, long long n, float* out_dev,
                     void* stream);

/* Space codec only (AEW_E_CONFIG otherwise).
 * Decode latents to the strain field only: e_dev[nz][ny][nx] = s_b * (decoded strain
 * part) with the block's power-of-two scale from block_max_dev (device FP32
 * [nblocks][4], as written by aew_codec_encode; field 0 is used), boundary nodes 0
 * (the boundary condition of Sec. 2). */
int aew_codec_decode_e(aew_handle* h, const uint16_t* latents_dev, const float* block_max_dev,
                       float* e_dev, void* stream);

/* Time codec only (AEW_E_CONFIG otherwise).  Encode one window of nsteps (1..16)
 * strain fields e_dev[nsteps][nz][ny][nx] (device, contiguous, 16-byte aligned; the
 * window's later states are taken as 0) into latents_dev, device FP16 [nvec][n_lat]
 * (nvec = (nz/2)(ny/8)(nx/8); 32-byte aligned, AEW_E_ARG otherwise).  scale_dev (may be NULL) receives what fixes each
 * vector's scale: with AEW_NORM_POW2 device FP32 [nvec], each vector's largest |e|;
 * with AEW_NORM_MINMAX device FP64 [2][nvec], the offsets (minima) then the ranges.
 * Synchronises the stream; AEW_E_OVERFLOW if a latent overflowed FP16. */
int aew_codec_encode_window(aew_handle* h, const float* e_dev, int nsteps, uint16_t* latents_dev,
                            void* scale_dev, void* stream);

/* Time codec only.  Decode one window: e_dev[16][nz][ny][nx] (device, written, 16-byte
 * aligned) = s_v * (decoded value) (AEW_NORM_MINMAX: decoded value * range + offset)
 * with each vector's scale_dev as aew_codec_encode_window writes it, 0 on boundary
 * nodes (Sec. 2). */
int aew_codec_decode_window(aew_handle* h, const uint16_t* latents_dev, const void* scale_dev,
                            float* e_dev, void* stream);

/* ---------------------------------------------------------------------------------
 * Solves
 * ------------------------------------------------------------------------------- */

/* Synchronise `stream` and report (and clear) a timed-out device wait of any earlier
 * call of this handle: AEW_OK or AEW_E_TIMEOUT. */
int aew_sync_check(aew_handle* h, void* stream);

/* Test hook for the failure path: enqueue one kernel whose bounded wait (wait_ns,
 * 1 ns .. 1 s) runs out because nothing completes it; it sets the handle's sticky
 * error flag exactly as a timed-out stencil or codec kernel would.  Nothing faults. */
int aew_test_wait_timeout(aew_handle* h, unsigned long long wait_ns, void* stream);

/* d = F(c): forward solve from zero initial state.  c_dev [nz][ny][nx] in m/s;
 * wavelet_host: s^n for n = 0..nt-1 (NULL = the default Ricker force);
 * d_dev: [nt+1][nrec][3] (written; row 0 = B v^0 = 0). */
int aew_forward(aew_handle* h, const float* c_dev, const float* wavelet_host,
                float* d_dev, void* stream);

/* Advance a caller-owned state {e, vx, vy, vz} (device, in place) by nsteps leapfrog
 * steps starting at time index n0, with source s^n = wavelet_host[n - n0] (NULL =
 * no source) and receiver record d_dev[nsteps+1][nrec][3] (NULL = none).  The four
 * state pointers must be 16-byte aligned (AEW_E_ARG otherwise). */
int aew_propagate(aew_handle* h, const float* c_dev, float* const state_dev[4], int n0,
                  int nsteps, const float* wavelet_host, float* d_dev, void* stream);

/* Gradient of J(c) = 1/2 sum_{n=1..nt} |d^n - d_obs^n|^2 with respect to c:
 * forward solve (storing the history per the storage mode), misfit, adjoint solve
 * with FP64 time accumulation of dJ/dm, g = 2 c dJ/dm.
 * d_obs_dev [nt+1][nrec][3]; g_dev [nz][ny][nx] (written); misfit_host (may be NULL)
 * receives J (this synchronises the stream).  Keeps the forward history for later
 * aew_hessvec / aew_jvp calls at the same c. */
int aew_gradient(aew_handle* h, const float* c_dev, const float* d_obs_dev,
                 float* g_dev, double* misfit_host, void* stream);

/* Gauss-Newton Hessian-vector product at the c of the last aew_gradient:
 * hdc_dev = J_F^T J_F dc_dev (incremental forward with dm = 2 c dc, then the
 * incremental adjoint with residual B dv).  AEW_E_NOGRADIENT if no gradient ran. */
int aew_hessvec(aew_handle* h, const float* dc_dev, float* hdc_dev, void* stream);

/* Full Newton Hessian-vector product at the c of the last aew_gradient (Sec. 4's
 * incremental forward and incremental adjoint problems with the second-order terms):
 *   hdc_dev = H dc = 2 c H_m(2 c dc) + 2 dc dJ/dm,
 *   H_m dm = sum_n dt (de^n q^n + e^n dq^n),
 * de^n the incremental forward strain, q^n = G^T lam^{n+1} the first-order adjoint of
 * the last gradient's residual, dq^n the second-order adjoint: the adjoint recursion
 * driven by the residual B dv plus the source dt dm q^n in its mu update.  The
 * incremental forward keeps its strain history (FP32 with full storage; compressed by
 * the time codec into a second latent store with AE storage), then the two adjoints run
 * backward in lockstep (two adjoint steps per time step).  Needs full storage or AE
 * storage with the time codec (AEW_E_CONFIG otherwise) and a prior aew_gradient
 * (AEW_E_NOGRADIENT).  The first call allocates the extra buffers -- with full storage a
 * second nt * nx*ny*nz FP32 history, with the time codec a second latent store and two
 * decoded windows, and in both cases the second adjoint's states and accumulators --
 * and returns AEW_E_NOMEM if they do not fit.  At zero residual the result equals
 * aew_hessvec's.  With the time codec the call synchronises the stream (latent
 * overflow check). */
int aew_hessvec_full(aew_handle* h, const float* dc_dev, float* hdc_dev, void* stream);

/* Jacobian-vector product dd_dev = J_F dc_dev [nt+1][nrec][3] (incremental forward
 * alone) at the c of the last aew_gradient. */
int aew_jvp(aew_handle* h, const float* dc_dev, float* dd_dev, void* stream);

/* Algorithm 1 (data generation): run the forward solve for c_dev and pack every
 * `every`-th state n (n = every, 2*every, ... < nt) into BF16 block vectors, each
 * field of each block divided by its power-of-two scale (see aew_codec_encode).
 * With the time codec the unit is the window instead: every `every`-th complete
 * window w (w = 0, every, 2*every, ...; 16 w + 15 <= nt - 1) is packed into normalised
 * window vectors, and block_max_dev is then FP32 [max_vectors] (each vector's largest
 * |e|), or with AEW_NORM_MINMAX FP32 [max_vectors][2] (each vector's offset and range).
 * out_dev: device BF16 (uint16 bit patterns) [max_vectors][2048], 16-byte aligned
 * (AEW_E_ARG otherwise); the forward step that reads a state packs it; *n_written receives
 * the number of vectors written (whole states only, at most max_vectors).
 * block_max_dev (may be NULL): device FP32 [max_vectors][4], 16-byte aligned
 * (AEW_E_ARG otherwise), receiving the block maxima of each written vector (the forward
 * step that writes a state stores them).  The history storage of the handle is not
 * touched. */
int aew_snapshots(aew_handle* h, const float* c_dev, int every, uint16_t* out_dev,
                  long long max_vectors, float* block_max_dev, long long* n_written,
                  void* stream);

/* Train the codec (Sec. 3.3, Table 2) on n normalised vectors vectors_dev (device BF16
 * [n][2048], 16-byte aligned, as aew_snapshots writes them), entirely on the device:
 * each epoch a fresh seeded shuffle (a Feistel bijection of [0, n), cycle-walked;
 * seed and epoch as key), floor(n / batch) minibatches gathered from it, one
 * aew_codec_train_step-like LAMB step each at lr = lr0 * 0.5^(epoch / halve_every).
 * maxima_dev: the vectors' maxima from aew_snapshots (device FP32 [n][4] for the space
 * codec, [n] for the time codec), read for the amplitude-weighted losses, whose
 * weights are computed on the device (NULL allowed for AEW_LOSS_STATE / _STRAIN; with
 * AEW_NORM_MINMAX only those two are accepted).
 * epoch_loss_host (may be NULL): host FP64 [epochs], each epoch's mean minibatch loss
 * (each taken before its update).  Synchronous. */
int aew_codec_train(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                    long long n, const aew_train_cfg* cfg, double* epoch_loss_host, void* stream);

/* Decoded error of the codec on n normalised vectors (BF16 [n][2048]) with their maxima
 * (as for aew_codec_train): err_host[10] (host FP64) = rel-L2 of decode(encode(y)) - y
 * in normalised units for the fields e, vx, vy, vz and over all values, then the same
 * in physical units (x = y s; AEW_NORM_MINMAX: maxima_dev FP32 [n][2] offsets and
 * ranges, x = y r + offset); with the time codec every value is strain (err_host[0] =
 * err_host[4]).  The strain errors are also kept in aew_stats.  Synchronous. */
int aew_codec_eval(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                   long long n, double* err_host, void* stream);

/* One training step of the codec on a minibatch: batch_dev = BF16 [batch][2048]
 * normalised vectors (batch a multiple of 8); loss = mean squared reconstruction error
 * (Sec. 3.3), each squared error of vector v in field f's columns multiplied by
 * weights_dev[v][f] (device FP32 [batch][4]; NULL = all ones, the plain error of
 * Table 2); LAMB update (You et al. 2019; beta1 0.9, beta2 0.999, eps 1e-6, no weight
 * decay) of the FP32 master weights with learning rate lr.  loss_host (may be NULL)
 * receives the loss before the update (this synchronises the stream). */
int aew_codec_train_step(aew_handle* h, const uint16_t* batch_dev, const float* weights_dev,
                         int batch, float lr, float* loss_host, void* stream);

/* Initialise the codec as the optimal rank-n_lat affine code of a data set (Sec. 1: a
 * linear autoencoder learns the principal subspace of its data), written into the GELU
 * layers of Eq. (5) through GELU(a) - GELU(-a) = a: hidden units j and n_lat + j carry
 * +a_j and -a_j of a = (y - mu) V (V the n_lat leading eigenvectors of the weighted
 * covariance, mu the weighted mean), the latent is GELU(a+) - GELU(a-) = a, and the
 * decoder returns mu + z V^T the same way (needs n_hid >= 2 n_lat; further hidden units
 * get zero weights).  Training steps may refine it from there.
 * vectors_dev: device BF16 [n][2048] normalised vectors (as aew_snapshots writes them),
 * 16-byte aligned; loss: the squared error the code minimises, AEW_LOSS_STATE (every
 * vector alike) or, with the time codec, AEW_LOSS_STRAIN (the same),
 * AEW_LOSS_STRAIN_AMPLITUDE (vector v weighted by its scale s_v) or
 * AEW_LOSS_STRAIN_ENERGY (by s_v^2: the error in physical units), the weights computed
 * on the device from maxima_dev (device FP32 [n], the vectors' maxima from
 * aew_snapshots; may be NULL for the unweighted losses); eigvals_host (may be NULL):
 * host FP64 [2048] receiving the covariance's eigenvalues in descending order (the
 * tail sum past n_lat is the code's weighted mean squared error per unit weight).
 * The second moments are tcgen05 GEMMs on the device (FP64 sums); the 2048 x 2048
 * eigenproblem is solved on the host (Householder + implicit QL).  Synchronous; resets
 * the training state.  AEW_E_NOMEM if the 34 MB moment buffer and 128 MB work buffer
 * cannot be allocated. */
int aew_codec_init_pca(aew_handle* h, const uint16_t* vectors_dev, const float* maxima_dev,
                       long long n, int loss, double* eigvals_host, void* stream);

/* ---------------------------------------------------------------------------------
 * Checks and host logic
 * ------------------------------------------------------------------------------- */

/* Measurement hook: nsteps launches of one kernel of the hot path, back to back on the
 * handle's own buffers (whatever they hold; the work does not depend on the values),
 * with m = c_dev^2 (device [nz][ny][nx]), timed with CUDA events on `stream`; *ms_host
 * receives the mean device time per launch.  kind: 0 forward step, 1 forward step that
 * also packs its output strain into a time-codec window, 2 adjoint step reading a
 * strain field (with the FP64 flush every accum_window steps), 3 incremental forward
 * step, 4 encoder of one window (both layers), 5 decoder of one window (both layers,
 * scattered to 16 FP32 strain slices), 6 adjoint step reading its strain field as BF16
 * (as the time codec's adjoint sweeps do; nx a multiple of 8), 7 decoder of one window
 * into BF16 strain slices, 8 incremental forward step reading its strain field as BF16,
 * 9 the space codec's fused strain decoder of one state (both layers, scattered to the
 * grid).  Kinds 1, 4, 5 and 7 need AE storage with the time codec, 9 with the space codec
 * (AEW_E_CONFIG otherwise), 4, 5, 7 and 9 codec weights.  Overwrites the handle's stored
 * history (a later aew_hessvec needs a new aew_gradient).  Synchronises the stream. */
int aew_profile_steps(aew_handle* h, const float* c_dev, int kind, int nsteps, double* ms_host,
                      void* stream);

/* Host only (no device work): all eigenpairs of the symmetric n x n FP64 matrix A_host
 * (row-major), the solver aew_codec_init_pca uses: eigenvalues w_host[n] in descending
 * order, eigenvectors as the columns of V_host (row-major n x n).  AEW_E_ARG for bad
 * arguments or if the QL iteration does not converge. */
int aew_sym_eig(int n, const double* A_host, double* w_host, double* V_host);

/* FP64 inner product sum a[i] b[i] of two device FP32 arrays of n elements
 * (for the adjoint-identity and finite-difference checks).  Synchronises `stream`. */
int aew_dot(const float* a_dev, const float* b_dev, size_t n, double* out_host, void* stream);

/* Test hook for the codec's activation (Sec. 3.3 layers; GELU, reading R5):
 * y_dev[i] = GELU(x_dev[i]) = x Phi(x) as the encoder and decoder kernels evaluate it
 * (Phi through Abramowitz & Stegun eq. 7.1.28, |error| <= 3e-7, within 1e-6 in FP32; two
 * values at a time on paired FP32 lanes, x_dev[2k] and x_dev[2k+1] together; NaN where
 * that differs in any bit from the same operations on one value),
 * dy_dev[i] = GELU'(x_dev[i]) = Phi(x) + x phi(x) as the training kernels evaluate it
 * (erff).  Device FP32 arrays of n elements, caller-owned;
 * asynchronous on `stream`.  AEW_E_ARG for n < 0 or NULL pointers with n > 0, AEW_E_CUDA
 * if the launch fails. */
int aew_test_gelu(const float* x_dev, float* y_dev, float* dy_dev, long long n, void* stream);

/* aew_dot without any device allocation, for callers that cannot allocate device
 * memory (an application whose allocations all go through its own pool, or a hook that
 * must not change the device memory footprint).  No counterpart in the paper: it is a
 * service variant of aew_dot.  The per-block partial sums live in a fixed array in
 * device memory inside the library (512 KiB per GPU, held until the process exits);
 * n must be at most 2^32 (AEW_E_ARG otherwise, before any device work).
 * out_dev: device FP64 scalar receiving sum a[i] b[i] (written on `stream`; the call
 * does not synchronise).  The first call on a device looks up the array's device
 * address (again after the device's context is created anew, e.g. by cudaDeviceReset),
 * so it must not be made during stream capture.  All calls share the array:
 * calls that overlap on the GPU race and must be serialised by the caller.  Returns
 * AEW_E_ARG for NULL pointers, AEW_E_CUDA if a launch fails. */
int aew_dot_noalloc(const float* a_dev, const float* b_dev, size_t n, double* out_dev,
                    void* stream);

/* The binomial checkpointing plan the library runs for nt steps with s state slots
 * (host only, no device work).  ops/args (host, capacity `cap`) receive the actions:
 * op 0 = advance args steps, 1 = store in slot args, 2 = restore slot args (-1 = the
 * zero initial state), 3 = final step nt-1 -> nt (its receiver record only; the live
 * state stays nt-1), 4 = adjoint step args.  *n_ops = number of actions (also when
 * it exceeds cap, in which case nothing beyond cap is written); *fwd_steps = forward
 * steps of the plan. */
int aew_revolve_plan(int nt, int s, int* ops, int* args, long long cap,
                     long long* n_ops, long long* fwd_steps);

/* ---------------------------------------------------------------------------------
 * MAP estimation with the BiLaplacian prior, and DIAS (Sec. 2, Sec. 4.3)
 *
 * Prior (Sec. 2): the elliptic operator of the prior PDE with an isotropic Theta =
 * theta I, discretised on the nodes with zero-flux boundaries,
 *     A q = alpha (q - theta Lap_N q),
 *     (Lap_N q)_i = sum over the grid neighbours nb that node i has of (q_nb - q_i) / h^2,
 * symmetric positive definite, and the prior precision is its square: the
 * regularisation is R(c) = 1/2 |A (c - c0)|^2.  With the projection P = I - W1^T W1
 * onto the inactive subspace (rows of W1 orthonormal) it is the DIAS-F form
 * 1/2 |A P (c - c0)|^2, precision P A^2 P (Sec. 4.3, the approximation of the
 * pseudo-inverse by the projected inverse covariance).
 * --------------------------------------------------------------------------------- */
typedef struct aew_newton_cfg {
  double alpha;         /* prior weight alpha (> 0) */
  double theta;         /* prior length scale theta [m^2] (>= 0) */
  int newton_iters;     /* Newton iterations (>= 1) */
  int cg_max;           /* CG iterations per Newton step (>= 1) */
  int full_hessian;     /* 0: Gauss-Newton misfit Hessian (aew_hessvec); 1: full
                           (aew_hessvec_full, which needs full or time-codec storage) */
  double c1;            /* Armijo constant (typically 1e-4) */
  int max_backtracks;   /* step halvings tried (>= 1) */
  double eta_max;       /* cap of the CG forcing term (typically 0.5) */
  double gtol;          /* stop once |g| <= gtol |g_0| (0: run every iteration) */
} aew_newton_cfg;

/* One Newton iteration, at the iterate it starts from. */
typedef struct aew_newton_iter {
  double cost;          /* misfit + regularisation */
  double misfit;
  double reg;
  double gnorm;         /* |g|, g = misfit gradient + regularisation gradient */
  int cg_iters;         /* CG iterations taken (0 if the first direction had d^T H d <= 0:
                           the step is then along -g) */
  int backtracks;       /* step halvings before the Armijo condition held */
  double step;          /* step length taken */
} aew_newton_iter;

/* out_dev = A q_dev (FP32; [nz][ny][nx] of the handle's grid and spacing).
 * Asynchronous on `stream`.  AEW_E_ARG for NULL pointers, alpha <= 0 or theta < 0.
 * q_dev and out_dev must not overlap.  The vectors of aew_prior_apply, aew_prior_solve,
 * aew_newton_cg and aew_dias_subspace are read as float4: they must be 16-byte aligned
 * (AEW_E_ARG otherwise; a torch allocation is). */
int aew_prior_apply(aew_handle* h, double alpha, double theta, const float* q_dev,
                    float* out_dev, void* stream);

/* x_dev = A^{-1} w_dev by conjugate gradients on FP32 vectors with FP64 inner products
 * (A is SPD with spectrum inside [alpha, alpha (1 + 12 theta / h^2)]), stopped when the
 * recursive residual |r| <= rtol |w| (tolerances down to about 1e-7 are reached) or
 * after max_iter iterations; *iters_host (may be NULL) receives the iterations taken.
 * Prior samples are c + A^{-1} w for white noise w.  Synchronises `stream` (the
 * convergence test reads the residual every 8 iterations).  AEW_E_ARG for bad
 * arguments; AEW_E_NOMEM if the three FP32 work vectors cannot be allocated (they are
 * freed on return); AEW_E_NOCONVERGE if the residual test did not pass within max_iter
 * (x_dev then holds the last iterate). */
int aew_prior_solve(aew_handle* h, double alpha, double theta, const float* w_dev,
                    float* x_dev, double rtol, int max_iter, int* iters_host, void* stream);

/* Inexact Newton-CG for the MAP point (Sec. 2, Sec. 4.3):
 *   minimise J(c) = 1/2 sum_n |d^n(c) - d_obs^n|^2 + R(c),
 * R as above (projected by W1 when W1_dev is not NULL: the DIAS-F problem).  Iteration
 * k: the gradient g = g_misfit + dR/dc at c_k; CG from 0 on H p = -g with
 * H v = H_misfit v + (P) A^2 (P) v, H_misfit the Gauss-Newton (aew_hessvec) or full
 * (aew_hessvec_full) Hessian of the misfit at c_k, stopped at |r| <= eta |g| with
 * eta = min(eta_max, sqrt(|g| / |g_0|)) (Eisenstat-Walker), after cg_max iterations,
 * or at a direction with d^T H d <= 0; then Armijo backtracking (step 1, halved up to
 * max_backtracks times, J(c + s p) <= J(c) + c1 s g^T p).  Each trial point runs the
 * gradient solve, whose adjoint half is skipped when the trial's misfit already fails
 * the Armijo test -- so an accepted trial already holds the next iterate's gradient
 * and history (with revolve storage the adjoint always runs).  A trial outside the
 * stability bound (max c dt / h > 1/sqrt(3)) or with c <= 0 fails the test.  If no
 * trial passes, c stays, the iteration is recorded with step 0 and the call returns.
 *   c_dev        in: the initial iterate; out: the final one [nz][ny][nx]
 *   d_obs_dev    [nt+1][nrec][3]
 *   c0_dev       prior mean [nz][ny][nx]
 *   W1_dev, r    NULL/0, or r orthonormal rows [r][nz*ny*nx] spanning the active subspace
 *   hist_host    newton_iters entries (may be NULL); *iters_host (may be NULL) receives
 *                the iterations recorded (fewer than newton_iters when gtol stopped it)
 * Allocates nine FP32 work vectors for the call and frees them on return.  Returns the
 * errors of aew_gradient / aew_hessvec(_full) (AEW_E_CFL if the initial c leaves the
 * stability bound), AEW_E_ARG for bad arguments, AEW_E_NOMEM. */
int aew_newton_cg(aew_handle* h, float* c_dev, const float* d_obs_dev, const float* c0_dev,
                  const aew_newton_cfg* cfg, const float* W1_dev, int r,
                  aew_newton_iter* hist_host, int* iters_host, void* stream);

/* DIAS active subspace (Sec. 4.3), centred at c_dev (the two-step algorithm centres it
 * at the MAP point): for each of the N white-noise fields w_i (noise_dev [N][nz*ny*nx],
 * caller-drawn), the prior sample c_i = c + A^{-1} w_i (aew_prior_solve, rtol 1e-10),
 * the misfit gradient g_i at c_i (aew_gradient) into G_dev[i], then the eigenpairs of
 * C = (1/N) sum_i g_i g_i^T through the N x N Gram matrix M = G G^T / N (FP64 sums of
 * FP32 products over 64-node tiles): C's leading eigenvectors are
 * W1_k = G^T u_k / sqrt(N lambda_k) for M's eigenpairs (lambda_k, u_k).
 *   G_dev       [N][nz*ny*nx] workspace, receives the sample gradients
 *   W1_dev      [r][nz*ny*nx] receives the r leading eigenvectors (orthonormal rows)
 *   lambda_host [N] receives all eigenvalues of M (= the nonzero ones of C), descending
 * 1 <= r <= N <= 64, r <= 32.  Synchronises `stream`.  Errors of aew_prior_solve and
 * aew_gradient (AEW_E_CFL if a sample leaves the stability bound); AEW_E_ARG if fewer
 * than r eigenvalues are positive. */
int aew_dias_subspace(aew_handle* h, const float* c_dev, const float* d_obs_dev,
                      const float* noise_dev, int N, double alpha, double theta, int r,
                      float* G_dev, float* W1_dev, double* lambda_host, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* AEWAVE_H */
