// Internal interface of the codec (per-block autoencoder) and its training kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

namespace aew {

struct Codec;

constexpr int kNIn = 2048;   // 8x8x8 nodes x 4 fields, or 2x8x8 nodes x 16 steps
constexpr int kNHid = 512;   // hidden width of the space codec
constexpr int kTSteps = 16;  // steps per window of the time codec

// space codec: n_hid = 512, n_lat 32 or 64; time codec: n_hid = 2 n_lat, n_lat 256 or 512
Codec* codec_new(int n_lat, bool time);
// time codec: normalisation (0 power of two, 1 min-max with floor beta), activation
// (0 GELU, 1 ELU)
void codec_set_variant(Codec* c, int norm, int act, double beta);
bool codec_minmax(const Codec* c);
double codec_beta(const Codec* c);
void codec_free(Codec* c);
int codec_nlat(const Codec* c);
int codec_nhid(const Codec* c);
// drop the optimiser state (LAMB moments, step count): training starts afresh
void codec_reset_training(Codec* c);
size_t codec_device_bytes(const Codec* c);
bool codec_ready(const Codec* c);

// w[8] = W1, b1, W2, b2, W3, b3, W4, b4 (host FP32, row-major, layer y -> y W + b)
cudaError_t codec_set_weights(Codec* c, const float* const w[8]);
// y = GELU(x) as the inference epilogues evaluate it, dy = GELU'(x) as the training
// kernels evaluate it (test hook)
cudaError_t launch_activation_probe(const float* x, float* y, float* dy, long long n,
                                    cudaStream_t s);
cudaError_t codec_get_weights(const Codec* c, float* const w[8]);

// Rebuild the tensor-core operand copies of the weights from the FP32 masters.
cudaError_t codec_refresh(Codec* c, cudaStream_t s);

// Encode one grid state: BF16 block vectors plus per-block, per-field maxima of |f|
// (bmax, float bits [nblocks][4], written), normalised by the power-of-two block scales,
// then the encoder.  latents FP16 [nblocks][n_lat].
cudaError_t codec_encode_grid(Codec* c, const float* const f[4], int nx, int ny, int nz,
                              unsigned* bmax, uint16_t* lat, int* overflow, cudaStream_t s);

// Encode already normalised BF16 block vectors [n][2048] into FP16 latents [n][n_lat].
// ctas > 0 caps the GEMMs' persistent CTAs (room for a concurrent stencil step)
cudaError_t codec_encode_vectors(Codec* c, const uint16_t* vec, long long n, uint16_t* lat,
                                 int* overflow, cudaStream_t s, int ctas = 0);

// Decode the strain part of latents into the grid: e = s_b * dec_e(z) with the block's
// power-of-two scale s_b from bmax[b][0]; 0 on boundary nodes.
cudaError_t codec_decode_grid_e(Codec* c, const uint16_t* lat, int nx, int ny, int nz,
                                const unsigned* bmax, float* e_out, cudaStream_t s,
                                int ctas = 0);

// Decode latents to normalised vectors FP32 [nvec][2048].
cudaError_t codec_decode_vectors(Codec* c, const uint16_t* lat, long long nvec, float* out,
                                 cudaStream_t s);

// ---- compression in time (16-step strain windows of 2 x 8 x 8-node blocks) ----
// Encode one window: raw BF16 strain vectors [nvec][2048] (as the forward step packs
// them) and each vector's max |e| (vmax, float bits [nvec]); the layer-1 epilogue
// divides by the vector's power-of-two scale.  latents FP16 [nvec][n_lat].
// With min-max normalisation (codec_minmax) the window is normalised in place first and
// each vector's offset and range are written to mn / rr (FP64 [nvec]; vmax unused).
cudaError_t codec_encode_window(Codec* c, uint16_t* raw, const unsigned* vmax,
                                long long nvec, uint16_t* lat, int* overflow, cudaStream_t s,
                                int ctas = 0, double* mn = nullptr, double* rr = nullptr);
// Decode one window into 16 strain slices e_out[t][nz][ny][nx] (slice stride nx ny nz):
// e = s_v * decoded value (min-max: decoded value * rr + mn), 0 on boundary nodes.
// bf16_out: the slices as BF16 instead ([16][nz][ny][nx] uint16 from e_out), for the
// adjoint-type sweeps.
cudaError_t codec_decode_window(Codec* c, const uint16_t* lat, const unsigned* vmax, int nx,
                                int ny, int nz, float* e_out, cudaStream_t s, int ctas = 0,
                                const double* mn = nullptr, const double* rr = nullptr,
                                bool bf16_out = false);
// The paper's min-max normalisation of raw BF16 window vectors (in place allowed):
// y = (x - min) / r, r = max(max - min, beta); offsets and ranges to mn / rr (FP64).
cudaError_t window_minmax(const uint16_t* raw, long long nvec, double beta, uint16_t* out,
                          double* mn, double* rr, cudaStream_t s, float* pair32 = nullptr);
// Pack nsteps (<= 16) strain fields e[t][nz][ny][nx] into raw BF16 window vectors
// [nvec][2048] (missing steps 0) and fold max |e| per vector into vmax (zeroed here).
cudaError_t window_pack(const float* e, int nsteps, int nx, int ny, int nz, uint16_t* raw,
                        unsigned* vmax, cudaStream_t s);
// Weighted moments of n normalised BF16 vectors Y [n][2048] for the PCA initialisation:
// G64 [2048][2048] = sum_v w_v y_v y_v^T (tcgen05 GEMMs of transposed, sqrt(w)-scaled
// chunks of the vectors, FP32 within a chunk, summed in FP64 across chunks) and
// s64 [2049] = (sum_v w_v y_v, sum_v w_v) (deterministic FP64 sums); w null = all 1.
// Work buffers are allocated and freed inside.
cudaError_t codec_moments(Codec* c, const uint16_t* Y, long long n, const float* w, double* G64,
                          double* s64, cudaStream_t s);
// w[v] = s_v^pw (pw 1 or 2) with s_v the power-of-two scale of the vector maximum mx[v]
cudaError_t vector_weights(const float* mx, long long n, int pw, float* w, cudaStream_t s);
// out = bf16(raw / s_v) per vector (in place allowed): Algorithm 1's normalised vectors.
cudaError_t window_normalise(const uint16_t* raw, const unsigned* vmax, long long nvec,
                             uint16_t* out, cudaStream_t s);

// Algorithm 1 packing of one grid state: normalised BF16 block vectors [nblocks][2048]
// (each block-field divided by its power-of-two scale) and the block maxima (bmax,
// float bits [nblocks][4], written; work buffer X [nblocks][2048] for the raw values).
cudaError_t snapshot_pack(const float* const f[4], int nx, int ny, int nz, unsigned* bmax,
                          uint16_t* raw, uint16_t* out, cudaStream_t s);

// Device error flag of the codec kernels (set by a bounded wait that gave up); read and
// clear it (synchronises the stream).  Returns true if it was set.
bool codec_take_error(Codec* c, cudaStream_t s);
// the device error flag the codec kernels and the stencil steps set on a timed-out wait
int* codec_err_flag(Codec* c);

// One training step (MSE + LAMB); loss (device float) written if loss_dev != null and
// added to *loss_acc (device double) if loss_acc != null.
// weights: FP32 [B][4] per vector and field (null: the plain mean squared error)
cudaError_t codec_train_step(Codec* c, const uint16_t* batch, const float* weights, int B,
                             float lr, float* loss_dev, cudaStream_t s, std::string* err,
                             double* loss_acc = nullptr);

// Training epochs (Table 2): per epoch a seeded shuffle of the n vectors, minibatches
// gathered on the device, learning rate lr0 * 0.5^(epoch / halve_every), loss weights
// from the vectors' maxima.  epoch_loss (host, may be null): mean loss of each epoch.
enum { kLossState = 0, kLossStrain = 1, kLossStrainAmplitude = 2, kLossStrainEnergy = 3 };
struct TrainCfg {
  int epochs, batch, halve_every, loss;
  double lr0;
  uint64_t seed;
};
cudaError_t codec_train(Codec* c, const uint16_t* Y, const float* maxima, long long n,
                        const TrainCfg& cfg, double* epoch_loss, cudaStream_t s,
                        std::string* err);

// Decoded error of n normalised vectors: out[0..4] rel-L2 of decode(encode(y)) - y in
// normalised units per field (e, vx, vy, vz) and overall, out[5..9] the same in physical
// units (x = y s with the vectors' scales from their maxima; time codec: every column is
// strain, out[0] = out[4]).  maxima: [n][4] block maxima or [n] vector maxima; with
// min-max normalisation [n][2] (offset, range), x = y r + offset.
cudaError_t codec_eval(Codec* c, const uint16_t* Y, const float* maxima, long long n,
                       double* out, cudaStream_t s);

}  // namespace aew
