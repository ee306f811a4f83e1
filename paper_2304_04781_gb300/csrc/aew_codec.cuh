// Internal interface of the codec (per-block autoencoder) and its training kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

namespace aew {

struct Codec;

constexpr int kNIn = 2048;   // 8x8x8 nodes x 4 fields
constexpr int kNHid = 512;

Codec* codec_new(int n_lat);
void codec_free(Codec* c);
int codec_nlat(const Codec* c);
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

// One training step (MSE + LAMB); loss (device float) written if loss_dev != null.
// weights: FP32 [B][4] per vector and field (null: the plain mean squared error)
cudaError_t codec_train_step(Codec* c, const uint16_t* batch, const float* weights, int B,
                             float lr, float* loss_dev, cudaStream_t s, std::string* err);

}  // namespace aew
