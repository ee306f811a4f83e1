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
cudaError_t codec_get_weights(const Codec* c, float* const w[8]);

// Rebuild the tensor-core operand copies of the weights from the FP32 masters.
cudaError_t codec_refresh(Codec* c, cudaStream_t s);

// Encode one grid state.  s_f = max(scale_prev[f], amax[f]) (either may be null: 0),
// written to scale_out[f] (may be null).  latents FP16 [nblocks][n_lat].
cudaError_t codec_encode_grid(Codec* c, const float* const f[4], int nx, int ny, int nz,
                              const float* scale_prev, const unsigned* amax, float* scale_out,
                              uint16_t* lat, int* overflow, cudaStream_t s);

// Encode BF16 block vectors [n][2048] into FP16 latents [n][n_lat].
cudaError_t codec_encode_vectors(Codec* c, const uint16_t* vec, long long n, uint16_t* lat,
                                 int* overflow, cudaStream_t s);

// Decode the strain part of latents into the grid: e = s_e * dec_e(z), 0 on boundary.
cudaError_t codec_decode_grid_e(Codec* c, const uint16_t* lat, int nx, int ny, int nz,
                                const float* scale_e, float* e_out, cudaStream_t s);

// Decode latents to normalised vectors FP32 [nvec][2048].
cudaError_t codec_decode_vectors(Codec* c, const uint16_t* lat, long long nvec, float* out,
                                 cudaStream_t s);

// Algorithm 1 packing: normalised BF16 block vectors of one grid state.
cudaError_t snapshot_pack(const float* const f[4], int nx, int ny, int nz, const float* scale,
                          uint16_t* out, cudaStream_t s);

// One training step (MSE + LAMB); loss (device float) written if loss_dev != null.
cudaError_t codec_train_step(Codec* c, const uint16_t* batch, int B, float lr, float* loss_dev,
                             cudaStream_t s, std::string* err);

}  // namespace aew
