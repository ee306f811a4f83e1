// Definition of the codec state shared by the codec and training translation units.
#pragma once

#include <cstddef>
#include <cstdint>

namespace aew {

struct Codec {
  int n_lat = 64;
  int n_hid = 512;           // hidden width: 512 (space codec) or 2 n_lat (time codec)
  bool time = false;         // compression in time (16-step strain windows)
  // time codec only: normalisation (0: power-of-two scale, 1: the paper's min-max to
  // [0, 1] with the range floored at beta) and hidden activation (0: GELU, 1: ELU)
  int norm = 0;
  int act = 0;
  double beta = 1e-7;
  bool ready = false;
  // FP32 master weights: W1 [2048][nh], b1, W2 [nh][nl], b2, W3 [nl][nh], b3,
  // W4 [nh][2048], b4
  float* w[8] = {};
  size_t wn[8] = {};
  // operand copies (K-major rows): W1t [nh][2048] bf16, W2t [nl][nh] bf16,
  // W3t [nh][nl] fp16, W4t [2048][nh] bf16
  uint16_t* W1t = nullptr;
  uint16_t* W2t = nullptr;
  uint16_t* W3t = nullptr;
  uint16_t* W4t = nullptr;
  uint16_t* W4e = nullptr;   // space codec: the 512 strain rows of W4t, [512][512]
  // workspace: hidden activations H [rows][nh] bf16, packed inputs X [rows][2048] bf16
  uint16_t* H = nullptr;
  size_t H_rows = 0;
  uint16_t* X = nullptr;
  size_t X_rows = 0;
  float* sc_tmp = nullptr;
  int* err = nullptr;
  int max_ctas = 0;          // CTA cap of the codec GEMMs (0: one per SM)
  int max_stages = 0;        // stage cap of the codec GEMMs (0: as many as fit)
  bool pair_gemm = true;     // encoder layer 1 on SM pairs (cta_group::2)
  size_t bytes = 0;
  // training state (allocated by the training unit)
  void* train = nullptr;
};

void train_state_free(void* t);
size_t train_state_bytes(const void* t);

}  // namespace aew
