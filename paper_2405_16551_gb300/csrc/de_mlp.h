// de_mlp.h -- device state and launchers of the surrogate network (de_mlp.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace de {

constexpr int kMlpIn = 20;      // parameters of the objective
constexpr int kMlpH = 256;      // hidden units per layer
constexpr int kMlpBatch = 256;  // minibatch rows of one training step (two 128-row halves)
constexpr int kMlpPart = 260;   // per-half partial sums: dw3 (256), db3, loss
// FP32 parameter vector: W1 (256 x 20), b1, W2 (256 x 256), b2, w3, b3
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpH * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpH;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpH * kMlpH;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpH;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpH;
constexpr int kMlpParams = kMlpOffB3 + 1;  // 71,425
// BF16 operand copies (canonical K-major tiles)
constexpr uint32_t kMlpW1Bytes = kMlpH * 32 * 2;       // W1 with b1 in column 20: 256 x 32
constexpr uint32_t kMlpW2Bytes = kMlpH * kMlpH * 2;    // 256 x 256
constexpr uint32_t kMlpA1tBytes = 32 * kMlpBatch * 2;  // inputs, transposed: 32 x 256

struct MlpDev {
  float *W1, *b1, *W2, *b2, *w3, *b3;        // FP32 masters (views into one vector)
  float *mW1, *mb1, *mW2, *mb2, *mw3, *mb3;  // Adam first moments
  float *vW1, *vb1, *vW2, *vb2, *vw3, *vb3;  // Adam second moments
  uint8_t *w1k, *w2k, *w2t;                  // BF16 operands: W1|b1 (256 x 32), W2 (256 x 256), W2^T (2 x 128 x 256)
  uint8_t *h1t, *dz2t, *dz1t, *a1t;          // transposed activations of one minibatch
  float* part;                               // 2 x kMlpPart partial sums
  float* grad;                               // kMlpParams raw gradients (gradient-only steps)
  float* loss;                               // loss of the last step
  int* err;                                  // device error bits (a bounded wait gave up)
};

struct MlpStepArgs {
  uint64_t seed;     // Philox key of the minibatch draws
  long long step;    // training steps taken before this one (counter of the draws, Adam's t - 1)
  int sample_n;      // rows to draw from (0: take rows 0..255 in order)
  int sample_base;   // first row of the window in a ring of sample_cap rows
  int sample_cap;
};

void set_last_error(const std::string& m);  // de_api.cu
void mlp_configure();
void mlp_pack_launch(const MlpDev& P, cudaStream_t s);
void mlp_forward_launch(const MlpDev& P, const double* x, int64_t ld, int n, float* y, cudaStream_t s);
void mlp_step_launch(const MlpDev& P, const MlpStepArgs& a, const double* x, int64_t ld, const float* t, float lr,
                     bool apply, cudaStream_t s);

}  // namespace de
