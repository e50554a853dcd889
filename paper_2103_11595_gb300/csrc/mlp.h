// The learned merge scorer: a small MLP over features of a candidate pairwise merge.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ajf {

constexpr int kMlpFeatures = 16;
constexpr int kMlpHidden1 = 224;
constexpr int kMlpHidden2 = 192;
constexpr int kMlpParams = kMlpHidden1 * kMlpFeatures + kMlpHidden1 + kMlpHidden2 * kMlpHidden1 + kMlpHidden2 +
                           kMlpHidden2 + 1;  // 47,201

// Glorot-uniform initial weights from a seed (biases zero).
void mlp_init(float* w, uint64_t seed);

// Score of one feature vector on the host (same arithmetic as the device forward pass, FP32).
float mlp_score_host(const float* w, const float* x);

// Batched scoring on the current CUDA device (hand-written forward kernels). The object keeps a
// device buffer between calls and uploads the weights again only when their host address changes.
class MlpScorer {
 public:
  ~MlpScorer();
  cudaError_t score(const float* weights_host, const float* x, int n, float* out);
  void release();

 private:
  float* dev_ = nullptr;
  size_t cap_ = 0;
  const float* loaded_ = nullptr;
};

// Train from scratch on `n_pairs` ranking examples (each 2 x kMlpFeatures floats: the chosen merge,
// then another candidate of the same planner state): minibatches of `batch` pairs, Adam with
// learning rate lr, `epochs` passes. Writes kMlpParams weights and the last epoch's mean loss.
cudaError_t mlp_train(const float* pairs, int n_pairs, int epochs, int batch, float lr, uint64_t seed, float* weights,
                      double* final_loss);

}  // namespace ajf
