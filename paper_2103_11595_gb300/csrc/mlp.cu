// The learned merge scorer's MLP: inference and training kernels (sm_103a).
//
// score(x) = w3 . relu(W2 relu(W1 x + b1) + b2) + b3, x = 16 features of a candidate pairwise merge
// (planner_learned.cpp). Parameters (float32, in this order): W1[H1][F], b1[H1], W2[H2][H1],
// b2[H2], w3[H2], b3 -- 16*224 + 224 + 224*192 + 192 + 192 + 1 = 47,201 values.
//
// Training is pairwise ranking: for a planner state, the merge the reference path took (x_c) and
// another candidate (x_o) give the loss softplus(score(x_o) - score(x_c)). The kernels below run
// the forward pass for a batch, the backward pass (gradients accumulated over the batch) and Adam.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "mlp.h"

namespace ajf {
namespace {

constexpr int F = kMlpFeatures, H1 = kMlpHidden1, H2 = kMlpHidden2;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H1 * F, OFF_W2 = OFF_B1 + H1, OFF_B2 = OFF_W2 + H2 * H1,
              OFF_W3 = OFF_B2 + H2, OFF_B3 = OFF_W3 + H2;

// y[b][o] = act(sum_i W[o][i] x[b][i] + bias[o]); one thread per (b, o).
__global__ void k_dense(const float* __restrict__ x, const float* __restrict__ W, const float* __restrict__ bias,
                        float* __restrict__ y, int B, int I, int O, int relu) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(B) * O) return;
  const int b = static_cast<int>(t / O), o = static_cast<int>(t % O);
  const float* xr = x + int64_t(b) * I;
  const float* wr = W + int64_t(o) * I;
  float s = bias[o];
  for (int i = 0; i < I; ++i) s += wr[i] * xr[i];
  y[t] = relu ? fmaxf(s, 0.0f) : s;
}

// score[b] = w3 . h2[b] + b3 (one warp per example)
__global__ void k_head(const float* __restrict__ h2, const float* __restrict__ w3, const float* __restrict__ b3,
                       float* __restrict__ score, int B) {
  const int b = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
  if (b >= B) return;
  float s = 0;
  for (int j = lane; j < H2; j += 32) s += w3[j] * h2[int64_t(b) * H2 + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) score[b] = s + b3[0];
}

// Ranking loss over pairs: rows [0, P) of the batch are chosen merges, rows [P, 2P) the others.
// dscore = d/ds softplus(s_o - s_c); loss accumulated (for reporting).
__global__ void k_rank_loss(const float* __restrict__ score, float* __restrict__ dscore, float* __restrict__ loss,
                            int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float z = score[P + i] - score[i];
  const float sg = 1.0f / (1.0f + expf(-z));
  dscore[i] = -sg / P;
  dscore[P + i] = sg / P;
  const float l = z > 20.f ? z : log1pf(expf(z));
  atomicAdd(loss, l / P);
}

// dh[b][j] = (sum_o dy[b][o] W[o][j]) * [h[b][j] > 0]   (W is [O][J])
__global__ void k_back_hidden(const float* __restrict__ dy, const float* __restrict__ W, const float* __restrict__ h,
                              float* __restrict__ dh, int B, int O, int J) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(B) * J) return;
  const int b = static_cast<int>(t / J), j = static_cast<int>(t % J);
  if (h[t] <= 0.0f) {
    dh[t] = 0.0f;
    return;
  }
  float s = 0;
  for (int o = 0; o < O; ++o) s += dy[int64_t(b) * O + o] * W[int64_t(o) * J + j];
  dh[t] = s;
}

// dh2[b][j] = dscore[b] * w3[j] * [h2 > 0]
__global__ void k_back_head(const float* __restrict__ dscore, const float* __restrict__ w3, const float* __restrict__ h2,
                            float* __restrict__ dh2, int B) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= int64_t(B) * H2) return;
  const int b = static_cast<int>(t / H2), j = static_cast<int>(t % H2);
  dh2[t] = h2[t] > 0.0f ? dscore[b] * w3[j] : 0.0f;
}

// gW[o][i] = sum_b dy[b][o] x[b][i]; gb[o] = sum_b dy[b][o]   (one thread per weight)
__global__ void k_grad_dense(const float* __restrict__ dy, const float* __restrict__ x, float* __restrict__ gW,
                             float* __restrict__ gb, int B, int I, int O) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= O * (I + 1)) return;
  const int o = t / (I + 1), i = t % (I + 1);
  float s = 0;
  if (i < I) {
    for (int b = 0; b < B; ++b) s += dy[int64_t(b) * O + o] * x[int64_t(b) * I + i];
    gW[int64_t(o) * I + i] = s;
  } else {
    for (int b = 0; b < B; ++b) s += dy[int64_t(b) * O + o];
    gb[o] = s;
  }
}

// gw3[j] = sum_b dscore[b] h2[b][j]; gb3 = sum_b dscore[b]
__global__ void k_grad_head(const float* __restrict__ dscore, const float* __restrict__ h2, float* __restrict__ gw3,
                            float* __restrict__ gb3, int B) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > H2) return;
  float s = 0;
  if (j < H2) {
    for (int b = 0; b < B; ++b) s += dscore[b] * h2[int64_t(b) * H2 + j];
    gw3[j] = s;
  } else {
    for (int b = 0; b < B; ++b) s += dscore[b];
    gb3[0] = s;
  }
}

// Batch rows: x[i] = chosen features of pair perm[b0 + i], x[P + i] = the other candidate's.
__global__ void k_gather_pairs(const float* __restrict__ data, const int* __restrict__ perm, int b0, int P,
                               float* __restrict__ x) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * P * F) return;
  const int row = t / F, f = t % F;
  const int i = row < P ? row : row - P;
  const float* src = data + size_t(perm[b0 + i]) * 2 * F + (row < P ? 0 : F);
  x[t] = src[f];
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float b1t, float b2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  m[i] = b1 * m[i] + (1 - b1) * gi;
  v[i] = b2 * v[i] + (1 - b2) * gi * gi;
  const float mh = m[i] / (1 - b1t), vh = v[i] / (1 - b2t);
  w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

unsigned blocks(int64_t n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

void forward(const float* w, const float* x, float* h1, float* h2, float* score, int B, cudaStream_t s) {
  k_dense<<<blocks(int64_t(B) * H1, 256), 256, 0, s>>>(x, w + OFF_W1, w + OFF_B1, h1, B, F, H1, 1);
  k_dense<<<blocks(int64_t(B) * H2, 256), 256, 0, s>>>(h1, w + OFF_W2, w + OFF_B2, h2, B, H1, H2, 1);
  k_head<<<blocks(B, 8), 256, 0, s>>>(h2, w + OFF_W3, w + OFF_B3, score, B);
}

}  // namespace

void mlp_init(float* w, uint64_t seed) {
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
  auto uni = [&]() {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return (static_cast<double>(st >> 11) / 9007199254740992.0) * 2.0 - 1.0;
  };
  std::memset(w, 0, sizeof(float) * kMlpParams);
  const double s1 = std::sqrt(6.0 / (F + H1)), s2 = std::sqrt(6.0 / (H1 + H2)), s3 = std::sqrt(6.0 / (H2 + 1));
  for (int i = 0; i < H1 * F; ++i) w[OFF_W1 + i] = static_cast<float>(s1 * uni());
  for (int i = 0; i < H2 * H1; ++i) w[OFF_W2 + i] = static_cast<float>(s2 * uni());
  for (int i = 0; i < H2; ++i) w[OFF_W3 + i] = static_cast<float>(s3 * uni());
}

float mlp_score_host(const float* w, const float* x) {
  float h1[H1], h2[H2];
  for (int o = 0; o < H1; ++o) {
    float s = w[OFF_B1 + o];
    for (int i = 0; i < F; ++i) s += w[OFF_W1 + o * F + i] * x[i];
    h1[o] = s > 0 ? s : 0;
  }
  for (int o = 0; o < H2; ++o) {
    float s = w[OFF_B2 + o];
    for (int i = 0; i < H1; ++i) s += w[OFF_W2 + o * H1 + i] * h1[i];
    h2[o] = s > 0 ? s : 0;
  }
  float s = w[OFF_B3];
  for (int j = 0; j < H2; ++j) s += w[OFF_W3 + j] * h2[j];
  return s;
}

MlpScorer::~MlpScorer() { release(); }

void MlpScorer::release() {
  if (dev_) cudaFree(dev_);
  dev_ = nullptr;
  cap_ = 0;
}

cudaError_t MlpScorer::score(const float* weights_host, const float* x, int n, float* out) {
  if (n <= 0) return cudaSuccess;
  const size_t need = kMlpParams + size_t(n) * (F + H1 + H2 + 1);
  if (need > cap_) {
    release();
    cudaError_t e = cudaMalloc(&dev_, need * sizeof(float));
    if (e != cudaSuccess) return e;
    cap_ = need;
    loaded_ = nullptr;
  }
  float* w = dev_;
  float* dx = w + kMlpParams;
  float* h1 = dx + size_t(n) * F;
  float* h2 = h1 + size_t(n) * H1;
  float* sc = h2 + size_t(n) * H2;
  cudaError_t e = cudaSuccess;
  if (loaded_ != weights_host) {
    e = cudaMemcpy(w, weights_host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    loaded_ = weights_host;
  }
  e = cudaMemcpy(dx, x, size_t(n) * F * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  forward(w, dx, h1, h2, sc, n, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpy(out, sc, size_t(n) * sizeof(float), cudaMemcpyDeviceToHost);
}

cudaError_t mlp_train(const float* pairs, int n_pairs, int epochs, int batch, float lr, uint64_t seed, float* weights,
                      double* final_loss) {
  if (n_pairs <= 0 || batch <= 0) return cudaErrorInvalidValue;
  const int P = batch < n_pairs ? batch : n_pairs, B = 2 * P;
  std::vector<float> w(kMlpParams);
  mlp_init(w.data(), seed);
  float *d_w, *d_g, *d_m, *d_v, *d_data, *d_x, *d_h1, *d_h2, *d_s, *d_ds, *d_dh1, *d_dh2, *d_loss;
  const size_t np = kMlpParams;
  std::vector<void**> ptrs = {(void**)&d_w, (void**)&d_g, (void**)&d_m, (void**)&d_v};
  for (auto p : ptrs) {
    if (cudaMalloc(p, np * sizeof(float)) != cudaSuccess) return cudaErrorMemoryAllocation;
    cudaMemset(*p, 0, np * sizeof(float));
  }
  if (cudaMalloc(&d_data, size_t(n_pairs) * 2 * F * sizeof(float)) != cudaSuccess) return cudaErrorMemoryAllocation;
  cudaMalloc(&d_x, size_t(B) * F * sizeof(float));
  cudaMalloc(&d_h1, size_t(B) * H1 * sizeof(float));
  cudaMalloc(&d_h2, size_t(B) * H2 * sizeof(float));
  cudaMalloc(&d_s, size_t(B) * sizeof(float));
  cudaMalloc(&d_ds, size_t(B) * sizeof(float));
  cudaMalloc(&d_dh1, size_t(B) * H1 * sizeof(float));
  cudaMalloc(&d_dh2, size_t(B) * H2 * sizeof(float));
  cudaMalloc(&d_loss, sizeof(float));
  cudaMemcpy(d_w, w.data(), np * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(d_data, pairs, size_t(n_pairs) * 2 * F * sizeof(float), cudaMemcpyHostToDevice);
  // order of pairs per epoch: a seeded permutation (host), batches gathered by copies
  std::vector<int> perm(n_pairs);
  for (int i = 0; i < n_pairs; ++i) perm[i] = i;
  uint64_t st = seed + 12345;
  auto rnd = [&]() {
    st ^= st << 13;
    st ^= st >> 7;
    st ^= st << 17;
    return st;
  };
  int* d_perm = nullptr;
  if (cudaMalloc(&d_perm, size_t(n_pairs) * sizeof(int)) != cudaSuccess) return cudaErrorMemoryAllocation;
  int step = 0;
  float loss_h = 0;
  double epoch_loss = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = n_pairs - 1; i > 0; --i) std::swap(perm[i], perm[rnd() % (i + 1)]);
    cudaMemcpy(d_perm, perm.data(), size_t(n_pairs) * sizeof(int), cudaMemcpyHostToDevice);
    epoch_loss = 0;
    int nb = 0;
    for (int b0 = 0; b0 + P <= n_pairs; b0 += P, ++nb) {
      k_gather_pairs<<<blocks(int64_t(2) * P * F, 256), 256>>>(d_data, d_perm, b0, P, d_x);
      cudaMemsetAsync(d_loss, 0, sizeof(float), 0);
      forward(d_w, d_x, d_h1, d_h2, d_s, B, 0);
      k_rank_loss<<<blocks(P, 256), 256>>>(d_s, d_ds, d_loss, P);
      k_grad_head<<<blocks(H2 + 1, 256), 256>>>(d_ds, d_h2, d_g + OFF_W3, d_g + OFF_B3, B);
      k_back_head<<<blocks(int64_t(B) * H2, 256), 256>>>(d_ds, d_w + OFF_W3, d_h2, d_dh2, B);
      k_grad_dense<<<blocks(H2 * (H1 + 1), 256), 256>>>(d_dh2, d_h1, d_g + OFF_W2, d_g + OFF_B2, B, H1, H2);
      k_back_hidden<<<blocks(int64_t(B) * H1, 256), 256>>>(d_dh2, d_w + OFF_W2, d_h1, d_dh1, B, H2, H1);
      k_grad_dense<<<blocks(H1 * (F + 1), 256), 256>>>(d_dh1, d_x, d_g + OFF_W1, d_g + OFF_B1, B, F, H1);
      ++step;
      const float b1 = 0.9f, b2 = 0.999f;
      k_adam<<<blocks(np, 256), 256>>>(d_w, d_g, d_m, d_v, static_cast<int>(np), lr, b1, b2,
                                       std::pow(b1, static_cast<float>(step)), std::pow(b2, static_cast<float>(step)));
      cudaMemcpy(&loss_h, d_loss, sizeof(float), cudaMemcpyDeviceToHost);
      epoch_loss += loss_h;
    }
    if (nb) epoch_loss /= nb;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(weights, d_w, np * sizeof(float), cudaMemcpyDeviceToHost);
  if (final_loss) *final_loss = epoch_loss;
  for (float* p : {d_w, d_g, d_m, d_v, d_data, d_x, d_h1, d_h2, d_s, d_ds, d_dh1, d_dh2, d_loss}) cudaFree(p);
  cudaFree(d_perm);
  return e;
}

}  // namespace ajf
