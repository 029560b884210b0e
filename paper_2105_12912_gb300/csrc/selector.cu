// Learned codec selector: batched inference and full-batch training of the per-block
// MLP (8 -> 32 -> 32 -> 3, ReLU) that predicts log2 bits per element of each codec.
// Training rows come from the method itself (csz_selector_rows: features and exact
// encoded sizes of every block).  The loss is the mean over rows and outputs of the
// squared error; the optimiser is Adam.
//
// Kernel layout: one warp per row at a time, lane i owning hidden unit i of both
// layers, so the forward pass is a shuffle-broadcast of the activations and the
// backward pass accumulates each lane's rows of dW1 and dW2 in registers.  Partial
// sums per CTA go to the workspace and are added in a fixed order by the update
// kernel, so a training run is reproducible bit for bit on one GPU model.
#include <cmath>
#include <cstring>

#include "cszp.h"
#include "kernels.h"

namespace cszp {
namespace {

constexpr int kTrainThreads = 256;
constexpr int kTrainWarps = kTrainThreads / 32;
constexpr int kPart = kMlpParams + 2;  // gradient sums, loss sum, row count
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;

__global__ __launch_bounds__(256) void mlp_predict_kernel(const float* __restrict__ w,
                                                          const float* __restrict__ feat, uint64_t n,
                                                          float* __restrict__ out) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (uint64_t r = warp; r < n; r += nwarps) {
    float f[kMlpIn];
#pragma unroll
    for (int j = 0; j < kMlpIn; j++) f[j] = __ldg(&feat[r * kMlpIn + j]);
    float y[kMlpOut];
    mlp_forward_warp(w, f, y);
    const float mine = lane == 0 ? y[0] : (lane == 1 ? y[1] : y[2]);
    if (lane < kMlpOut) out[r * kMlpOut + lane] = mine;
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
  return v;
}

// Forward and backward over rows gw, gw + nw, ... of every warp; per-CTA sums of the
// unscaled gradient (d(e^2)/dy = 2e), of e^2 and of the row count go to part[cta].
__global__ __launch_bounds__(kTrainThreads) void mlp_grad_kernel(const float* __restrict__ w,
                                                                 const float* __restrict__ feat,
                                                                 const float* __restrict__ tgt,
                                                                 const uint8_t* __restrict__ valid,
                                                                 uint64_t n, float* __restrict__ part) {
  __shared__ float s_red[kTrainWarps][kPart];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float w1[kMlpIn], w2r[kMlpHid], w2c[kMlpHid], w3[kMlpOut], b3[kMlpOut];
  const float b1 = w[kMlpB1 + lane], b2 = w[kMlpB2 + lane];
#pragma unroll
  for (int j = 0; j < kMlpIn; j++) w1[j] = w[kMlpW1 + lane * kMlpIn + j];
#pragma unroll
  for (int j = 0; j < kMlpHid; j++) {
    w2r[j] = w[kMlpW2 + lane * kMlpHid + j];
    w2c[j] = w[kMlpW2 + j * kMlpHid + lane];
  }
#pragma unroll
  for (int c = 0; c < kMlpOut; c++) {
    w3[c] = w[kMlpW3 + c * kMlpHid + lane];
    b3[c] = w[kMlpB3 + c];
  }
  float g1[kMlpIn], g2[kMlpHid], g3[kMlpOut], gb3[kMlpOut];
  float gb1 = 0.0f, gb2 = 0.0f, loss = 0.0f, cnt = 0.0f;
#pragma unroll
  for (int j = 0; j < kMlpIn; j++) g1[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < kMlpHid; j++) g2[j] = 0.0f;
#pragma unroll
  for (int c = 0; c < kMlpOut; c++) g3[c] = gb3[c] = 0.0f;

  const uint64_t nw = (uint64_t)gridDim.x * kTrainWarps;
  for (uint64_t r = (uint64_t)blockIdx.x * kTrainWarps + wid; r < n; r += nw) {
    if (valid && !valid[r]) continue;  // warp-uniform
    float x[kMlpIn];
#pragma unroll
    for (int j = 0; j < kMlpIn; j++) x[j] = __ldg(&feat[r * kMlpIn + j]);
    // forward
    float a1 = b1;
#pragma unroll
    for (int j = 0; j < kMlpIn; j++) a1 = fmaf(w1[j], x[j], a1);
    const float h1 = a1 > 0.0f ? a1 : 0.0f;
    float h1all[kMlpHid];
    float a2 = b2;
#pragma unroll
    for (int j = 0; j < kMlpHid; j++) {
      h1all[j] = __shfl_sync(~0u, h1, j);
      a2 = fmaf(w2r[j], h1all[j], a2);
    }
    const float h2 = a2 > 0.0f ? a2 : 0.0f;
    float dy[kMlpOut];
#pragma unroll
    for (int c = 0; c < kMlpOut; c++) {
      const float y = b3[c] + warp_sum_f(w3[c] * h2);
      const float e = y - __ldg(&tgt[r * kMlpOut + c]);
      loss = fmaf(e, e, loss);
      dy[c] = 2.0f * e;
    }
    cnt += 1.0f;
    // backward
    float dh2 = 0.0f;
#pragma unroll
    for (int c = 0; c < kMlpOut; c++) {
      g3[c] = fmaf(dy[c], h2, g3[c]);
      gb3[c] += dy[c];
      dh2 = fmaf(dy[c], w3[c], dh2);
    }
    const float da2 = a2 > 0.0f ? dh2 : 0.0f;
#pragma unroll
    for (int j = 0; j < kMlpHid; j++) g2[j] = fmaf(da2, h1all[j], g2[j]);
    gb2 += da2;
    float dh1 = 0.0f;
#pragma unroll
    for (int i = 0; i < kMlpHid; i++) dh1 = fmaf(w2c[i], __shfl_sync(~0u, da2, i), dh1);
    const float da1 = a1 > 0.0f ? dh1 : 0.0f;
#pragma unroll
    for (int j = 0; j < kMlpIn; j++) g1[j] = fmaf(da1, x[j], g1[j]);
    gb1 += da1;
  }

  float* my = s_red[wid];
#pragma unroll
  for (int j = 0; j < kMlpIn; j++) my[kMlpW1 + lane * kMlpIn + j] = g1[j];
  my[kMlpB1 + lane] = gb1;
#pragma unroll
  for (int j = 0; j < kMlpHid; j++) my[kMlpW2 + lane * kMlpHid + j] = g2[j];
  my[kMlpB2 + lane] = gb2;
#pragma unroll
  for (int c = 0; c < kMlpOut; c++) my[kMlpW3 + c * kMlpHid + lane] = g3[c];
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < kMlpOut; c++) my[kMlpB3 + c] = gb3[c];
    my[kMlpParams] = loss;
    my[kMlpParams + 1] = cnt;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kPart; p += kTrainThreads) {
    float acc = 0.0f;
#pragma unroll
    for (int wv = 0; wv < kTrainWarps; wv++) acc += s_red[wv][p];
    part[(uint64_t)blockIdx.x * kPart + p] = acc;
  }
}

// Sum of the CTA partials in CTA order (double), scaled to the mean over rows and
// outputs; optionally one Adam step on the weights.  Thread p handles parameter p;
// thread kMlpParams writes the loss.
__global__ __launch_bounds__(256) void mlp_update_kernel(const float* __restrict__ part, int nparts,
                                                         float* __restrict__ w, float* __restrict__ grad_out,
                                                         double* __restrict__ loss_out, float* __restrict__ m,
                                                         float* __restrict__ v, uint32_t step, float lr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kMlpParams) return;
  double cnt = 0.0, acc = 0.0;
  for (int g = 0; g < nparts; g++) {
    cnt += part[(uint64_t)g * kPart + kMlpParams + 1];
    acc += part[(uint64_t)g * kPart + p];
  }
  const double scale = cnt > 0.0 ? 1.0 / (3.0 * cnt) : 0.0;
  if (p == kMlpParams) {
    if (loss_out) *loss_out = acc * scale;
    return;
  }
  const float gr = (float)(acc * scale);
  if (grad_out) grad_out[p] = gr;
  if (step) {
    const float mt = kAdamB1 * m[p] + (1.0f - kAdamB1) * gr;
    const float vt = kAdamB2 * v[p] + (1.0f - kAdamB2) * gr * gr;
    m[p] = mt;
    v[p] = vt;
    const float c1 = (float)(1.0 - pow((double)kAdamB1, (double)step));
    const float c2 = (float)(1.0 - pow((double)kAdamB2, (double)step));
    w[p] -= lr * (mt / c1) / (sqrtf(vt / c2) + kAdamEps);
  }
}

int g_sms = 0;

int train_grid(uint64_t nrows) {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  const uint64_t want = (nrows + 4 * kTrainWarps - 1) / (4 * kTrainWarps);
  const uint64_t cap = 2ull * g_sms;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

uint64_t a256(uint64_t v) { return (v + 255) & ~255ull; }

// workspace: partials [grid][kPart] f32 | Adam m, v [params] f32 | loss f64
struct TrainLayout {
  uint64_t part, m, v, loss, total;
};

TrainLayout train_layout(int grid) {
  TrainLayout L;
  L.part = 0;
  L.m = a256((uint64_t)grid * kPart * 4);
  L.v = L.m + a256(kMlpParams * 4);
  L.loss = L.v + a256(kMlpParams * 4);
  L.total = L.loss + 256;
  return L;
}

template <typename T>
T* at(void* base, uint64_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(base) + off);
}

}  // namespace

cudaError_t launch_mlp_grad(const float* w, const float* feat, const float* tgt, const uint8_t* valid,
                            uint64_t n, float* part, int grid, cudaStream_t s) {
  trace_begin(K_MLP_GRAD, s);
  mlp_grad_kernel<<<grid, kTrainThreads, 0, s>>>(w, feat, tgt, valid, n, part);
  trace_end(K_MLP_GRAD, s);
  return cudaGetLastError();
}

cudaError_t launch_mlp_update(const float* part, int nparts, float* w, float* grad, double* loss, float* m,
                              float* v, uint32_t step, float lr, cudaStream_t s) {
  trace_begin(K_MLP_UPDATE, s);
  mlp_update_kernel<<<(kMlpParams + 1 + 255) / 256, 256, 0, s>>>(part, nparts, w, grad, loss, m, v, step, lr);
  trace_end(K_MLP_UPDATE, s);
  return cudaGetLastError();
}

}  // namespace cszp

using namespace cszp;

extern "C" {

size_t csz_selector_workspace_bytes(uint64_t nrows) { return (size_t)train_layout(train_grid(nrows)).total; }

csz_status csz_selector_predict(const float* d_w, const float* d_feat, uint64_t nrows, float* d_out, void* stream) {
  if (!d_w || (nrows && (!d_feat || !d_out))) return CSZ_E_ARG;
  if (nrows == 0) return CSZ_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t blocks = (nrows + 7) / 8;
  const unsigned grid = (unsigned)(blocks < 4096 ? blocks : 4096);
  trace_begin(K_MLP_PREDICT, s);
  mlp_predict_kernel<<<grid, 256, 0, s>>>(d_w, d_feat, nrows, d_out);
  trace_end(K_MLP_PREDICT, s);
  if (cudaGetLastError() != cudaSuccess) return CSZ_E_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? CSZ_OK : CSZ_E_CUDA;
}

csz_status csz_selector_grad(const float* d_w, const float* d_feat, const float* d_target, const uint8_t* d_valid,
                             uint64_t nrows, float* d_grad, double* h_loss, void* d_ws, size_t ws_bytes,
                             void* stream) {
  if (!d_w || !d_grad || !d_ws || (nrows && (!d_feat || !d_target))) return CSZ_E_ARG;
  const int grid = train_grid(nrows);
  const TrainLayout L = train_layout(grid);
  if (ws_bytes < L.total) return CSZ_E_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = at<float>(d_ws, L.part);
  double* loss = at<double>(d_ws, L.loss);
  if (launch_mlp_grad(d_w, d_feat, d_target, d_valid, nrows, part, grid, s) != cudaSuccess) return CSZ_E_CUDA;
  if (launch_mlp_update(part, grid, nullptr, d_grad, loss, nullptr, nullptr, 0, 0.0f, s) != cudaSuccess)
    return CSZ_E_CUDA;
  double hl = 0.0;
  if (cudaMemcpyAsync(&hl, loss, sizeof(hl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  if (h_loss) *h_loss = hl;
  return CSZ_OK;
}

csz_status csz_selector_train(float* d_w, const float* d_feat, const float* d_target, const uint8_t* d_valid,
                              uint64_t nrows, uint32_t steps, float lr, void* d_ws, size_t ws_bytes,
                              double* h_loss, void* stream) {
  if (!d_w || !d_ws || (nrows && (!d_feat || !d_target))) return CSZ_E_ARG;
  if (!(lr > 0.0f) || !std::isfinite(lr)) return CSZ_E_ARG;
  const int grid = train_grid(nrows);
  const TrainLayout L = train_layout(grid);
  if (ws_bytes < L.total) return CSZ_E_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* part = at<float>(d_ws, L.part);
  float* m = at<float>(d_ws, L.m);
  float* v = at<float>(d_ws, L.v);
  double* loss = at<double>(d_ws, L.loss);
  if (cudaMemsetAsync(m, 0, L.loss - L.m, s) != cudaSuccess) return CSZ_E_CUDA;
  for (uint32_t t = 1; t <= steps; t++) {
    // learning rate decays linearly to a tenth of lr over the run
    const float lr_t = lr * (1.0f - 0.9f * (float)(t - 1) / (float)steps);
    if (launch_mlp_grad(d_w, d_feat, d_target, d_valid, nrows, part, grid, s) != cudaSuccess) return CSZ_E_CUDA;
    if (launch_mlp_update(part, grid, d_w, nullptr, loss, m, v, t, lr_t, s) != cudaSuccess) return CSZ_E_CUDA;
  }
  double hl = 0.0;
  if (steps && cudaMemcpyAsync(&hl, loss, sizeof(hl), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  if (h_loss) *h_loss = hl;
  return CSZ_OK;
}

}  // extern "C"
