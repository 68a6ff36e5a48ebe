// Small MLP for learned Schwarz smoother parameters (spec extension; the
// paper fixes omega = 1 and the weight transition).  Maps level features
// (P_l, N_o, element aspect ratios, level) to two raw outputs that the caller
// turns into the damping omega_l and the transition width tau_l.
//
// Network: 6 -> 64 (tanh) -> 64 (tanh) -> 2, fp32, parameters packed as
// W1[6][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2].
// Loss: weighted mean squared error (1/B) sum_b w_b sum_o (y_bo - t_bo)^2.
// Backward: per-sample gradients into a work buffer, then a fixed-order sum
// over samples (deterministic), then Adam.
#include "pmg_internal.h"

namespace pmg {

constexpr int kIn = PMG_MLP_IN, kHid = PMG_MLP_HIDDEN, kOut = PMG_MLP_OUT;
constexpr int oW1 = 0, oB1 = oW1 + kIn * kHid, oW2 = oB1 + kHid, oB2 = oW2 + kHid * kHid,
              oW3 = oB2 + kHid, oB3 = oW3 + kHid * kOut, kNParam = oB3 + kOut;
static_assert(kNParam == PMG_MLP_NPARAM, "parameter count");

// One CTA (64 threads) per sample: h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), y = h2 W3 + b3.
__global__ void __launch_bounds__(kHid)
mlp_forward_kernel(const float* __restrict__ th, const float* __restrict__ x, int B,
                   float* __restrict__ y, float* __restrict__ h1g, float* __restrict__ h2g) {
  __shared__ float sx[kIn], s1[kHid], s2[kHid];
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  if (j < kIn) sx[j] = x[(size_t)b * kIn + j];
  __syncthreads();
  float a = th[oB1 + j];
#pragma unroll
  for (int i = 0; i < kIn; ++i) a = fmaf(sx[i], th[oW1 + i * kHid + j], a);
  s1[j] = tanhf(a);
  __syncthreads();
  a = th[oB2 + j];
#pragma unroll 8
  for (int k = 0; k < kHid; ++k) a = fmaf(s1[k], th[oW2 + k * kHid + j], a);
  s2[j] = tanhf(a);
  __syncthreads();
  if (h1g) h1g[(size_t)b * kHid + j] = s1[j];
  if (h2g) h2g[(size_t)b * kHid + j] = s2[j];
  if (j < kOut) {
    float o = th[oB3 + j];
    for (int k = 0; k < kHid; ++k) o = fmaf(s2[k], th[oW3 + k * kOut + j], o);
    y[(size_t)b * kOut + j] = o;
  }
}

// Per-sample gradient of w_b / B * sum_o (y_bo - t_bo)^2 into work[b][kNParam].
__global__ void __launch_bounds__(kHid)
mlp_backward_kernel(const float* __restrict__ th, const float* __restrict__ x,
                    const float* __restrict__ h1g, const float* __restrict__ h2g,
                    const float* __restrict__ y, const float* __restrict__ t,
                    const float* __restrict__ wgt, int B, float* __restrict__ work) {
  __shared__ float sx[kIn], s1[kHid], s2[kHid], dy[kOut], dz2[kHid];
  const int b = blockIdx.x, j = threadIdx.x;
  if (b >= B) return;
  float* g = work + (size_t)b * kNParam;
  if (j < kIn) sx[j] = x[(size_t)b * kIn + j];
  s1[j] = h1g[(size_t)b * kHid + j];
  s2[j] = h2g[(size_t)b * kHid + j];
  if (j < kOut) {
    const float wb = wgt ? wgt[b] : 1.0f;
    dy[j] = 2.0f * wb / (float)B * (y[(size_t)b * kOut + j] - t[(size_t)b * kOut + j]);
  }
  __syncthreads();
  // output layer
  float d2 = 0.0f;
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    g[oW3 + j * kOut + o] = s2[j] * dy[o];
    d2 = fmaf(dy[o], th[oW3 + j * kOut + o], d2);
  }
  if (j < kOut) g[oB3 + j] = dy[j];
  const float z2 = d2 * (1.0f - s2[j] * s2[j]);
  dz2[j] = z2;
  g[oB2 + j] = z2;
  __syncthreads();
  // hidden layer 2: dW2[k][j] = h1[k] dz2[j]; dh1[j] = sum_m dz2[m] W2[j][m]
  for (int k = 0; k < kHid; ++k) g[oW2 + k * kHid + j] = s1[k] * dz2[j];
  float d1 = 0.0f;
#pragma unroll 8
  for (int m = 0; m < kHid; ++m) d1 = fmaf(dz2[m], th[oW2 + j * kHid + m], d1);
  const float z1 = d1 * (1.0f - s1[j] * s1[j]);
  g[oB1 + j] = z1;
#pragma unroll
  for (int i = 0; i < kIn; ++i) g[oW1 + i * kHid + j] = sx[i] * z1;
}

// grad[p] = sum_b work[b][p] (fixed order); loss = sum_b w_b / B sum_o (y - t)^2.
__global__ void mlp_reduce_kernel(const float* __restrict__ work, int B, float* __restrict__ grad,
                                  const float* __restrict__ y, const float* __restrict__ t,
                                  const float* __restrict__ wgt, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kNParam) {
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += work[(size_t)b * kNParam + p];
    grad[p] = s;
  }
  if (p == 0 && loss) {
    float l = 0.0f;
    for (int b = 0; b < B; ++b) {
      const float wb = wgt ? wgt[b] : 1.0f;
      for (int o = 0; o < kOut; ++o) {
        const float e = y[(size_t)b * kOut + o] - t[(size_t)b * kOut + o];
        l += wb * e * e;
      }
    }
    *loss = l / (float)B;
  }
}

// Adam (Kingma & Ba), bias-corrected, step >= 1.
__global__ void mlp_adam_kernel(float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int n, int step, float lr, float b1, float b2,
                                float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  const float mh = mp / (1.0f - powf(b1, (float)step));
  const float vh = vp / (1.0f - powf(b2, (float)step));
  th[p] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace pmg

using namespace pmg;

extern "C" {

int pmg_mlp_forward(const float* theta, const float* x, int batch, float* y, float* h1, float* h2,
                    void* stream) {
  if (!theta || !x || !y || batch < 0) return PMG_EINVAL;
  if (batch == 0) return PMG_OK;
  count_launch();
  mlp_forward_kernel<<<batch, kHid, 0, (cudaStream_t)stream>>>(theta, x, batch, y, h1, h2);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

int pmg_mlp_backward(const float* theta, const float* x, const float* h1, const float* h2,
                     const float* y, const float* target, const float* weight, int batch, float* grad,
                     float* loss, float* work, void* stream) {
  if (!theta || !x || !h1 || !h2 || !y || !target || !grad || !work || batch <= 0) return PMG_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  count_launch();
  mlp_backward_kernel<<<batch, kHid, 0, s>>>(theta, x, h1, h2, y, target, weight, batch, work);
  count_launch();
  mlp_reduce_kernel<<<(kNParam + 127) / 128, 128, 0, s>>>(work, batch, grad, y, target, weight, loss);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

int pmg_mlp_adam(float* theta, const float* grad, float* m, float* v, int n, int step, float lr,
                 float beta1, float beta2, float eps, void* stream) {
  if (!theta || !grad || !m || !v || n <= 0 || step < 1 || !(lr > 0.0f)) return PMG_EINVAL;
  count_launch();
  mlp_adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, grad, m, v, n, step, lr,
                                                                      beta1, beta2, eps);
  return cudaGetLastError() == cudaSuccess ? PMG_OK : PMG_ECUDA;
}

}  // extern "C"
