// Cost model of the learned planner: a 3-layer perceptron, 64 units wide,
//     h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), yhat = h2 W3 + b3,
// trained on measured plan times with mean squared error on log-time and Adam.
// Forward, backward and the optimiser step are hand-written kernels; parameters are one
// flat FP32 buffer [W1 (d x 64) | b1 (64) | W2 (64 x 64) | b2 (64) | W3 (64) | b3 (1)].
#include <cuda_runtime.h>

#include "../../include/lmfao.h"

namespace lmfao {

namespace {

constexpr int H = 64;

__host__ __device__ inline int64_t off_b1(int d) { return (int64_t)d * H; }
__host__ __device__ inline int64_t off_w2(int d) { return off_b1(d) + H; }
__host__ __device__ inline int64_t off_b2(int d) { return off_w2(d) + H * H; }
__host__ __device__ inline int64_t off_w3(int d) { return off_b2(d) + H; }
__host__ __device__ inline int64_t off_b3(int d) { return off_w3(d) + H; }

// one CTA of 64 threads per sample: thread j owns hidden unit j of both layers
__global__ void mlp_forward_kernel(const float *x, int n, int d, const float *p, float *h1, float *h2, float *y) {
  __shared__ float sx[256];
  __shared__ float s1[H];
  __shared__ float red[H];
  const int i = blockIdx.x, j = threadIdx.x;
  if (i >= n) return;
  for (int k = j; k < d; k += H) sx[k] = x[(int64_t)i * d + k];
  __syncthreads();
  float a = p[off_b1(d) + j];
  for (int k = 0; k < d; ++k) a += sx[k] * p[(int64_t)k * H + j];
  a = a > 0.f ? a : 0.f;
  s1[j] = a;
  if (h1) h1[(int64_t)i * H + j] = a;
  __syncthreads();
  float b = p[off_b2(d) + j];
  for (int k = 0; k < H; ++k) b += s1[k] * p[off_w2(d) + k * H + j];
  b = b > 0.f ? b : 0.f;
  if (h2) h2[(int64_t)i * H + j] = b;
  red[j] = b * p[off_w3(d) + j];
  __syncthreads();
  for (int s = H / 2; s > 0; s >>= 1) {
    if (j < s) red[j] += red[j + s];
    __syncthreads();
  }
  if (j == 0) y[i] = red[0] + p[off_b3(d)];
}

// per-sample output gradient of the loss mean((yhat - t)^2): g_i = 2 (yhat_i - t_i) / n
__global__ void mlp_loss_kernel(const float *y, const float *t, int n, float *g, float *loss) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    float e = y[i] - t[i];
    g[i] = 2.f * e / n;
    atomicAdd(loss, e * e / n);
  }
}

// backward through both hidden layers, one CTA of 64 threads per sample; parameter
// gradients are accumulated with atomics into grad (zeroed by the caller)
__global__ void mlp_backward_kernel(const float *x, int n, int d, const float *p, const float *h1, const float *h2,
                                    const float *g, float *grad) {
  __shared__ float sx[256];
  __shared__ float d2[H];
  __shared__ float s1[H];
  const int i = blockIdx.x, j = threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  for (int k = j; k < d; k += H) sx[k] = x[(int64_t)i * d + k];
  const float a1 = h1[(int64_t)i * H + j], a2 = h2[(int64_t)i * H + j];
  s1[j] = a1;
  // layer 3
  atomicAdd(grad + off_w3(d) + j, gi * a2);
  if (j == 0) atomicAdd(grad + off_b3(d), gi);
  // layer 2
  const float dz2 = a2 > 0.f ? gi * p[off_w3(d) + j] : 0.f;
  d2[j] = dz2;
  __syncthreads();
  for (int k = 0; k < H; ++k)
    if (dz2 != 0.f) atomicAdd(grad + off_w2(d) + k * H + j, s1[k] * dz2);
  atomicAdd(grad + off_b2(d) + j, dz2);
  // layer 1
  float dh1 = 0.f;
  for (int q = 0; q < H; ++q) dh1 += p[off_w2(d) + j * H + q] * d2[q];
  const float dz1 = a1 > 0.f ? dh1 : 0.f;
  for (int k = 0; k < d; ++k)
    if (dz1 != 0.f) atomicAdd(grad + (int64_t)k * H + j, sx[k] * dz1);
  atomicAdd(grad + off_b1(d) + j, dz1);
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int64_t np, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

int64_t mlp_param_count(int d) { return off_b3(d) + 1; }

}  // namespace lmfao

using namespace lmfao;

extern "C" {

int64_t lmfao_mlp_param_count(int d) { return (d <= 0 || d > 256) ? -1 : mlp_param_count(d); }

int lmfao_mlp_forward(const float *x, int n, int d, const float *params, float *h1, float *h2, float *y, void *stream) {
  if (n < 0 || d <= 0 || d > 256 || (n && (!x || !params || !y))) return LMFAO_ERR_ARG;
  if (n == 0) return LMFAO_OK;
  mlp_forward_kernel<<<n, H, 0, (cudaStream_t)stream>>>(x, n, d, params, h1, h2, y);
  return cudaGetLastError() == cudaSuccess ? LMFAO_OK : LMFAO_ERR_CUDA;
}

int lmfao_mlp_backward(const float *x, int n, int d, const float *params, const float *h1, const float *h2,
                       const float *gy, float *grad, void *stream) {
  if (n < 0 || d <= 0 || d > 256 || (n && (!x || !params || !h1 || !h2 || !gy || !grad))) return LMFAO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(grad, 0, mlp_param_count(d) * sizeof(float), s) != cudaSuccess) return LMFAO_ERR_CUDA;
  if (n) mlp_backward_kernel<<<n, H, 0, s>>>(x, n, d, params, h1, h2, gy, grad);
  return cudaGetLastError() == cudaSuccess ? LMFAO_OK : LMFAO_ERR_CUDA;
}

int lmfao_mlp_loss(const float *y, const float *t, int n, float *gy, float *loss, void *stream) {
  if (n < 0 || (n && (!y || !t || !gy || !loss))) return LMFAO_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return LMFAO_ERR_CUDA;
  if (n) mlp_loss_kernel<<<(n + 255) / 256, 256, 0, s>>>(y, t, n, gy, loss);
  return cudaGetLastError() == cudaSuccess ? LMFAO_OK : LMFAO_ERR_CUDA;
}

int lmfao_mlp_adam(float *params, const float *grad, float *m, float *v, int64_t np, int step, float lr, void *stream) {
  if (np <= 0 || step < 1 || !params || !grad || !m || !v) return LMFAO_ERR_ARG;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f, c2 = 1.f;
  for (int i = 0; i < step; ++i) { c1 *= b1; c2 *= b2; }
  adam_kernel<<<(int)((np + 255) / 256), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, np, lr, b1, b2, 1e-8f,
                                                                         1.f - c1, 1.f - c2);
  return cudaGetLastError() == cudaSuccess ? LMFAO_OK : LMFAO_ERR_CUDA;
}

}  // extern "C"
