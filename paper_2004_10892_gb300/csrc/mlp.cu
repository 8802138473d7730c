// mlp.cu -- training and inference kernels of the learned slicing proposer:
// a 3-layer MLP (features -> H -> H -> 1, ReLU, FP32) trained with a mean
// squared error on log2 contraction costs. Parameters are one flat array:
// W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1), weights row-major
// (output x input). Every reduction runs in a fixed order (no atomics), so
// a training step is deterministic.
#include <cuda_runtime.h>

#include <string>

#include "../../include/tnq.h"

namespace tnq {
void set_error(const std::string& msg);

namespace {
constexpr int TS = 16;  // matmul tile

// C[M x P] = opA(A) . opB(B) (+ bias[P]) (ReLU if relu): opA(A) is M x K
// (A stored M x K, or K x M when ta), opB(B) is K x P (B stored P x K when
// tb, else K x P). FP32 accumulation over K in increasing order.
__global__ void k_mm(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ bias,
                     float* __restrict__ C, int M, int K, int P, int ta, int tb, int relu) {
  __shared__ float sa[TS][TS + 1], sb[TS][TS + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * TS + ty, col = blockIdx.x * TS + tx;
  float acc = 0.f;
  for (int k0 = 0; k0 < K; k0 += TS) {
    const int ka = k0 + tx, kb = k0 + ty;
    float va = 0.f, vb = 0.f;
    if (row < M && ka < K) va = ta ? A[(size_t)ka * M + row] : A[(size_t)row * K + ka];
    if (col < P && kb < K) vb = tb ? B[(size_t)col * K + kb] : B[(size_t)kb * P + col];
    sa[ty][tx] = va;
    sb[ty][tx] = vb;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TS; ++k) acc += sa[ty][k] * sb[k][tx];
    __syncthreads();
  }
  if (row < M && col < P) {
    if (bias) acc += bias[col];
    if (relu) acc = acc > 0.f ? acc : 0.f;
    C[(size_t)row * P + col] = acc;
  }
}

// g[i] *= (z[i] > 0): ReLU derivative applied to an upstream gradient.
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!(z[i] > 0.f)) g[i] = 0.f;
}

// out[c] = sum_r X[r, c] over rows in increasing order (one thread per column).
__global__ void k_colsum(const float* __restrict__ X, float* __restrict__ out, int rows, int cols) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float a = 0.f;
  for (int r = 0; r < rows; ++r) a += X[(size_t)r * cols + c];
  out[c] = a;
}

// d[i] = (pred[i] - y[i]) / n ; loss = sum (pred - y)^2 / (2n), summed in order by one block.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ y, float* __restrict__ d,
                      float* __restrict__ loss, int n) {
  __shared__ float part[256];
  float a = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float e = pred[i] - y[i];
    d[i] = e / (float)n;
    a += e * e;
  }
  part[threadIdx.x] = a;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    float t = 0.f;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
    *loss = t / (2.f * (float)n);
  }
}

// SGD with momentum: v = mu v + g ; w -= lr v.
__global__ void k_sgd(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ v, size_t n, float lr,
                      float mu) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float vi = mu * v[i] + g[i];
    v[i] = vi;
    w[i] -= lr * vi;
  }
}

void mm(const float* A, const float* B, const float* bias, float* C, int M, int K, int P, int ta, int tb, int relu,
       cudaStream_t s) {
  dim3 blk(TS, TS), grd((P + TS - 1) / TS, (M + TS - 1) / TS);
  k_mm<<<grd, blk, 0, s>>>(A, B, bias, C, M, K, P, ta, tb, relu);
}

struct Views {
  const float *W1, *b1, *W2, *b2, *W3, *b3;
};
Views views(const float* p, int F, int H) {
  Views v;
  v.W1 = p;
  v.b1 = v.W1 + (size_t)H * F;
  v.W2 = v.b1 + H;
  v.b2 = v.W2 + (size_t)H * H;
  v.W3 = v.b2 + H;
  v.b3 = v.W3 + H;
  return v;
}
}  // namespace
}  // namespace tnq

using namespace tnq;

extern "C" {

int32_t tnq_learned_features(void);
size_t tnq_learned_param_count(int32_t hidden);

size_t tnq_mlp_workspace_floats(int32_t hidden, size_t n) { return n * (5 * (size_t)hidden + 4) + 16; }

// Forward pass for n rows of features x (device, n x F) -> out (device, n).
tnq_status tnq_mlp_forward(const float* params, int32_t hidden, const float* x, size_t n, float* out, float* work,
                           void* stream) {
  if (!params || !x || !out || !work || hidden <= 0) { set_error("NULL argument"); return TNQ_EINVAL; }
  const int F = tnq_learned_features(), H = hidden, N = (int)n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Views v = views(params, F, H);
  float* H1 = work;
  float* H2 = H1 + (size_t)N * H;
  mm(x, v.W1, v.b1, H1, N, F, H, 0, 1, 1, s);
  mm(H1, v.W2, v.b2, H2, N, H, H, 0, 1, 1, s);
  mm(H2, v.W3, v.b3, out, N, H, 1, 0, 1, 0, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return TNQ_ECUDA; }
  return TNQ_OK;
}

// Gradient of the mean squared error (1/2n) sum (f(x) - y)^2 with respect to
// every parameter, into grads (device, same layout as params); *loss (device).
tnq_status tnq_mlp_backward(const float* params, int32_t hidden, const float* x, const float* y, size_t n,
                            float* grads, float* loss, float* work, void* stream) {
  if (!params || !x || !y || !grads || !work || hidden <= 0 || n == 0) { set_error("bad argument"); return TNQ_EINVAL; }
  const int F = tnq_learned_features(), H = hidden, N = (int)n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Views v = views(params, F, H);
  float* Z1 = work;                       // N x H pre-activations, then dZ1
  float* H1 = Z1 + (size_t)N * H;         // N x H
  float* Z2 = H1 + (size_t)N * H;         // N x H, then dZ2
  float* H2 = Z2 + (size_t)N * H;         // N x H
  float* D = H2 + (size_t)N * H;          // N x H scratch (dH)
  float* P = D + (size_t)N * H;           // N
  float* dP = P + N;                      // N
  float* g_W1 = grads;
  float* g_b1 = g_W1 + (size_t)H * F;
  float* g_W2 = g_b1 + H;
  float* g_b2 = g_W2 + (size_t)H * H;
  float* g_W3 = g_b2 + H;
  float* g_b3 = g_W3 + H;
  // forward, keeping pre-activations
  mm(x, v.W1, v.b1, Z1, N, F, H, 0, 1, 0, s);
  mm(x, v.W1, v.b1, H1, N, F, H, 0, 1, 1, s);
  mm(H1, v.W2, v.b2, Z2, N, H, H, 0, 1, 0, s);
  mm(H1, v.W2, v.b2, H2, N, H, H, 0, 1, 1, s);
  mm(H2, v.W3, v.b3, P, N, H, 1, 0, 1, 0, s);
  k_mse<<<1, 256, 0, s>>>(P, y, dP, loss, N);
  // layer 3: dW3 = dP^T H2 ; db3 = sum dP ; dH2 = dP W3
  mm(dP, H2, nullptr, g_W3, 1, N, H, 1, 0, 0, s);
  k_colsum<<<1, 32, 0, s>>>(dP, g_b3, N, 1);
  mm(dP, v.W3, nullptr, D, N, 1, H, 0, 0, 0, s);
  // layer 2
  const size_t nh = (size_t)N * H;
  const int blocks = (int)((nh + 255) / 256 < 4096 ? (nh + 255) / 256 : 4096);
  k_relu_mask<<<blocks, 256, 0, s>>>(D, Z2, nh);  // D = dZ2
  mm(D, H1, nullptr, g_W2, H, N, H, 1, 0, 0, s);
  k_colsum<<<(H + 127) / 128, 128, 0, s>>>(D, g_b2, N, H);
  mm(D, v.W2, nullptr, Z2, N, H, H, 0, 0, 0, s);  // Z2 <- dH1
  // layer 1
  k_relu_mask<<<blocks, 256, 0, s>>>(Z2, Z1, nh);  // Z2 = dZ1
  mm(Z2, x, nullptr, g_W1, H, N, F, 1, 0, 0, s);
  k_colsum<<<(H + 127) / 128, 128, 0, s>>>(Z2, g_b1, N, H);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return TNQ_ECUDA; }
  return TNQ_OK;
}

tnq_status tnq_mlp_sgd(float* params, const float* grads, float* momentum, size_t count, float lr, float mu,
                       void* stream) {
  if (!params || !grads || !momentum) { set_error("NULL argument"); return TNQ_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int blocks = (int)((count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024);
  k_sgd<<<blocks > 0 ? blocks : 1, 256, 0, s>>>(params, grads, momentum, count, lr, mu);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return TNQ_ECUDA; }
  return TNQ_OK;
}

}  // extern "C"
