// Forward and backward passes of the multilayer perceptron that predicts an initial CTMRG
// environment from the site tensors (the learned warm start: a starting point for the iterations
// of Sec. SLF, step ii), and the Adam step that trains it.
//
//   h_0 = x;  h_{k+1} = GELU(h_k W_k^t + b_k) for the hidden layers;  y = h_L W_L^t + b_L
//
// W_k is [out][in] row-major (the layout of torch.nn.Linear), x is [batch][in], y [batch][out],
// all FP32.  Each layer is one GEMM (the library's CUDA-core or tensor-core path by size) and one
// fused bias + GELU kernel; GELU is the exact form 0.5 x (1 + erf(x / sqrt 2)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.h"

namespace ctm {
namespace {

__global__ void bias_gelu_k(float* y, const float* b, int64_t rows, int64_t cols, int gelu) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float v = y[e] + (b ? b[e % cols] : 0.f);
    if (gelu) v = 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
    y[e] = v;
  }
}

}  // namespace

void mlp_forward(const float* x, int batch, int n_layers, const int* dims, const float* const* W,
                 const float* const* b, float* work, float* y, cudaStream_t st) {
  int64_t maxd = 0;
  for (int k = 1; k < n_layers; ++k) maxd = std::max<int64_t>(maxd, dims[k]);
  const float* in = x;
  for (int k = 0; k < n_layers; ++k) {
    const bool last = k == n_layers - 1;
    float* out = last ? y : work + (int64_t)(k % 2) * batch * maxd;
    GemmSpec g;
    g.M = batch; g.N = dims[k + 1]; g.K = dims[k];
    g.transB = true; g.lda = dims[k]; g.ldb = dims[k]; g.ldc = dims[k + 1];
    gemm_f32(in, W[k], out, g, st);
    const int64_t n = (int64_t)batch * dims[k + 1];
    const int blocks = (int)std::min<int64_t>(65535 * 4, (n + 255) / 256);
    bias_gelu_k<<<std::max(blocks, 1), 256, 0, st>>>(out, b ? b[k] : nullptr, batch, dims[k + 1], last ? 0 : 1);
    CTM_LAUNCHED();
    in = out;
  }
}

namespace {

// z += b (stored), h = GELU(z)
__global__ void bias_gelu_keep_k(float* z, float* h, const float* b, int64_t rows, int64_t cols) {
  const int64_t n = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = z[e] + (b ? b[e % cols] : 0.f);
    z[e] = v;
    h[e] = 0.5f * v * (1.f + erff(v * 0.70710678118654752f));
  }
}

__global__ void bias_k(float* y, const float* b, int64_t rows, int64_t cols) {
  const int64_t n = rows * cols;
  if (!b) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] += b[e % cols];
}

// g = 2 (y - t) / n; per-block partial sums of (y - t)^2
__global__ void mse_grad_k(const float* y, const float* t, float* g, int64_t n, float* part) {
  __shared__ float sh[256];
  float acc = 0.f;
  const float sc = 2.f / (float)n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[e] - t[e];
    g[e] = sc * d;
    acc = fmaf(d, d, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void loss_final_k(const float* part, int nb, int64_t n, float* loss) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (float)n;
}

// dz = dh * GELU'(z), GELU'(z) = Phi(z) + z phi(z)
__global__ void gelu_back_k(const float* dh, const float* z, float* dz, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = z[e];
    const float Phi = 0.5f * (1.f + erff(v * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * v * v);
    dz[e] = dh[e] * (Phi + v * phi);
  }
}

// db[j] = sum over rows of dz[row][j]
__global__ void col_sum_k(const float* dz, float* db, int64_t rows, int64_t cols) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int64_t r = 0; r < rows; ++r) acc += dz[r * cols + j];
    db[j] = acc;
  }
}

__global__ void adam_k(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = b1 * m[e] + (1.f - b1) * ge;
    const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
  }
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(65535 * 4, (n + 255) / 256)); }

}  // namespace

int64_t mlp_work_floats(int batch, int n_layers, const int* dims) {
  int64_t maxd = 0, acts = 0;
  for (int k = 1; k <= n_layers; ++k) maxd = std::max<int64_t>(maxd, dims[k]);
  for (int k = 0; k < n_layers - 1; ++k) acts += 2 * (int64_t)batch * dims[k + 1];
  return acts + (int64_t)batch * dims[n_layers] + 2 * (int64_t)batch * maxd + 1024;
}

void mlp_backward(const float* x, const float* target, int batch, int n_layers, const int* dims,
                  const float* const* W, const float* const* b, float* const* dW, float* const* db, float* work,
                  float* loss, cudaStream_t st) {
  int64_t maxd = 0;
  for (int k = 1; k <= n_layers; ++k) maxd = std::max<int64_t>(maxd, dims[k]);
  // work: Z_0, H_0, ..., Z_{L-2}, H_{L-2} | Y | G0 | G1 | partial sums
  std::vector<float*> Z(n_layers), H(n_layers);
  float* p = work;
  for (int k = 0; k < n_layers - 1; ++k) {
    Z[k] = p;
    p += (int64_t)batch * dims[k + 1];
    H[k] = p;
    p += (int64_t)batch * dims[k + 1];
  }
  float* Y = p;
  p += (int64_t)batch * dims[n_layers];
  float* G[2] = {p, p + (int64_t)batch * maxd};
  float* part = p + 2 * (int64_t)batch * maxd;
  // forward, keeping the pre-activations
  const float* in = x;
  for (int k = 0; k < n_layers; ++k) {
    const bool last = k == n_layers - 1;
    float* out = last ? Y : Z[k];
    GemmSpec g;
    g.M = batch; g.N = dims[k + 1]; g.K = dims[k];
    g.transB = true; g.lda = dims[k]; g.ldb = dims[k]; g.ldc = dims[k + 1];
    gemm_f32(in, W[k], out, g, st);
    const int64_t n = (int64_t)batch * dims[k + 1];
    if (last) {
      bias_k<<<grid_for(n), 256, 0, st>>>(out, b ? b[k] : nullptr, batch, dims[k + 1]);
    } else {
      bias_gelu_keep_k<<<grid_for(n), 256, 0, st>>>(out, H[k], b ? b[k] : nullptr, batch, dims[k + 1]);
      in = H[k];
    }
    CTM_LAUNCHED();
  }
  // dL/dY and the loss
  const int64_t ny = (int64_t)batch * dims[n_layers];
  const int nb = std::min(1024, grid_for(ny));
  mse_grad_k<<<nb, 256, 0, st>>>(Y, target, G[0], ny, part);
  CTM_LAUNCHED();
  if (loss) {
    loss_final_k<<<1, 256, 0, st>>>(part, nb, ny, loss);
    CTM_LAUNCHED();
  }
  int cur = 0;
  for (int k = n_layers - 1; k >= 0; --k) {
    const float* hin = k > 0 ? H[k - 1] : x;
    const float* dz = G[cur];
    // dW_k = dZ_k^t h_{k}
    GemmSpec gw;
    gw.M = dims[k + 1]; gw.N = dims[k]; gw.K = batch;
    gw.transA = true; gw.lda = dims[k + 1]; gw.ldb = dims[k]; gw.ldc = dims[k];
    gemm_f32(dz, hin, dW[k], gw, st);
    if (db && db[k]) {
      col_sum_k<<<grid_for(dims[k + 1]), 256, 0, st>>>(dz, db[k], batch, dims[k + 1]);
      CTM_LAUNCHED();
    }
    if (k > 0) {
      // dH_{k-1} = dZ_k W_k, then through GELU'
      float* dh = G[1 - cur];
      GemmSpec gh;
      gh.M = batch; gh.N = dims[k]; gh.K = dims[k + 1];
      gh.lda = dims[k + 1]; gh.ldb = dims[k]; gh.ldc = dims[k];
      gemm_f32(dz, W[k], dh, gh, st);
      const int64_t n = (int64_t)batch * dims[k];
      gelu_back_k<<<grid_for(n), 256, 0, st>>>(dh, Z[k - 1], dh, n);
      CTM_LAUNCHED();
      cur = 1 - cur;
    }
  }
}

void adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int t,
               cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_k<<<grid_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  CTM_LAUNCHED();
}

}  // namespace ctm
