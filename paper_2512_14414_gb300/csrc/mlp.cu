// Forward pass of the multilayer perceptron that predicts an initial CTMRG environment from the
// site tensors (the learned warm start: a starting point for the iterations of Sec. SLF, step ii).
//
//   h_0 = x;  h_{k+1} = GELU(h_k W_k^t + b_k) for the hidden layers;  y = h_L W_L^t + b_L
//
// W_k is [out][in] row-major (the layout of torch.nn.Linear), x is [batch][in], y [batch][out],
// all FP32.  Each layer is one GEMM (the library's CUDA-core or tensor-core path by size) and one
// fused bias + GELU kernel; GELU is the exact form 0.5 x (1 + erf(x / sqrt 2)).
#include <cmath>

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

}  // namespace ctm
