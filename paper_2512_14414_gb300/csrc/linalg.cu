// Dense linear algebra of the projector step: batched Householder QR (FP64;
// Golub & Van Loan, Alg. 5.2.1 with LAPACK's reflector convention) and batched
// one-sided Jacobi SVD (Hestenes 1958; Rutishauser's rotation; cyclic
// round-robin ordering as in Brent & Luk 1985, or a block-cyclic ordering of
// groups of four columns), with an optional FP32 pre-pass before the FP64
// sweeps (see svd_product_full).
//
// Columns move between blocks from one step to the next, so every load of
// shared state in these kernels bypasses L1 (ld.global.cg).
//
// The QR and Jacobi kernels are persistent cooperative launches whose
// blocks meet at a software grid barrier between dependent steps.  Every
// wait is bounded: a block that waits too long raises DEV_TIMEOUT in the
// status word, sets the shared abort flag and returns; the others see the
// flag in their own waits and return as well.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "jacobi_order.h"
#include "kernels.h"

namespace ctm {
namespace {

struct Sync {
  unsigned* bar;  // [0] arrival count, [1] generation
  int* abort;
  int* status;
  long long limit;  // spins before a wait gives up (2^22 by default: a few seconds with the back-off below)
};

// Returns false if the barrier was abandoned (timeout or abort).
__device__ bool grid_barrier(const Sync& s) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = s.bar + 1;
    volatile int* vab = s.abort;
    unsigned g = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(s.bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(s.bar, 0u);
      __threadfence();
      atomicAdd(s.bar + 1, 1u);
    } else {
      long spins = 0;
      while (*vgen == g) {
        if (*vab) {
          ok = 0;
          break;
        }
        if (++spins > s.limit) {
          atomicOr(s.status, DEV_TIMEOUT);
          atomicExch(s.abort, 1);
          ok = 0;
          break;
        }
        if (spins > 64) __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reflector for column j of a column-major m x n matrix (ld = m): on exit A[j][j] = beta,
// A[j+1:, j] = v[1:], tau[j].  Executed by one full warp.
__device__ void make_reflector(double* A, double* tau, int m, int j, int lane) {
  double* col = A + (int64_t)j * m;
  double alpha = __ldcg(col + j);
  double s = 0.0;
  for (int i = j + 1 + lane; i < m; i += 32) {
    double v = __ldcg(col + i);
    s = fma(v, v, s);
  }
  s = warp_sum(s);
  double t = 0.0;
  if (s > 0.0) {
    double beta = -copysign(sqrt(alpha * alpha + s), alpha);
    t = (beta - alpha) / beta;
    double sc = 1.0 / (alpha - beta);
    for (int i = j + 1 + lane; i < m; i += 32) col[i] = __ldcg(col + i) * sc;
    __syncwarp();
    if (lane == 0) col[j] = beta;
  }
  if (lane == 0) tau[j] = t;
  __syncwarp();
}

// X[:, c] -= tau_j v_j (v_j . X[j:, c]) for one column (one warp).
__device__ void apply_reflector(const double* Acol_j, double tau_j, double* x, int m, int j, int lane) {
  if (tau_j == 0.0) return;
  double w = (lane == 0) ? __ldcg(x + j) : 0.0;
  for (int i = j + 1 + lane; i < m; i += 32) w = fma(__ldcg(Acol_j + i), __ldcg(x + i), w);
  w = warp_sum(w) * tau_j;
  if (lane == 0) x[j] = __ldcg(x + j) - w;
  for (int i = j + 1 + lane; i < m; i += 32) x[i] = fma(-w, __ldcg(Acol_j + i), __ldcg(x + i));
  __syncwarp();
}

__global__ void qr_kernel(double* A, double* tau, int batch, int m, int n, int64_t strideA, Sync s) {
  const int lane = threadIdx.x % 32;
  const int wpb = blockDim.x / 32;
  const int64_t gw = (int64_t)blockIdx.x * wpb + threadIdx.x / 32;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  // reflector of column 0
  for (int64_t b = gw; b < batch; b += nw) make_reflector(A + b * strideA, tau + b * n, m, 0, lane);
  for (int j = 0; j < n - 1; ++j) {
    if (!grid_barrier(s)) return;
    const int64_t ncols = n - j - 1;
    const int64_t tasks = (int64_t)batch * ncols;
    for (int64_t t = gw; t < tasks; t += nw) {
      const int64_t b = t / ncols;
      const int c = j + 1 + (int)(t % ncols);
      double* Ab = A + b * strideA;
      const double tj = __ldcg(tau + b * n + j);
      apply_reflector(Ab + (int64_t)j * m, tj, Ab + (int64_t)c * m, m, j, lane);
      if (c == j + 1) make_reflector(Ab, tau + b * n, m, j + 1, lane);
    }
  }
}

// X := Q X column by column: the k columns are independent, so one warp carries its column through
// all n reflectors (H_{n-1} first) with no grid-wide synchronisation; the reflectors are shared by
// every warp and stay in L2.
__global__ void apply_q_cols_kernel(const double* A, const double* tau, double* X, int batch, int m, int n, int k,
                                    int64_t strideA, int64_t strideX) {
  const int lane = threadIdx.x % 32;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t tasks = (int64_t)batch * k;
  for (int64_t t = gw; t < tasks; t += nw) {
    const int64_t b = t / k;
    const int c = (int)(t % k);
    double* x = X + b * strideX + (int64_t)c * m;
    for (int j = n - 1; j >= 0; --j)
      apply_reflector(A + b * strideA + (int64_t)j * m, __ldg(tau + b * n + j), x, m, j, lane);
  }
}

// ---- register-resident variants (m <= 32 * MAXE): a warp holds a whole column in registers, lane l
// owning rows l + 32 e, so that each reflector step issues all of its loads at once instead of one
// L2 round trip per element.

template <int MAXE>
__device__ __forceinline__ void load_col_r(const double* col, int m, int lane, double (&x)[MAXE]) {
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    x[e] = i < m ? __ldcg(col + i) : 0.0;
  }
}

template <int MAXE>
__device__ __forceinline__ void store_col_r(double* col, int m, int lane, const double (&x)[MAXE]) {
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    if (i < m) col[i] = x[e];
  }
}

// x -= tau v (v . x) with v = (.., 1 at row j, A[j+1:, j]) given in registers (rows > j of vcol).
template <int MAXE>
__device__ __forceinline__ void reflect_r(double (&x)[MAXE], const double (&v)[MAXE], double tj, int j, int lane) {
  double w = 0.0;
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    w = (i > j) ? fma(v[e], x[e], w) : (i == j ? w + x[e] : w);
  }
  w = warp_sum(w) * tj;
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    x[e] = (i > j) ? fma(-w, v[e], x[e]) : (i == j ? x[e] - w : x[e]);
  }
}

// Reflector of the column in registers at row j (the column is column j of the matrix): rows > j
// become v[1:], row j becomes beta; returns tau.
template <int MAXE>
__device__ __forceinline__ double make_reflector_r(double (&x)[MAXE], int j, int lane) {
  double alpha = 0.0, s = 0.0;
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    if (i == j) alpha = x[e];
    if (i > j) s = fma(x[e], x[e], s);
  }
  alpha = warp_sum(alpha);  // only the owning lane contributes
  s = warp_sum(s);
  if (!(s > 0.0)) return 0.0;
  const double beta = -copysign(sqrt(alpha * alpha + s), alpha);
  const double t = (beta - alpha) / beta;
  const double sc = 1.0 / (alpha - beta);
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int i = lane + 32 * e;
    if (i > j) x[e] *= sc;
    if (i == j) x[e] = beta;
  }
  return t;
}

template <int MAXE>
__global__ void qr_kernel_r(double* A, double* tau, int batch, int m, int n, int64_t strideA, Sync s) {
  const int lane = threadIdx.x % 32;
  const int wpb = blockDim.x / 32;
  const int64_t gw = (int64_t)blockIdx.x * wpb + threadIdx.x / 32;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  for (int64_t b = gw; b < batch; b += nw) {
    double x[MAXE];
    load_col_r<MAXE>(A + b * strideA, m, lane, x);
    const double t = make_reflector_r<MAXE>(x, 0, lane);
    store_col_r<MAXE>(A + b * strideA, m, lane, x);
    if (lane == 0) tau[b * n] = t;
  }
  for (int j = 0; j < n - 1; ++j) {
    if (!grid_barrier(s)) return;
    const int64_t ncols = n - j - 1;
    const int64_t tasks = (int64_t)batch * ncols;
    for (int64_t t = gw; t < tasks; t += nw) {
      const int64_t b = t / ncols;
      const int c = j + 1 + (int)(t % ncols);
      double* Ab = A + b * strideA;
      double x[MAXE], v[MAXE];
      load_col_r<MAXE>(Ab + (int64_t)c * m, m, lane, x);
      load_col_r<MAXE>(Ab + (int64_t)j * m, m, lane, v);
      const double tj = __ldcg(tau + b * n + j);
      if (tj != 0.0) reflect_r<MAXE>(x, v, tj, j, lane);
      if (c == j + 1) {
        const double tn = make_reflector_r<MAXE>(x, j + 1, lane);
        if (lane == 0) tau[b * n + j + 1] = tn;
      }
      store_col_r<MAXE>(Ab + (int64_t)c * m, m, lane, x);
    }
  }
}

// X := Q X with the column of X in registers through all n reflectors.
template <int MAXE>
__global__ void apply_q_cols_kernel_r(const double* A, const double* tau, double* X, int batch, int m, int n, int k,
                                      int64_t strideA, int64_t strideX) {
  const int lane = threadIdx.x % 32;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t tasks = (int64_t)batch * k;
  for (int64_t t = gw; t < tasks; t += nw) {
    const int64_t b = t / k;
    const int c = (int)(t % k);
    double* xc = X + b * strideX + (int64_t)c * m;
    double x[MAXE];
    load_col_r<MAXE>(xc, m, lane, x);
    for (int j = n - 1; j >= 0; --j) {
      const double tj = __ldg(tau + b * n + j);
      if (tj == 0.0) continue;
      double v[MAXE];
      load_col_r<MAXE>(A + b * strideA + (int64_t)j * m, m, lane, v);
      reflect_r<MAXE>(x, v, tj, j, lane);
    }
    store_col_r<MAXE>(xc, m, lane, x);
  }
}

// FP32 copy of a batch of r x r matrices scaled to unit Frobenius norm, and an FP32 identity.
__global__ void to_f32_unit_kernel(const double* W, float* W32, float* V32, int r, const double* frob2) {
  const int b = blockIdx.y;
  const int64_t rr = (int64_t)r * r;
  const double sc = 1.0 / sqrt(frob2[b]);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rr; e += (int64_t)gridDim.x * blockDim.x) {
    W32[b * rr + e] = (float)(W[b * rr + e] * sc);
    V32[b * rr + e] = (e / r == e % r) ? 1.0f : 0.0f;
  }
}

__global__ void f32_to_f64_kernel(const float* x, double* y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (double)x[e];
}

__global__ void fill_kernel(double* x, int64_t n, double v) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) x[e] = v;
}

__global__ void extract_r_kernel(const double* A, double* R, int m, int n, int64_t strideA) {
  const int b = blockIdx.y;
  int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / n), c = (int)(e % n);
    R[(int64_t)b * total + e] = (c >= i) ? A[(int64_t)b * strideA + (int64_t)c * m + i] : 0.0;
  }
}

// ------------------------------------------------------------------ one-sided Jacobi
__device__ __forceinline__ void rr_pair(int round, int k, int rp, int& p, int& q) {
  const int n1 = rp - 1;
  if (k == 0) {
    p = round;
    q = n1;
  } else {
    p = (round + k) % n1;
    q = (round - k + n1) % n1;
  }
}

// One-sided Jacobi in a block-cyclic order.  The columns form G groups of 4; a sweep is G - 1 outer
// rounds in which every block holds a pair of groups (a, b) of one matrix -- its 8 columns of W and
// V staged in shared memory -- and rotates the 16 cross pairs (a_i, b_j) in 4 inner rounds of 4
// disjoint pairs (a warp each, separated by __syncthreads); the first outer round also rotates the
// 12 pairs inside a and b.  Every column pair is rotated once per sweep, as in the cyclic order,
// but only G - 1 grid barriers separate the outer rounds instead of r - 1.  Requires m = r and
// r <= 32 * MAXE.  Convergence bookkeeping as in jacobi_warp_kernel.
template <typename T, int MAXE>
__global__ void __launch_bounds__(128) jacobi_block_kernel(T* W, T* V, int batch, int r, int G, int max_sweeps,
                                                            double tol, int* flags, int* conv, int* sweeps_out,
                                                            const double* frob2, double* flop_acc, Sync s,
                                                            int report_noconv) {
  extern __shared__ unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);  // [8][r]
  T* sV = sW + 8 * r;                      // [8][r]
  const int t = threadIdx.x, lane = t % 32, wid = t / 32;
  const int half = G / 2;
  const int64_t tasks = (int64_t)batch * half;
  const int64_t rr = (int64_t)r * r;
  double my_flops = 0.0;
  int sweep = 0;
  __shared__ int any_rot;
  for (; sweep < max_sweeps; ++sweep) {
    int* fl = flags + (sweep % 3) * batch;
    if (blockIdx.x == 0) {
      int* nxt = flags + ((sweep + 1) % 3) * batch;
      for (int b = t; b < batch; b += blockDim.x) nxt[b] = 0;
      __threadfence();
    }
    for (int k = 0; k < G - 1; ++k) {
      for (int64_t task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int b = (int)(task / half);
        const int j = (int)(task % half);
        if (__ldcg(conv + b)) continue;  // uniform over the block
        const int ga = circle_group(k, j, G), gb = circle_group(k, G - 1 - j, G);
        T* Wb = W + b * rr;
        T* Vb = V + b * rr;
        // stage the 8 columns: a_0..a_3 in slots 0..3, b_0..b_3 in slots 4..7 (two per warp)
        for (int c = wid; c < 8; c += 4) {
          const int col = (c < 4 ? ga * 4 + c : gb * 4 + c - 4);
          for (int i = lane; i < r; i += 32) {
            sW[c * r + i] = col < r ? __ldcg(Wb + (int64_t)col * r + i) : T(0);
            sV[c * r + i] = col < r ? __ldcg(Vb + (int64_t)col * r + i) : T(0);
          }
        }
        if (t == 0) any_rot = 0;
        __syncthreads();
        const T floor2 = (T)(1e-32 * __ldcg(frob2 + b));
        const int n_inner = block_inner_rounds(k);
        for (int it = 0; it < n_inner; ++it) {
          int p, q;
          block_pair(k, it, wid, p, q);  // slots of this warp's pair (jacobi_order.h)
          T x[MAXE], y[MAXE], u[MAXE], w[MAXE];
#pragma unroll
          for (int e = 0; e < MAXE; ++e) {
            const int i = lane + 32 * e;
            x[e] = i < r ? sW[p * r + i] : T(0);
            y[e] = i < r ? sW[q * r + i] : T(0);
            u[e] = i < r ? sV[p * r + i] : T(0);
            w[e] = i < r ? sV[q * r + i] : T(0);
          }
          T al = 0, be = 0, ga_ = 0;
#pragma unroll
          for (int e = 0; e < MAXE; ++e) {
            al = fma(x[e], x[e], al);
            be = fma(y[e], y[e], be);
            ga_ = fma(x[e], y[e], ga_);
          }
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            ga_ += __shfl_xor_sync(0xffffffffu, ga_, o);
          }
          if (lane == 0) my_flops += 6.0 * r;
          if (al > floor2 && be > floor2 && fabs(ga_) > (T)tol * sqrt(al) * sqrt(be)) {
            if (lane == 0) my_flops += 12.0 * r;
            const T zeta = (be - al) / (T(2) * ga_);
            T tt;
            if (fabs(zeta) > (sizeof(T) == 8 ? T(1e150) : T(1e18)))
              tt = T(0.5) / zeta;
            else
              tt = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
            const T c = T(1) / sqrt(T(1) + tt * tt);
            const T sn = c * tt;
#pragma unroll
            for (int e = 0; e < MAXE; ++e) {
              const int i = lane + 32 * e;
              if (i < r) {
                sW[p * r + i] = c * x[e] - sn * y[e];
                sW[q * r + i] = sn * x[e] + c * y[e];
                sV[p * r + i] = c * u[e] - sn * w[e];
                sV[q * r + i] = sn * u[e] + c * w[e];
              }
            }
            if (lane == 0) any_rot = 1;
          }
          __syncthreads();
        }
        // write the 8 columns back
        for (int c = wid; c < 8; c += 4) {
          const int col = (c < 4 ? ga * 4 + c : gb * 4 + c - 4);
          if (col < r)
            for (int i = lane; i < r; i += 32) {
              Wb[(int64_t)col * r + i] = sW[c * r + i];
              Vb[(int64_t)col * r + i] = sV[c * r + i];
            }
        }
        if (t == 0 && any_rot) fl[b] = 1;
        __syncthreads();
      }
      if (!grid_barrier(s)) {
        if (lane == 0) atomicAdd(flop_acc, my_flops);
        return;
      }
    }
    int all = 1;
    {
      volatile int* vf = fl;
      volatile int* vc = conv;
      for (int b = 0; b < batch; ++b)
        if (!vc[b] && vf[b] != 0) all = 0;
    }
    if (!grid_barrier(s)) {
      if (lane == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (blockIdx.x == 0 && t == 0) {
      volatile int* vf = fl;
      for (int b = 0; b < batch; ++b)
        if (vf[b] == 0) conv[b] = 1;
      __threadfence();
    }
    if (!grid_barrier(s)) {
      if (lane == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (all) {
      ++sweep;
      break;
    }
  }
  if (lane == 0) atomicAdd(flop_acc, my_flops);
  if (blockIdx.x == 0 && t == 0) {
    atomicAdd(sweeps_out, sweep);
    if (report_noconv)
      for (int b = 0; b < batch; ++b)
        if (!conv[b]) atomicOr(s.status, DEV_SVD_NOCONV);
  }
}

// Squared Frobenius norm of each matrix (deterministic, one block per matrix).
__global__ void frob2_kernel(const double* W, int64_t rr, double* out) {
  __shared__ double sh[256];
  const double* Wb = W + blockIdx.x * rr;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < rr; e += blockDim.x) acc = fma(Wb[e], Wb[e], acc);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// Cyclic one-sided Jacobi sweeps (round-robin pairing, a grid barrier per round).  A pair is rotated
// when |g| > tol sqrt(a) sqrt(b) (products of square roots cannot underflow) and both columns lie
// above the rounding floor 1e-32 ||M||_F^2: below it a column is noise whose direction no further
// rotation can settle, and its singular value is a numerical zero.
// One 128-thread block per column pair: every thread holds MAXE rows of the
// two columns of W and of V in registers (loads issued together), the three dot products are
// reduced across the block, and the rotation is applied in registers before the stores.
// Requires max(m, r) <= 128 * MAXE.  The rotation test and the rotation itself (square roots and
// divisions, software sequences in FP64) are computed once per pair by thread 0 and broadcast.
// W holds r columns of length m per matrix (column-major, stride m*r), V r columns of length r.
template <int MAXE>
__global__ void __launch_bounds__(128) jacobi_team_kernel(double* W, double* V, int batch, int m, int r, int rp,
                                                           int max_sweeps, double tol, int* flags, int* conv,
                                                           int* sweeps_out, const double* frob2, double* flop_acc,
                                                           Sync s) {
  __shared__ double red[3][4];
  __shared__ double rot[3];  // rotate?, c, s
  const int t = threadIdx.x, lane = t % 32, warp = t / 32;
  const int npairs = rp / 2;
  const int64_t tasks = (int64_t)batch * npairs;
  const int64_t mr = (int64_t)m * r, rr = (int64_t)r * r;
  double my_flops = 0.0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int* fl = flags + (sweep % 3) * batch;
    if (blockIdx.x == 0) {
      int* nxt = flags + ((sweep + 1) % 3) * batch;
      for (int b = t; b < batch; b += blockDim.x) nxt[b] = 0;
      __threadfence();
    }
    for (int round = 0; round < rp - 1; ++round) {
      for (int64_t task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int b = (int)(task / npairs);
        if (__ldcg(conv + b)) continue;
        int p, q;
        rr_pair(round, (int)(task % npairs), rp, p, q);
        if (p >= r || q >= r) continue;
        double* ap = W + b * mr + (int64_t)p * m;
        double* aq = W + b * mr + (int64_t)q * m;
        double* vp = V + b * rr + (int64_t)p * r;
        double* vq = V + b * rr + (int64_t)q * r;
        double x[MAXE], y[MAXE], u[MAXE], w[MAXE];
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
          const int i = t + 128 * e;
          x[e] = i < m ? __ldcg(ap + i) : 0.0;
          y[e] = i < m ? __ldcg(aq + i) : 0.0;
          u[e] = i < r ? __ldcg(vp + i) : 0.0;
          w[e] = i < r ? __ldcg(vq + i) : 0.0;
        }
        double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
          al = fma(x[e], x[e], al);
          be = fma(y[e], y[e], be);
          ga = fma(x[e], y[e], ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (lane == 0) {
          red[0][warp] = al;
          red[1][warp] = be;
          red[2][warp] = ga;
        }
        __syncthreads();
        if (t == 0) {
          al = red[0][0] + red[0][1] + red[0][2] + red[0][3];
          be = red[1][0] + red[1][1] + red[1][2] + red[1][3];
          ga = red[2][0] + red[2][1] + red[2][2] + red[2][3];
          const double f2 = __ldcg(frob2 + b);
          const double floor2 = 1e-32 * f2;
          my_flops += 6.0 * m;
          double go = 0.0, c = 1.0, sn = 0.0;
          if (al > floor2 && be > floor2 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
            my_flops += 6.0 * m + 6.0 * r;
            const double zeta = (be - al) / (2.0 * ga);
            double tt;
            if (fabs(zeta) > 1e150)
              tt = 0.5 / zeta;
            else
              tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            c = 1.0 / sqrt(1.0 + tt * tt);
            sn = c * tt;
            go = 1.0;
            fl[b] = 1;
          }
          rot[0] = go;
          rot[1] = c;
          rot[2] = sn;
        }
        __syncthreads();
        if (rot[0] != 0.0) {
          const double c = rot[1], sn = rot[2];
#pragma unroll
          for (int e = 0; e < MAXE; ++e) {
            const int i = t + 128 * e;
            if (i < m) {
              ap[i] = c * x[e] - sn * y[e];
              aq[i] = sn * x[e] + c * y[e];
            }
            if (i < r) {
              vp[i] = c * u[e] - sn * w[e];
              vq[i] = sn * u[e] + c * w[e];
            }
          }
        }
      }
      if (!grid_barrier(s)) {
        if (t == 0) atomicAdd(flop_acc, my_flops);
        return;
      }
    }
    int all = 1;
    {
      volatile int* vf = fl;
      volatile int* vc = conv;
      for (int b = 0; b < batch; ++b)
        if (!vc[b] && vf[b] != 0) all = 0;
    }
    if (!grid_barrier(s)) {
      if (t == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (blockIdx.x == 0 && t == 0) {
      volatile int* vf = fl;
      for (int b = 0; b < batch; ++b)
        if (vf[b] == 0) conv[b] = 1;
      __threadfence();
    }
    if (!grid_barrier(s)) {
      if (t == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (all) {
      ++sweep;
      break;
    }
  }
  if (t == 0) atomicAdd(flop_acc, my_flops);
  if (blockIdx.x == 0 && t == 0) {
    atomicAdd(sweeps_out, sweep);
    for (int b = 0; b < batch; ++b)
      if (!conv[b]) atomicOr(s.status, DEV_SVD_NOCONV);
  }
}

// The same sweeps with one warp per column pair (four pairs per 128-thread block): the three dot
// products are reduced with warp shuffles only, every lane derives the rotation from the same
// sums, and no block-wide synchronisation separates the load, the test and the rotation.  A round
// is then bound by the FP64 pipes of the SMs rather than by block barriers, and a quarter as many
// blocks meet at each grid barrier.  Requires max(m, r) <= 32 * MAXE.
template <typename T, int MAXE>
__global__ void __launch_bounds__(128) jacobi_warp_kernel(T* W, T* V, int batch, int m, int r, int rp,
                                                           int max_sweeps, double tol, int* flags, int* conv,
                                                           int* sweeps_out, const double* frob2, double* flop_acc,
                                                           Sync s, int report_noconv) {
  const int t = threadIdx.x, lane = t % 32;
  const int wpb = blockDim.x / 32;
  const int64_t gw = (int64_t)blockIdx.x * wpb + t / 32;
  const int64_t nw = (int64_t)gridDim.x * wpb;
  const int npairs = rp / 2;
  const int64_t tasks = (int64_t)batch * npairs;
  const int64_t mr = (int64_t)m * r, rr = (int64_t)r * r;
  double my_flops = 0.0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int* fl = flags + (sweep % 3) * batch;
    if (blockIdx.x == 0) {
      int* nxt = flags + ((sweep + 1) % 3) * batch;
      for (int b = t; b < batch; b += blockDim.x) nxt[b] = 0;
      __threadfence();
    }
    for (int round = 0; round < rp - 1; ++round) {
      for (int64_t task = gw; task < tasks; task += nw) {
        const int b = (int)(task / npairs);
        if (__ldcg(conv + b)) continue;
        int p, q;
        rr_pair(round, (int)(task % npairs), rp, p, q);
        if (p >= r || q >= r) continue;
        T* ap = W + b * mr + (int64_t)p * m;
        T* aq = W + b * mr + (int64_t)q * m;
        T* vp = V + b * rr + (int64_t)p * r;
        T* vq = V + b * rr + (int64_t)q * r;
        T x[MAXE], y[MAXE], u[MAXE], w[MAXE];
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
          const int i = lane + 32 * e;
          x[e] = i < m ? __ldcg(ap + i) : T(0);
          y[e] = i < m ? __ldcg(aq + i) : T(0);
          u[e] = i < r ? __ldcg(vp + i) : T(0);
          w[e] = i < r ? __ldcg(vq + i) : T(0);
        }
        T al = 0, be = 0, ga = 0;
#pragma unroll
        for (int e = 0; e < MAXE; ++e) {
          al = fma(x[e], x[e], al);
          be = fma(y[e], y[e], be);
          ga = fma(x[e], y[e], ga);
        }
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        const T floor2 = (T)(1e-32 * __ldcg(frob2 + b));
        if (lane == 0) my_flops += 6.0 * m;
        if (al > floor2 && be > floor2 && fabs(ga) > (T)tol * sqrt(al) * sqrt(be)) {
          if (lane == 0) my_flops += 6.0 * m + 6.0 * r;
          const T zeta = (be - al) / (T(2) * ga);
          T tt;
          if (fabs(zeta) > (sizeof(T) == 8 ? T(1e150) : T(1e18)))
            tt = T(0.5) / zeta;
          else
            tt = copysign(T(1), zeta) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + tt * tt);
          const T sn = c * tt;
#pragma unroll
          for (int e = 0; e < MAXE; ++e) {
            const int i = lane + 32 * e;
            if (i < m) {
              ap[i] = c * x[e] - sn * y[e];
              aq[i] = sn * x[e] + c * y[e];
            }
            if (i < r) {
              vp[i] = c * u[e] - sn * w[e];
              vq[i] = sn * u[e] + c * w[e];
            }
          }
          if (lane == 0) fl[b] = 1;
        }
        __syncwarp();
      }
      if (!grid_barrier(s)) {
        if (lane == 0) atomicAdd(flop_acc, my_flops);
        return;
      }
    }
    int all = 1;
    {
      volatile int* vf = fl;
      volatile int* vc = conv;
      for (int b = 0; b < batch; ++b)
        if (!vc[b] && vf[b] != 0) all = 0;
    }
    if (!grid_barrier(s)) {
      if (lane == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (blockIdx.x == 0 && t == 0) {
      volatile int* vf = fl;
      for (int b = 0; b < batch; ++b)
        if (vf[b] == 0) conv[b] = 1;
      __threadfence();
    }
    if (!grid_barrier(s)) {
      if (lane == 0) atomicAdd(flop_acc, my_flops);
      return;
    }
    if (all) {
      ++sweep;
      break;
    }
  }
  if (lane == 0) atomicAdd(flop_acc, my_flops);
  if (blockIdx.x == 0 && t == 0) {
    atomicAdd(sweeps_out, sweep);
    if (report_noconv)
      for (int b = 0; b < batch; ++b)
        if (!conv[b]) atomicOr(s.status, DEV_SVD_NOCONV);
  }
}

// Launch the Jacobi sweeps (cooperative) with the register-resident team kernel.
void launch_jacobi(double* W, double* V, int batch, int m, int r, int max_sweeps, int* flags, int* conv,
                   int* sweeps_out, double* frob2, double* facc, const Sync& sy, cudaStream_t st);

// Column norms, descending order, normalised left vectors.  One block per matrix.
__global__ void svd_finalize_kernel(const double* W, const double* V, double* lam, double* Uo, double* Vo, int r,
                                    int* status) {
  extern __shared__ double sm[];
  double* nrm = sm;              // r
  int* rank = (int*)(sm + r);    // r
  const int b = blockIdx.x;
  const int64_t rr = (int64_t)r * r;
  const double* Wb = W + b * rr;
  const double* Vb = V + b * rr;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
  for (int k = warp; k < r; k += nwarp) {
    double s = 0.0;
    for (int i = lane; i < r; i += 32) s = fma(Wb[(int64_t)k * r + i], Wb[(int64_t)k * r + i], s);
    s = warp_sum(s);
    if (lane == 0) {
      nrm[k] = sqrt(s);
      if (!isfinite(s)) atomicOr(status, DEV_NONFINITE);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    int rk = 0;
    double v = nrm[k];
    for (int j = 0; j < r; ++j) rk += (nrm[j] > v) || (nrm[j] == v && j < k);
    rank[k] = rk;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x) lam[(int64_t)b * r + rank[k]] = nrm[k];
  for (int64_t e = threadIdx.x; e < rr; e += blockDim.x) {
    int k = (int)(e / r), i = (int)(e % r);  // column k, row i
    double inv = nrm[k] > 0.0 ? 1.0 / nrm[k] : 0.0;
    Uo[b * rr + (int64_t)i * r + rank[k]] = Wb[e] * inv;
    Vo[b * rr + (int64_t)i * r + rank[k]] = Vb[e];
  }
}

// Finalize of the Jacobi SVD of B^t (m x l, column-major W; V l x l column-major), where
// B = V W^t.  Sorted descending: lam[rank], Vm (m x ldv row-major, first l columns) = W_k / lam_k,
// Ul (l x l row-major) = V's column k; flags[b] = 1 when the smallest value is not below
// 1e-14 lam_max (the sketch may have missed directions); rank_out[b] = number of values above
// 1e-14 lam_max.
__global__ void svd_rect_finalize_kernel(const double* W, const double* V, double* lam, int64_t lam_stride, double* Vm,
                                         int64_t ldv, double* Ul, int m, int l, int* incomplete, int* rank_out,
                                         int* status) {
  extern __shared__ double sm[];
  double* nrm = sm;
  int* rank = (int*)(sm + l);
  const int b = blockIdx.x;
  const double* Wb = W + (int64_t)b * m * l;
  const double* Vb = V + (int64_t)b * l * l;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nwarp = blockDim.x / 32;
  for (int k = warp; k < l; k += nwarp) {
    double s2 = 0.0;
    for (int i = lane; i < m; i += 32) s2 = fma(Wb[(int64_t)k * m + i], Wb[(int64_t)k * m + i], s2);
    s2 = warp_sum(s2);
    if (lane == 0) {
      nrm[k] = sqrt(s2);
      if (!isfinite(s2)) atomicOr(status, DEV_NONFINITE);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < l; k += blockDim.x) {
    int rk = 0;
    double v = nrm[k];
    for (int j = 0; j < l; ++j) rk += (nrm[j] > v) || (nrm[j] == v && j < k);
    rank[k] = rk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double mx = 0.0, mn = 1e308;
    for (int k = 0; k < l; ++k) {
      mx = fmax(mx, nrm[k]);
      mn = fmin(mn, nrm[k]);
    }
    incomplete[b] = (mn > 1e-14 * mx) ? 1 : 0;
    int nk = 0;
    for (int k = 0; k < l; ++k) nk += nrm[k] > 1e-14 * mx;
    rank_out[b] = nk;
  }
  for (int k = threadIdx.x; k < l; k += blockDim.x) lam[(int64_t)b * lam_stride + rank[k]] = nrm[k];
  for (int64_t e = threadIdx.x; e < (int64_t)m * l; e += blockDim.x) {
    int k = (int)(e / m), i = (int)(e % m);
    double inv = nrm[k] > 0.0 ? 1.0 / nrm[k] : 0.0;
    Vm[(int64_t)b * m * ldv + (int64_t)i * ldv + rank[k]] = Wb[e] * inv;
  }
  for (int64_t e = threadIdx.x; e < (int64_t)l * l; e += blockDim.x) {
    int k = (int)(e / l), j = (int)(e % l);
    Ul[(int64_t)b * l * l + (int64_t)j * l + rank[k]] = Vb[e];
  }
}

// Deterministic test matrix: splitmix64 of the element index, mapped to (-1, 1).
__global__ void sketch_omega_kernel(double* O, int64_t n, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)e * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    O[e] = ((double)(z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
  }
}

// X (r x l column-major) = [I_l; 0]
__global__ void eye_rect_kernel(double* X, int r, int l) {
  const int b = blockIdx.y;
  int64_t n = (int64_t)r * l;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    X[b * n + e] = ((e / r) == (e % r)) ? 1.0 : 0.0;
}

__global__ void identity_kernel(double* V, int r) {
  const int b = blockIdx.y;
  int64_t rr = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rr; e += (int64_t)gridDim.x * blockDim.x)
    V[b * rr + e] = (e / r == e % r) ? 1.0 : 0.0;
}

// Per-device scratch for the barriers and flags of the cooperative kernels.
struct CoopScratch {
  unsigned* bar = nullptr;
  int* abort = nullptr;
  int* flags = nullptr;
  int* conv = nullptr;
  double* frob2 = nullptr;
  int flags_cap = 0;
  double* flop_acc = nullptr;
};

// One set per (device, stream) and host thread: cooperative kernels enqueued on different streams
// may run at the same time and must not share barrier words.
CoopScratch& coop_of(cudaStream_t st) {
  static thread_local std::map<std::pair<int, cudaStream_t>, CoopScratch> m;
  int dev = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  return m[{dev, st}];
}

CoopScratch& ensure_coop(int batch, cudaStream_t st) {
  CoopScratch& g_coop = coop_of(st);
  if (!g_coop.bar) {
    CTM_CUDA(cudaMalloc(&g_coop.bar, 2 * sizeof(unsigned)));
    CTM_CUDA(cudaMalloc(&g_coop.abort, sizeof(int)));
    CTM_CUDA(cudaMalloc(&g_coop.flop_acc, sizeof(double)));
    CTM_CUDA(cudaMemset(g_coop.flop_acc, 0, sizeof(double)));
  }
  if (g_coop.flags_cap < batch) {
    if (g_coop.flags) {
      CTM_CUDA(cudaFree(g_coop.flags));
      CTM_CUDA(cudaFree(g_coop.conv));
      CTM_CUDA(cudaFree(g_coop.frob2));
    }
    g_coop.flags_cap = std::max(batch, 64);
    CTM_CUDA(cudaMalloc(&g_coop.flags, 3 * g_coop.flags_cap * sizeof(int)));
    CTM_CUDA(cudaMalloc(&g_coop.conv, g_coop.flags_cap * sizeof(int)));
    CTM_CUDA(cudaMalloc(&g_coop.frob2, g_coop.flags_cap * sizeof(double)));
  }
  CTM_CUDA(cudaMemsetAsync(g_coop.bar, 0, 2 * sizeof(unsigned), st));
  CTM_CUDA(cudaMemsetAsync(g_coop.abort, 0, sizeof(int), st));
  return g_coop;
}

int coop_grid(const void* kernel, int threads) {
  int dev = 0, sms = 0, per_sm = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  CTM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0));
  CTM_CHECK(per_sm > 0, CTM_ERR_CUDA, "cooperative kernel cannot be resident");
  return sms * per_sm;
}

// Block-ordered Jacobi (m = r): G = ceil(r / 8) * 2 groups of 4 columns, batch * G / 2 blocks.
template <typename T, int MAXE>
void launch_jacobi_b(T* W, T* V, int batch, int r, int max_sweeps, double tol, int* flags, int* conv,
                     int* sweeps_out, const double* frob2, double* facc, const Sync& sy, int report, cudaStream_t st) {
  const int threads = 128;
  const int G = ((r + 7) / 8) * 2;
  const size_t smem = sizeof(T) * 16 * (size_t)r;
  const void* fn = (const void*)jacobi_block_kernel<T, MAXE>;
  int dev = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count({fn, dev})) {
      CTM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
      done.insert({fn, dev});
    }
  }
  int sms = 0, per_sm = 0;
  CTM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CTM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  CTM_CHECK(per_sm > 0, CTM_ERR_CUDA, "cooperative kernel cannot be resident");
  int64_t need = (int64_t)batch * (G / 2);
  int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, need));
  Sync s = sy;
  int Gv = G;
  void* args[] = {&W, &V, &batch, &r, &Gv, &max_sweeps, &tol, &flags, &conv, &sweeps_out, &frob2, &facc, &s,
                  &report};
  CTM_CUDA(cudaLaunchCooperativeKernel(fn, grid, threads, args, smem, st));
  CTM_LAUNCHED();
}

template <int MAXE>
void launch_jacobi_t(double* W, double* V, int batch, int m, int r, int max_sweeps, int* flags, int* conv,
                     int* sweeps_out, double* frob2, double* facc, const Sync& sy, cudaStream_t st) {
  const int threads = 128;
  int rp = r + (r & 1);
  int grid = coop_grid((const void*)jacobi_team_kernel<MAXE>, threads);
  int64_t need = (int64_t)batch * (rp / 2);
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  double tol = 2.220446049250313e-16 * std::max(m, r);
  Sync s = sy;
  void* args[] = {&W, &V, &batch, &m, &r, &rp, &max_sweeps, &tol, &flags, &conv, &sweeps_out, &frob2, &facc, &s};
  CTM_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_team_kernel<MAXE>, grid, threads, args, 0, st));
  CTM_LAUNCHED();
}

template <typename T, int MAXE>
void launch_jacobi_w(T* W, T* V, int batch, int m, int r, int max_sweeps, double tol, int* flags, int* conv,
                     int* sweeps_out, const double* frob2, double* facc, const Sync& sy, int report, cudaStream_t st) {
  const int threads = 128;
  int rp = r + (r & 1);
  int grid = coop_grid((const void*)jacobi_warp_kernel<T, MAXE>, threads);
  int64_t need = ((int64_t)batch * (rp / 2) + 3) / 4;
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  Sync s = sy;
  void* args[] = {&W, &V, &batch, &m, &r, &rp, &max_sweeps, &tol, &flags, &conv, &sweeps_out, &frob2, &facc, &s,
                  &report};
  CTM_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_warp_kernel<T, MAXE>, grid, threads, args, 0, st));
  CTM_LAUNCHED();
}

void launch_jacobi(double* W, double* V, int batch, int m, int r, int max_sweeps, int* flags, int* conv,
                   int* sweeps_out, double* frob2, double* facc, const Sync& sy, cudaStream_t st) {
  const int e = std::max(m, r);
  CTM_CHECK(e <= 128 * 16, CTM_ERR_INVALID_ARG, "Jacobi SVD: size too large");
  // warp-per-pair kernel for columns up to 384 long (12 doubles per lane and column in registers)
  const double tol = 2.220446049250313e-16 * std::max(m, r);
  if (e <= 128) {
    launch_jacobi_w<double, 4>(W, V, batch, m, r, max_sweeps, tol, flags, conv, sweeps_out, frob2, facc, sy, 1, st);
    return;
  }
  if (e <= 256) {
    launch_jacobi_w<double, 8>(W, V, batch, m, r, max_sweeps, tol, flags, conv, sweeps_out, frob2, facc, sy, 1, st);
    return;
  }
  if (e <= 384) {
    launch_jacobi_w<double, 12>(W, V, batch, m, r, max_sweeps, tol, flags, conv, sweeps_out, frob2, facc, sy, 1, st);
    return;
  }
  if (e <= 256) launch_jacobi_t<2>(W, V, batch, m, r, max_sweeps, flags, conv, sweeps_out, frob2, facc, sy, st);
  else if (e <= 512) launch_jacobi_t<4>(W, V, batch, m, r, max_sweeps, flags, conv, sweeps_out, frob2, facc, sy, st);
  else if (e <= 768) launch_jacobi_t<6>(W, V, batch, m, r, max_sweeps, flags, conv, sweeps_out, frob2, facc, sy, st);
  else if (e <= 1024) launch_jacobi_t<8>(W, V, batch, m, r, max_sweeps, flags, conv, sweeps_out, frob2, facc, sy, st);
  else launch_jacobi_t<16>(W, V, batch, m, r, max_sweeps, flags, conv, sweeps_out, frob2, facc, sy, st);
}

}  // namespace

namespace {
template <int MAXE>
void launch_qr_r(double* A, double* tau, int batch, int m, int n, int64_t strideA, const Sync& sy, cudaStream_t st) {
  const int threads = 256;
  int grid = coop_grid((const void*)qr_kernel_r<MAXE>, threads);
  int64_t need = ((int64_t)batch * n + threads / 32 - 1) / (threads / 32);
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  Sync s = sy;
  void* args[] = {&A, &tau, &batch, &m, &n, &strideA, &s};
  CTM_CUDA(cudaLaunchCooperativeKernel((const void*)qr_kernel_r<MAXE>, grid, threads, args, 0, st));
  CTM_LAUNCHED();
}

template <int MAXE>
void launch_apply_q_r(const double* A, const double* tau, double* X, int batch, int m, int n, int k, int64_t strideA,
                      int64_t strideX, cudaStream_t st) {
  const int threads = 128;
  const int64_t need = ((int64_t)batch * k + threads / 32 - 1) / (threads / 32);
  apply_q_cols_kernel_r<MAXE><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(need, 65535)), threads, 0, st>>>(
      A, tau, X, batch, m, n, k, strideA, strideX);
  CTM_LAUNCHED();
}
}  // namespace

void qr_householder(double* A, double* tau, int batch, int m, int n, int64_t strideA, int* status, cudaStream_t st) {
  if (batch == 0 || n == 0) return;
  ProfScope ps(PROF_QR, st, batch * (2.0 * m * n * n - 2.0 * n * n * n / 3.0), 8.0 * batch * m * n * 2,
               prof_tag("qr", batch, m, n, 0));
  CoopScratch& g_coop = ensure_coop(batch, st);
  Sync s{g_coop.bar, g_coop.abort, status, (long long)lim_spins()};
  // columns of up to 768 rows stay in registers (4 .. 24 doubles per lane)
  if (m <= 128) return launch_qr_r<4>(A, tau, batch, m, n, strideA, s, st);
  if (m <= 256) return launch_qr_r<8>(A, tau, batch, m, n, strideA, s, st);
  if (m <= 384) return launch_qr_r<12>(A, tau, batch, m, n, strideA, s, st);
  if (m <= 512) return launch_qr_r<16>(A, tau, batch, m, n, strideA, s, st);
  if (m <= 768) return launch_qr_r<24>(A, tau, batch, m, n, strideA, s, st);
  const int threads = 256;
  int grid = coop_grid((const void*)qr_kernel, threads);
  int64_t need = ((int64_t)batch * n + threads / 32 - 1) / (threads / 32);
  grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, need));
  void* args[] = {&A, &tau, &batch, &m, &n, &strideA, &s};
  CTM_CUDA(cudaLaunchCooperativeKernel((const void*)qr_kernel, grid, threads, args, 0, st));
  CTM_LAUNCHED();
}

void qr_extract_R(const double* A, double* R, int batch, int m, int n, int64_t strideA, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>(4096, ((int64_t)n * n + 255) / 256), batch);
  extract_r_kernel<<<grid, 256, 0, st>>>(A, R, m, n, strideA);
  CTM_LAUNCHED();
}

void qr_apply_Q(const double* A, const double* tau, double* X, int batch, int m, int n, int k, int64_t strideA,
                int64_t strideX, int* status, cudaStream_t st) {
  if (batch == 0 || n == 0) return;
  ProfScope ps(PROF_QR, st, batch * 4.0 * m * n * k - 2.0 * batch * n * n * k, 8.0 * batch * (m * n + 2.0 * m * k),
               prof_tag("apply_q", batch, m, n, k));
  (void)status;
  if (m <= 128) return launch_apply_q_r<4>(A, tau, X, batch, m, n, k, strideA, strideX, st);
  if (m <= 256) return launch_apply_q_r<8>(A, tau, X, batch, m, n, k, strideA, strideX, st);
  if (m <= 384) return launch_apply_q_r<12>(A, tau, X, batch, m, n, k, strideA, strideX, st);
  if (m <= 512) return launch_apply_q_r<16>(A, tau, X, batch, m, n, k, strideA, strideX, st);
  if (m <= 768) return launch_apply_q_r<24>(A, tau, X, batch, m, n, k, strideA, strideX, st);
  const int threads = 128;
  const int64_t need = ((int64_t)batch * k + threads / 32 - 1) / (threads / 32);
  apply_q_cols_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(need, 65535)), threads, 0, st>>>(
      A, tau, X, batch, m, n, k, strideA, strideX);
  CTM_LAUNCHED();
}

// Test matrix of the sketches: element e is splitmix64(seed + e * golden) mapped to (-1, 1),
// so a longer buffer extends a shorter one and every shape reads the same leading values.
static const double* sketch_omega(int64_t n, cudaStream_t st) {
  struct Buf {
    double* p = nullptr;
    int64_t n = 0;
  };
  static thread_local std::map<int, Buf> per_dev;
  int dev = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  double*& omega = per_dev[dev].p;
  int64_t& omega_n = per_dev[dev].n;
  if (omega_n < n) {
    if (omega) CTM_CUDA(cudaFree(omega));
    CTM_CUDA(cudaMalloc(&omega, sizeof(double) * n));
    omega_n = n;
    sketch_omega_kernel<<<256, 256, 0, st>>>(omega, n, 0x2512144140ull);
    CTM_LAUNCHED();
  }
  return omega;
}

size_t svd_sketch_product_ws(int batch, int nr, int nl, int l) {
  const size_t per = (size_t)2 * nl * l + (size_t)3 * nr * l + (size_t)2 * l * l + l;
  return sizeof(double) * batch * per + sizeof(int) * 2 * batch + 256;
}

void svd_sketch_product(const double* const* N, const double* const* S, const int* nrs, const int* nls, int batch,
                        int l, const double* const* warm, int ldw, int kw, double* ws, double* lam, double* Uo,
                        double* Vo, int* status, int* sweeps_out, std::vector<int>& incomplete_host,
                        std::vector<int>& rank_host, cudaStream_t st) {
  // Matrices of different n_r share one batch: every n_r-long object is stored with the batch's
  // largest n_r and zero rows below its own; zero rows change neither the Householder QR nor
  // the one-sided Jacobi rotations, and they come out as zero rows of U and V.
  int nr = 0, nl = 0;
  for (int b = 0; b < batch; ++b) nr = std::max(nr, nrs[b]), nl = std::max(nl, nls[b]);
  const int64_t Ln = (int64_t)nl * l, Lr = (int64_t)nr * l, ll = (int64_t)l * l;
  const double* omega = sketch_omega(Lr, st);
  double* T = ws;                    // S^t Omega, n_l x l row-major
  double* Yt = T + batch * Ln;       // (N T)^t, l x n_r row-major = Y column-major
  double* Qc = Yt + batch * Lr;      // Q column-major (n_r x l)
  double* Z = Qc + batch * Lr;       // Q^t N, l x n_l row-major
  double* Bt = Z + batch * Ln;       // B = Z S^t, l x n_r row-major = B^t column-major
  double* Vl = Bt + batch * Lr;      // l x l Jacobi rotation (column-major)
  double* Ul = Vl + batch * ll;      // l x l sorted
  double* tau = Ul + batch * ll;     // l per matrix
  int* inc = (int*)(tau + batch * l);
  bool ragged = false;
  for (int b = 0; b < batch; ++b) ragged = ragged || nrs[b] != nr;
  if (ragged) {
    CTM_CUDA(cudaMemsetAsync(Yt, 0, sizeof(double) * batch * Lr, st));
    CTM_CUDA(cudaMemsetAsync(Bt, 0, sizeof(double) * batch * Lr, st));
  }
  GemmSpec g;
  if (!warm) kw = 0;
  for (int b = 0; b < batch; ++b) {
    const int mr = nrs[b], ml = nls[b];
    // T = S^t Omega, Omega = [warm_b(:, :kw) | random columns]
    if (kw > 0) {
      g = GemmSpec();
      g.M = ml; g.N = kw; g.K = mr; g.transA = true; g.lda = ml; g.ldb = ldw; g.ldc = l;
      gemm_f64(S[b], warm[b], T + b * Ln, g, st);
    }
    g = GemmSpec();
    g.M = ml; g.N = l - kw; g.K = mr; g.transA = true; g.lda = ml; g.ldb = l; g.ldc = l;
    gemm_f64(S[b], omega + kw, T + b * Ln + kw, g, st);
    // Y^t = T^t N^t
    g = GemmSpec();
    g.M = l; g.N = mr; g.K = ml; g.transA = true; g.lda = l; g.transB = true; g.ldb = ml; g.ldc = nr;
    gemm_f64(T + b * Ln, N[b], Yt + b * Lr, g, st);
  }
  qr_householder(Yt, tau, batch, nr, l, Lr, status, st);
  eye_rect_kernel<<<dim3((unsigned)std::min<int64_t>(4096, (Lr + 255) / 256), batch), 256, 0, st>>>(Qc, nr, l);
  CTM_LAUNCHED();
  qr_apply_Q(Yt, tau, Qc, batch, nr, l, l, Lr, Lr, status, st);
  for (int b = 0; b < batch; ++b) {
    const int mr = nrs[b], ml = nls[b];
    // Z = Q^t N (Qc read row-major is Q^t; its rows beyond mr are zero)
    g = GemmSpec();
    g.M = l; g.N = ml; g.K = mr; g.lda = nr; g.ldb = ml; g.ldc = nl;
    gemm_f64(Qc + b * Lr, N[b], Z + b * Ln, g, st);
    // B = Z S^t
    g = GemmSpec();
    g.M = l; g.N = mr; g.K = ml; g.lda = nl; g.transB = true; g.ldb = ml; g.ldc = nr;
    gemm_f64(Z + b * Ln, S[b], Bt + b * Lr, g, st);
  }
  CoopScratch& g_coop = ensure_coop(batch, st);
  CTM_CUDA(cudaMemsetAsync(g_coop.flags, 0, 3 * batch * sizeof(int), st));
  CTM_CUDA(cudaMemsetAsync(g_coop.conv, 0, batch * sizeof(int), st));
  set_identity_colmajor(Vl, batch, l, st);
  frob2_kernel<<<batch, 256, 0, st>>>(Bt, Lr, g_coop.frob2);
  CTM_LAUNCHED();
  Sync s{g_coop.bar, g_coop.abort, status, (long long)lim_spins()};
  {
    ProfScope ps(PROF_SVD, st, 0.0, 8.0 * batch * Lr * 4, prof_tag("jacobi", batch, nr, l, 0));
    launch_jacobi(Bt, Vl, batch, nr, l, lim_sweeps(), g_coop.flags, g_coop.conv, sweeps_out, g_coop.frob2,
                  g_coop.flop_acc, s, st);
  }
  size_t smem = (size_t)l * (sizeof(double) + sizeof(int));
  svd_rect_finalize_kernel<<<batch, 256, smem, st>>>(Bt, Vl, lam, l, Vo, l, Ul, nr, l, inc, inc + batch, status);
  CTM_LAUNCHED();
  // U = Q Ul (n_r x l row-major)
  g = GemmSpec();
  g.M = nr; g.N = l; g.K = l; g.batch = batch; g.transA = true; g.lda = nr; g.ldb = l; g.ldc = l;
  g.strideA = Lr; g.strideB = ll; g.strideC = Lr;
  gemm_f64(Qc, Ul, Uo, g, st);
  std::vector<int> flags(2 * batch, 0);
  CTM_CUDA(cudaMemcpyAsync(flags.data(), inc, sizeof(int) * 2 * batch, cudaMemcpyDeviceToHost, st));
  CTM_CUDA(cudaStreamSynchronize(st));
  incomplete_host.assign(flags.begin(), flags.begin() + batch);
  rank_host.assign(flags.begin() + batch, flags.end());
}

size_t svd_product_full_ws(int batch, int nr, int nl, int r) {
  // Xc, Uc: batch x nr x r; Rx, R2, Vw, Ul, Uo, Wt: batch x r x r; tall extras: Sc nr x nl, Qc nr x r,
  // Rs r x r; reflector scalars of the three QRs
  const size_t per = (size_t)2 * nr * r + (size_t)6 * r * r + (size_t)nr * nl + (size_t)nr * r + (size_t)r * r + 3 * r;
  return sizeof(double) * batch * per + sizeof(int) * 2 * batch + 256;
}

void svd_product_full(const double* const* N, const double* const* S, const int* nrs, const int* nls, int batch, int r,
                      double* ws, double* lam, double* const* U, double* const* V, int* status, int* sweeps_out,
                      std::vector<int>& rank_host, cudaStream_t st) {
  int nr = 0, nl = 0;
  for (int b = 0; b < batch; ++b) {
    nr = std::max(nr, nrs[b]);
    nl = std::max(nl, nls[b]);
    CTM_CHECK(std::min(nrs[b], nls[b]) == r, CTM_ERR_INVALID_ARG, "svd_product_full: rank bound differs");
  }
  const int64_t Lr = (int64_t)nr * r, rr = (int64_t)r * r;
  double* Xc = ws;                    // X column-major (nr x r per pair; rows beyond n_r zero), then its QR
  double* Uc = Xc + batch * Lr;       // [V_J; 0] column-major, then U = Q_x [V_J; 0]
  double* Rx = Uc + batch * Lr;       // R_x row-major = A = R_x^t column-major, then A's QR
  double* R2 = Rx + batch * rr;       // R_2 row-major (A = Q_2 R_2) = R_2^t column-major: the Jacobi matrix
  double* Vw = R2 + batch * rr;       // Jacobi rotation V_J, column-major
  double* Ul = Vw + batch * rr;       // sorted V_J, row-major
  double* Uo = Ul + batch * rr;       // sorted U_J (normalised columns of R_2^t V_J), row-major
  double* Wt = Uo + batch * rr;       // W = Q_2 V_J, column-major
  double* Sc = Wt + batch * rr;       // tall pairs: S column-major (n_r x n_l)
  double* Qc = Sc + batch * (int64_t)nr * nl;  // tall pairs: Q_s column-major (n_r x r)
  double* Rs = Qc + batch * Lr;       // tall pairs: R_s row-major (r x r)
  double* taus = Rs + batch * rr;     // reflector scalars of S (tall pairs)
  double* taux = taus + batch * r;    // reflector scalars of X
  double* tau2 = taux + batch * r;    // reflector scalars of A = R_x^t
  int* inc = (int*)(tau2 + batch * r);
  bool ragged = false;
  for (int b = 0; b < batch; ++b) ragged = ragged || nrs[b] != nr;
  if (ragged) CTM_CUDA(cudaMemsetAsync(Xc, 0, sizeof(double) * batch * Lr, st));
  GemmSpec g;
  // tall pairs (n_r > n_l = r): S = Q_s R_s, X = N R_s^t; grouped by shape for the batched QR
  std::vector<int> done(batch, 0);
  for (int b0 = 0; b0 < batch; ++b0) {
    if (done[b0] || nrs[b0] <= nls[b0]) continue;
    std::vector<int> grp;
    for (int b = b0; b < batch; ++b)
      if (!done[b] && nrs[b] == nrs[b0] && nls[b] == nls[b0]) grp.push_back(b), done[b] = 1;
    const int mr = nrs[b0], ml = nls[b0], ng = (int)grp.size();
    const int64_t snl = (int64_t)mr * ml;
    for (int k = 0; k < ng; ++k) {  // column-major copies (slots indexed by position in the group)
      PermSpec ps;
      ps.rank = 2;
      ps.out_dims[0] = ml;
      ps.out_dims[1] = mr;
      ps.in_stride[0] = 1;
      ps.in_stride[1] = ml;
      permute(S[grp[k]], F64, Sc + k * snl, F64, ps, false, 1.0, st);
    }
    qr_householder(Sc, taus, ng, mr, ml, snl, status, st);
    qr_extract_R(Sc, Rs, ng, mr, ml, snl, st);
    // Q_s of the group is formed in Uc (free until the lift of U below), then moved to the pairs'
    // own slots of Qc
    eye_rect_kernel<<<dim3((unsigned)std::min<int64_t>(4096, ((int64_t)mr * r + 255) / 256), ng), 256, 0, st>>>(Uc, mr, r);
    CTM_LAUNCHED();
    qr_apply_Q(Sc, taus, Uc, ng, mr, ml, r, snl, (int64_t)mr * r, status, st);
    for (int k = 0; k < ng; ++k) {
      const int b = grp[k];
      // X^t = R_s N^t (r x n_r), i.e. X column-major with leading dimension nr
      g = GemmSpec();
      g.M = r; g.N = mr; g.K = ml; g.lda = r; g.transB = true; g.ldb = ml; g.ldc = nr;
      gemm_f64(Rs + k * rr, N[b], Xc + b * Lr, g, st);
      CTM_CUDA(cudaMemcpyAsync(Qc + b * Lr, Uc + k * (int64_t)mr * r, sizeof(double) * mr * r, cudaMemcpyDeviceToDevice,
                               st));
    }
  }
  for (int b = 0; b < batch; ++b) {
    if (nrs[b] > nls[b]) continue;
    // X^t = S N^t (n_r x n_r): X = rho = N S^t column-major
    const int mr = nrs[b], ml = nls[b];
    g = GemmSpec();
    g.M = mr; g.N = mr; g.K = ml; g.lda = ml; g.transB = true; g.ldb = ml; g.ldc = nr;
    gemm_f64(S[b], N[b], Xc + b * Lr, g, st);
  }
  // Preconditioning by two QR factorisations (as in Drmac and Veselic's one-sided Jacobi SVD):
  // X = Q_x R_x, then A = R_x^t = Q_2 R_2, and the one-sided Jacobi runs on the r columns of R_2^t.
  // After the QRs the graded spectrum sits on the diagonal and the sweeps converge in a fraction
  // of the sweeps they need on X itself (44 -> 8 on a 384-wide matrix graded over 13 decades).
  // R_2^t V_J = U_J S gives R_x = U_J S (Q_2 V_J)^t, hence X = (Q_x U_J) S (Q_2 V_J)^t.
  qr_householder(Xc, taux, batch, nr, r, Lr, status, st);
  qr_extract_R(Xc, Rx, batch, nr, r, Lr, st);
  qr_householder(Rx, tau2, batch, r, r, rr, status, st);
  qr_extract_R(Rx, R2, batch, r, r, rr, st);
  CoopScratch& g_coop = ensure_coop(batch, st);
  frob2_kernel<<<batch, 256, 0, st>>>(R2, rr, g_coop.frob2);
  CTM_LAUNCHED();
  Sync sy{g_coop.bar, g_coop.abort, status, (long long)lim_spins()};
  {
    ProfScope ps(PROF_SVD, st, 0.0, 8.0 * batch * rr * 4, prof_tag("jacobi_full", batch, r, r, 0));
    if (r <= 384) {
      // FP32 sweeps first (GB300 runs FP32 at 64x its FP64 rate): one-sided Jacobi on an FP32 copy
      // scaled to unit norm until the pairs are orthogonal to 1e-5, accumulating V32.  V32 is made
      // orthogonal in FP64 by two Newton-Schulz steps V <- V (3I - V^t V)/2 (orthogonality error
      // e -> ~e^2), the FP64 matrix is rotated by it, W <- W V, and the FP64 sweeps finish from
      // there: near convergence one-sided Jacobi converges quadratically, so two to three FP64
      // sweeps remain.  The result is the FP64 Jacobi SVD of R_2^t; only its starting rotation
      // came from FP32.  Scratch: Ul (FP32 W and V), Uo, Wt (Newton-Schulz), free until finalize.
      float* W32 = reinterpret_cast<float*>(Ul);
      float* V32 = W32 + batch * rr;
      double* ones = Wt;                 // unit Frobenius norms of the FP32 copies
      double* facc32 = Wt + batch;       // the FP32 sweeps' operations (not FP64 work: not reported)
      fill_kernel<<<1, 256, 0, st>>>(ones, batch + 1, 1.0);
      CTM_LAUNCHED();
      dim3 cg((unsigned)std::min<int64_t>(1024, (rr + 255) / 256), batch);
      to_f32_unit_kernel<<<cg, 256, 0, st>>>(R2, W32, V32, r, g_coop.frob2);
      CTM_LAUNCHED();
      CTM_CUDA(cudaMemsetAsync(g_coop.flags, 0, 3 * batch * sizeof(int), st));
      CTM_CUDA(cudaMemsetAsync(g_coop.conv, 0, batch * sizeof(int), st));
      if (r <= 128)
        launch_jacobi_b<float, 4>(W32, V32, batch, r, 30, 1e-5, g_coop.flags, g_coop.conv, sweeps_out, ones,
                                  facc32, sy, 0, st);
      else if (r <= 256)
        launch_jacobi_b<float, 8>(W32, V32, batch, r, 30, 1e-5, g_coop.flags, g_coop.conv, sweeps_out, ones,
                                  facc32, sy, 0, st);
      else
        launch_jacobi_b<float, 12>(W32, V32, batch, r, 30, 1e-5, g_coop.flags, g_coop.conv, sweeps_out, ones,
                                   facc32, sy, 0, st);
      f32_to_f64_kernel<<<(unsigned)std::min<int64_t>(4096, (batch * rr + 255) / 256), 256, 0, st>>>(V32, Vw,
                                                                                                      batch * rr);
      CTM_LAUNCHED();
      // Row-major views of the column-major arrays: Vs = V^t, Ws = W^t.  G = V^t V = Vs Vs^t;
      // V (3I - G)/2 has row-major view 1.5 Vs - 0.5 G Vs; W V has row-major view Vs Ws.
      GemmSpec gg;
      gg.M = r; gg.N = r; gg.K = r; gg.batch = batch; gg.lda = r; gg.ldb = r; gg.ldc = r;
      gg.strideA = rr; gg.strideB = rr; gg.strideC = rr;
      for (int it = 0; it < 2; ++it) {
        GemmSpec g1 = gg;
        g1.transB = true;
        gemm_f64(Vw, Vw, Uo, g1, st);  // G = Vs Vs^t
        CTM_CUDA(cudaMemcpyAsync(Wt, Vw, sizeof(double) * batch * rr, cudaMemcpyDeviceToDevice, st));
        GemmSpec g2 = gg;
        g2.alpha = -0.5;
        g2.beta = 1.5;
        gemm_f64(Uo, Vw, Wt, g2, st);  // 1.5 Vs - 0.5 G Vs
        CTM_CUDA(cudaMemcpyAsync(Vw, Wt, sizeof(double) * batch * rr, cudaMemcpyDeviceToDevice, st));
      }
      gemm_f64(Vw, R2, Ul, gg, st);  // Ws <- Vs Ws
      CTM_CUDA(cudaMemcpyAsync(R2, Ul, sizeof(double) * batch * rr, cudaMemcpyDeviceToDevice, st));
    } else {
      set_identity_colmajor(Vw, batch, r, st);
    }
    CTM_CUDA(cudaMemsetAsync(g_coop.flags, 0, 3 * batch * sizeof(int), st));
    CTM_CUDA(cudaMemsetAsync(g_coop.conv, 0, batch * sizeof(int), st));
    const double tol64 = 2.220446049250313e-16 * r;
    if (r <= 128)
      launch_jacobi_b<double, 4>(R2, Vw, batch, r, lim_sweeps(), tol64, g_coop.flags, g_coop.conv, sweeps_out,
                                 g_coop.frob2, g_coop.flop_acc, sy, 1, st);
    else if (r <= 256)
      launch_jacobi_b<double, 8>(R2, Vw, batch, r, lim_sweeps(), tol64, g_coop.flags, g_coop.conv, sweeps_out,
                                 g_coop.frob2, g_coop.flop_acc, sy, 1, st);
    else if (r <= 384)
      launch_jacobi_b<double, 12>(R2, Vw, batch, r, lim_sweeps(), tol64, g_coop.flags, g_coop.conv, sweeps_out,
                                  g_coop.frob2, g_coop.flop_acc, sy, 1, st);
    else
      launch_jacobi(R2, Vw, batch, r, r, lim_sweeps(), g_coop.flags, g_coop.conv, sweeps_out, g_coop.frob2,
                    g_coop.flop_acc, sy, st);
  }
  size_t smem = (size_t)r * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024)
    CTM_CUDA(cudaFuncSetAttribute(svd_rect_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // lam, Uo = U_J (normalised columns of R_2^t V_J, sorted), Ul = V_J sorted
  svd_rect_finalize_kernel<<<batch, 256, smem, st>>>(R2, Vw, lam, r, Uo, r, Ul, r, r, inc, inc + batch, status);
  CTM_LAUNCHED();
  // U = Q_x [U_J; 0] and W = Q_2 V_J (both column-major)
  for (int b = 0; b < batch; ++b) {
    embed_transpose(Uo + b * rr, r, Uc + b * Lr, nr, st);
    embed_transpose(Ul + b * rr, r, Wt + b * rr, r, st);
  }
  qr_apply_Q(Xc, taux, Uc, batch, nr, r, r, Lr, Lr, status, st);
  qr_apply_Q(Rx, tau2, Wt, batch, r, r, r, rr, rr, status, st);
  for (int b = 0; b < batch; ++b) {
    const int mr = nrs[b];
    PermSpec ps;  // row-major n_r x r from the column-major block (first n_r rows)
    ps.rank = 2;
    ps.out_dims[0] = mr;
    ps.out_dims[1] = r;
    ps.in_stride[0] = 1;
    ps.in_stride[1] = nr;
    permute(Uc + b * Lr, F64, U[b], F64, ps, false, 1.0, st);
    if (mr <= nls[b]) {
      PermSpec pw;  // V = W (row-major r x r)
      pw.rank = 2;
      pw.out_dims[0] = r;
      pw.out_dims[1] = r;
      pw.in_stride[0] = 1;
      pw.in_stride[1] = r;
      permute(Wt + b * rr, F64, V[b], F64, pw, false, 1.0, st);
    } else {
      // V = Q_s W (Q_s column-major n_r x r, W column-major r x r)
      g = GemmSpec();
      g.M = mr; g.N = r; g.K = r; g.transA = true; g.lda = mr; g.transB = true; g.ldb = r; g.ldc = r;
      gemm_f64(Qc + b * Lr, Wt + b * rr, V[b], g, st);
    }
  }
  std::vector<int> flags(2 * batch, 0);
  CTM_CUDA(cudaMemcpyAsync(flags.data(), inc, sizeof(int) * 2 * batch, cudaMemcpyDeviceToHost, st));
  CTM_CUDA(cudaStreamSynchronize(st));
  rank_host.assign(flags.begin() + batch, flags.end());
}

double jacobi_flops_read_reset(cudaStream_t st) {
  CoopScratch& g_coop = coop_of(st);
  if (!g_coop.flop_acc) return 0.0;
  double v = 0.0;
  CTM_CUDA(cudaMemcpyAsync(&v, g_coop.flop_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  CTM_CUDA(cudaStreamSynchronize(st));
  CTM_CUDA(cudaMemsetAsync(g_coop.flop_acc, 0, sizeof(double), st));
  return v;
}

void set_identity_colmajor(double* V, int batch, int r, cudaStream_t st) {
  dim3 grid((unsigned)std::min<int64_t>(4096, ((int64_t)r * r + 255) / 256), batch);
  identity_kernel<<<grid, 256, 0, st>>>(V, r);
  CTM_LAUNCHED();
}

void svd_jacobi(double* W, double* V, double* lam, double* Uo, double* Vo, int batch, int r, int max_sweeps,
                int* status, int* sweeps_out, cudaStream_t st) {
  if (batch == 0 || r == 0) return;
  ProfScope ps(PROF_SVD, st, 0.0, 8.0 * batch * r * r * 4);
  CoopScratch& g_coop = ensure_coop(batch, st);
  CTM_CUDA(cudaMemsetAsync(g_coop.flags, 0, 3 * batch * sizeof(int), st));
  CTM_CUDA(cudaMemsetAsync(g_coop.conv, 0, batch * sizeof(int), st));
  Sync s{g_coop.bar, g_coop.abort, status, (long long)lim_spins()};
  frob2_kernel<<<batch, 256, 0, st>>>(W, (int64_t)r * r, g_coop.frob2);
  CTM_LAUNCHED();
  launch_jacobi(W, V, batch, r, r, max_sweeps, g_coop.flags, g_coop.conv, sweeps_out, g_coop.frob2,
                g_coop.flop_acc, s, st);
  size_t smem = (size_t)r * (sizeof(double) + sizeof(int));
  if (smem > 48 * 1024) CTM_CUDA(cudaFuncSetAttribute(svd_finalize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  svd_finalize_kernel<<<batch, 256, smem, st>>>(W, V, lam, Uo, Vo, r, status);
  CTM_LAUNCHED();
}

}  // namespace ctm

// ==================================================================== allocation-free batched SVD
// For callers that may not allocate device memory (for example code that runs
// inside a caller-owned memory pool or under an allocator that forbids
// cudaMalloc): every byte of workspace of this entry point lives in one
// fixed-size array in the library's device image.
namespace ctm {
namespace {

constexpr int64_t kNoAllocMaxElems = int64_t(1) << 20;  // batch * r * r limit (8 MiB per working copy)
constexpr int kNoAllocMaxBatch = 1024;
// [W: max][V: max][frob2: 1024][flop acc: 8][ints: bar 2, abort 1, status 1, sweeps 1, pad, flags 3*1024, conv 1024]
constexpr int64_t kNoAllocInts = 8 + 4 * kNoAllocMaxBatch;
constexpr int64_t kNoAllocDoubles = 2 * kNoAllocMaxElems + kNoAllocMaxBatch + 8 + kNoAllocInts / 2;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

// Device address of the scratch array on the current device.  Looked up on every call (it
// allocates nothing and is cheap once the module is loaded), so that a reset device or a new
// primary context never leaves a stale address behind.
double* noalloc_base() {
  void* p = nullptr;
  CTM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  return (double*)p;
}

void svd_noalloc(const double* M, int batch, int r, double* U, double* sv, double* V, cudaStream_t st) {
  const int64_t rr = (int64_t)r * r;
  double* base = noalloc_base();
  double* W = base;
  double* Vw = base + kNoAllocMaxElems;
  double* frob2 = base + 2 * kNoAllocMaxElems;
  double* facc = frob2 + kNoAllocMaxBatch;
  int* ints = (int*)(facc + 8);
  unsigned* bar = (unsigned*)ints;
  int* abort_flag = ints + 2;
  int* status = ints + 3;
  int* sweeps = ints + 4;
  int* flags = ints + 8;
  int* conv = flags + 3 * kNoAllocMaxBatch;
  // everything that must start at zero, in stream order
  CTM_CUDA(cudaMemsetAsync(ints, 0, kNoAllocInts * sizeof(int), st));
  CTM_CUDA(cudaMemsetAsync(facc, 0, sizeof(double), st));
  PermSpec ps;  // column-major working copy: W_b[k*r + i] = M_b[i][k]
  ps.rank = 3;
  ps.out_dims[0] = batch;
  ps.out_dims[1] = r;
  ps.out_dims[2] = r;
  ps.in_stride[0] = rr;
  ps.in_stride[1] = 1;
  ps.in_stride[2] = r;
  permute(M, F64, W, F64, ps, false, 1.0, st);
  set_identity_colmajor(Vw, batch, r, st);
  frob2_kernel<<<batch, 256, 0, st>>>(W, rr, frob2);
  CTM_LAUNCHED();
  Sync s{bar, abort_flag, status, (long long)lim_spins()};
  launch_jacobi(W, Vw, batch, r, r, lim_sweeps(), flags, conv, sweeps, frob2, facc, s, st);
  size_t smem = (size_t)r * (sizeof(double) + sizeof(int));
  svd_finalize_kernel<<<batch, 256, smem, st>>>(W, Vw, sv, U, V, r, status);
  CTM_LAUNCHED();
  int hs = 0;
  CTM_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
  CTM_CUDA(cudaStreamSynchronize(st));
  if (hs & DEV_TIMEOUT) throw Error(CTM_ERR_TIMEOUT, "device wait timed out");
  if (hs & DEV_SVD_NOCONV) throw Error(CTM_ERR_SVD_NOCONV, "Jacobi SVD did not converge");
  if (hs & DEV_NONFINITE) throw Error(CTM_ERR_NONFINITE, "non-finite singular value");
}

}  // namespace
}  // namespace ctm

extern "C" int ctm_svd_noalloc(const double* M, int batch, int r, double* U, double* s, double* V, void* stream) {
  if (!M || !U || !s || !V || batch < 1 || r < 1 || batch > ctm::kNoAllocMaxBatch ||
      (int64_t)batch * r * r > ctm::kNoAllocMaxElems)
    return CTM_ERR_INVALID_ARG;
  try {
    ctm::svd_noalloc(M, batch, r, U, s, V, (cudaStream_t)stream);
    return CTM_OK;
  } catch (const ctm::Error& e) {
    fprintf(stderr, "libctm: %s\n", e.what());
    return e.status;
  }
}
