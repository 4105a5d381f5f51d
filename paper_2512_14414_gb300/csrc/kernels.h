// Launch wrappers of the CUDA kernels of libctm (all enqueue on `st`, no host sync).
#pragma once
#include "common.h"
#include "stride_map.h"

namespace ctm {

// ------------------------------------------------------------------ permutation
// out[i_0..i_{r-1}] (row-major over out_dims) = scale * in[sum_k i_k * in_stride[k]]
// (+= when acc).  in/out dtypes may differ (conversion fused into the copy).
struct PermSpec {
  int rank = 0;
  int64_t out_dims[8] = {0};
  int64_t in_stride[8] = {0};  // input stride (elements) of each output dimension
};
void permute(const void* in, DType tin, void* out, DType tout, const PermSpec& p, bool acc,
             double scale, cudaStream_t st);

// ------------------------------------------------------------------ GEMM (SIMT)
// C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b], row-major.
// op(A) is M x K: A[m*lda+k] (transA=0) or A[k*lda+m] (transA=1);
// op(B) is K x N: B[k*ldb+n] (transB=0) or B[n*ldb+k] (transB=1).
struct GemmSpec {
  int64_t M = 0, N = 0, K = 0, batch = 1;
  bool transA = false, transB = false;
  int64_t lda = 0, ldb = 0, ldc = 0;
  int64_t strideA = 0, strideB = 0, strideC = 0;
  double alpha = 1.0, beta = 0.0;
};
void gemm_f64(const double* A, const double* B, double* C, const GemmSpec& g, cudaStream_t st);
void gemm_f32(const float* A, const float* B, float* C, const GemmSpec& g, cudaStream_t st);
// The same products with operands and result addressed through group maps (stride_map.h) instead
// of leading dimensions: no permuted copies.  g supplies M, N, K, batch, alpha, beta; transA /
// transB only pick the load order (set the one whose inner index has unit stride).
void gemm_strided_f64(const double* A, const double* B, double* C, const GemmSpec& g, const StridedGemm& sm,
                      cudaStream_t st);
void gemm_strided_f32(const float* A, const float* B, float* C, const GemmSpec& g, const StridedGemm& sm,
                      cudaStream_t st);
// Tensor-core GEMM (tcgen05): C[b][m][n] (+)= sum_k A[b][m][k] B[b][n][k]; A, B BF16 or FP32 (as TF32),
// C FP32 row-major.  tc_gemm_ok tells whether TMA can address the operands.
bool tc_gemm_ok(bool bf16, int64_t M, int64_t N, int64_t K, const void* A, const void* B);
void gemm_tc(const void* A, const void* B, float* C, int64_t M, int64_t N, int64_t K, int64_t batch, bool bf16,
             double beta, int* status, cudaStream_t st);
// Error-compensated TF32: C (+)= Ahi Bhi^t + Ahi Blo^t + Alo Bhi^t (operands from split_tf32).
void gemm_tc_x3(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, float* C, int64_t M,
                int64_t N, int64_t K, int64_t batch, double beta, int* status, cudaStream_t st);
// hi = x rounded to TF32, lo = (x - hi) rounded to TF32.
void split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t st);
// Error-compensated BF16: C (+)= Ahi Bhi^t + Ahi Blo^t + Alo Bhi^t, operands BF16 (split_bf16).
void gemm_tc_x3_bf16(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, float* C, int64_t M,
                     int64_t N, int64_t K, int64_t batch, double beta, int* status, cudaStream_t st);
// MLP forward (FP32): hidden layers Linear + GELU, last layer Linear; W[k] is [dims[k+1]][dims[k]],
// b[k] has dims[k+1] entries (b may be null); work holds 2 * batch * max hidden width floats.
void mlp_forward(const float* x, int batch, int n_layers, const int* dims, const float* const* W,
                 const float* const* b, float* work, float* y, cudaStream_t st);
int64_t mlp_work_floats(int batch, int n_layers, const int* dims);
void mlp_backward(const float* x, const float* target, int batch, int n_layers, const int* dims,
                  const float* const* W, const float* const* b, float* const* dW, float* const* db, float* work,
                  float* loss, cudaStream_t st);
void adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2, float eps, int t,
               cudaStream_t st);
// hi = x rounded to BF16, lo = (x - hi) rounded to BF16 (BF16 outputs).
void split_bf16(const float* x, void* hi, void* lo, int64_t n, cudaStream_t st);

// ------------------------------------------------------------------ elementwise / reductions
void fill(void* p, DType t, int64_t n, double v, cudaStream_t st);
void cast(const void* in, DType tin, void* out, DType tout, int64_t n, bool acc, cudaStream_t st);
// partial[...] then out = sum of squares of x (deterministic two-pass); work >= 1024 doubles.
void sumsq(const void* x, DType t, int64_t n, double* out, double* work, cudaStream_t st);
// y = x * rsqrt(*ss) and *inv = rsqrt(*ss)
void scale_rsqrt(const void* x, DType t, int64_t n, const double* ss, void* y, double* inv, cudaStream_t st);
// dx (+)= dy * (*inv)
void scale_by(const void* dy, DType t, int64_t n, const double* inv, void* dx, bool acc, cudaStream_t st);

// ------------------------------------------------------------------ projector helpers (FP64)
// Singular values lam (batch x r, descending).  For k < kept: inv[b][k] = lam^-1/2 if
// lam > cut*lam_0 else 0.  Columns of U, V (n_r x r row-major, batch) whose lam <= rank_tol*lam_0
// are zeroed.  sinv[b][k] = 1/lam for lam > rank_tol*lam_0 else 0.
void proj_prepare(const double* lam, double* U, double* V, double* inv, double* sinv, int batch,
                  int64_t n_r, int r, int kept, double cut, double rank_tol, int* status, cudaStream_t st);
// Sign gauge: column k of V (n x r row-major) gets a positive entry of largest magnitude; U follows.
void sign_fix(double* U, double* V, int batch, int64_t n, int r, cudaStream_t st);
// Flip (U[:,k], V[:,k]) for k < ncols where V[:,k] . Vref[:,k] < 0 (V, U: n x ld row-major, Vref:
// n x ldr): aligns the sign gauge with a reference factorisation (the previous iteration's).
void sign_align(double* U, double* V, int64_t ld, const double* Vref, int64_t ldr, int64_t n, int ncols,
                cudaStream_t st);
// X[b][i][k] = Y[b][i*ldy + k] * s[b][k] for k < kept (X is n x kept row-major)
void scale_cols(const double* Y, int64_t ldy, int64_t strideY, const double* s, int64_t strideS, double* X,
                int batch, int64_t n, int kept, cudaStream_t st);
// dl[b][k] = -0.5 inv^3 (sum_i dZ[i][k] U[i][k] + sum_i dW[i][k] V[i][k]), k < kept
void proj_dlam(const double* dZ, const double* U, const double* dW, const double* V, const double* inv,
               double* dl, int batch, int64_t n_r, int r, int kept, cudaStream_t st);
// core (r x r) of the thin-SVD adjoint: F_ij (A_ij - A_ji) s_j + s_i F_ij (B_ij - B_ji) off the diagonal,
// dl on it, with F_ij = (s_j^2 - s_i^2) / ((s_j^2 - s_i^2)^2 + eps (s_i^2 + s_j^2)^2) on the triplets above
// rank_tol * s_1 (0 elsewhere)
void proj_core(const double* Aa, const double* Bb, const double* lam, const double* dl, double* core, int batch,
               int r, int kept, double rank_tol, double eps, cudaStream_t st);
// E[b] = (dU[b] - X[b]) * sinv[b] (n_r x kept)
void proj_resid(const double* dU, const double* X, const double* sinv, double* E, int batch, int64_t n_r,
                int r, int kept, cudaStream_t st);

// ------------------------------------------------------------------ dense linear algebra (FP64)
// Batched Householder QR of tall column-major matrices (m x n, m >= n, ld = m):
// on exit the upper triangle holds R, below it the reflectors (v_0 = 1 implicit), tau[n].
void qr_householder(double* A, double* tau, int batch, int m, int n, int64_t strideA, int* status,
                    cudaStream_t st);
// R (n x n, row-major, zeros below the diagonal) from the factored column-major workspace.
void qr_extract_R(const double* A, double* R, int batch, int m, int n, int64_t strideA, cudaStream_t st);
// X (m x k, column-major, ld m) := Q X with Q = H_0 ... H_{n-1} from qr_householder.
void qr_apply_Q(const double* A, const double* tau, double* X, int batch, int m, int n, int k,
                int64_t strideA, int64_t strideX, int* status, cudaStream_t st);
// Batched one-sided Jacobi SVD of square r x r matrices.
// W: column-major working copy (batch x r x r, destroyed); V (batch x r x r column-major) must hold
// the starting orthogonal matrix (identity for a cold start).  On exit: lam (descending),
// Uo and Vo row-major r x r with columns = singular vectors, sorted.
void svd_jacobi(double* W, double* V, double* lam, double* Uo, double* Vo, int batch, int r, int max_sweeps,
                int* status, int* sweeps_out, cudaStream_t st);
void set_identity_colmajor(double* V, int batch, int r, cudaStream_t st);
// Truncated SVD of rho_b = N_b S_b^t (N_b, S_b: n_r x n_l row-major) without forming rho:
// Y = N (S^t Omega), Q = orth(Y) (Householder), B^t = S (Q^t N)^t, one-sided Jacobi on the
// l columns of B^t.  lam: batch x l descending; Uo, Vo: batch x n_r x l row-major with
// rho ~= U diag(lam) V^t.  ws: svd_sketch_product_ws(...) bytes of device memory.
// incomplete_host[b] = 1 where the smallest of the l values is above 1e-14 lam_max;
// rank_host[b] = how many of the l values are above 1e-14 lam_max.
size_t svd_sketch_product_ws(int batch, int nr, int nl, int l);
// warm (nullable): per matrix an n_r x kw block (row-major, ld ldw) that replaces the first kw
// columns of the random test matrix -- the previous right singular vectors, so that rho Omega
// is already close to U Sigma and the Jacobi sweeps start near convergence.
// nrs / nls: per matrix n_r and n_l (host arrays); ws from svd_sketch_product_ws(batch, max n_r,
// max n_l, l); Uo / Vo hold batch x (max n_r) x l, rows beyond a matrix's own n_r zero.
void svd_sketch_product(const double* const* N, const double* const* S, const int* nrs, const int* nls, int batch,
                        int l, const double* const* warm, int ldw, int kw, double* ws, double* lam, double* Uo,
                        double* Vo, int* status, int* sweeps_out, std::vector<int>& incomplete_host,
                        std::vector<int>& rank_host, cudaStream_t st);
// Full thin SVD of rho_b = N_b S_b^t (n_r x n_r, rank <= r = min(n_r, n_l), the same r for the
// whole batch): X = N S^t for n_r <= n_l, X = N R_s^t with S = Q_s R_s (Householder) for n_r > n_l,
// so that rho = X B^t with B = I or Q_s.  X = Q_x R_x, R_x^t = Q_2 R_2 (Householder) and one-sided
// Jacobi on R_2^t: R_2^t V_J = U_J S, hence U = Q_x U_J and V = B Q_2 V_J.  Outputs per pair: lam (batch x r,
// descending), U[b], V[b] (n_r x r row-major), rank_host[b] = values above 1e-14 lam_max.
// ws: svd_product_full_ws(batch, max n_r, max n_l, r).
size_t svd_product_full_ws(int batch, int nr, int nl, int r);
void svd_product_full(const double* const* N, const double* const* S, const int* nrs, const int* nls, int batch, int r,
                      double* ws, double* lam, double* const* U, double* const* V, int* status, int* sweeps_out,
                      std::vector<int>& rank_host, cudaStream_t st);
// Flops counted by the Jacobi kernels since the last call (6r per pair test, 12r per rotation).
double jacobi_flops_read_reset(cudaStream_t st);
// X[k*m + i] = U[i*r + k] for i < r, 0 for r <= i < m  (k < r): [U; 0] stored column-major.
void embed_transpose(const double* U, int r, double* X, int64_t m, cudaStream_t st);

// ------------------------------------------------------------------ energy (FP64)
// rho: n_terms x (d^2 x d^2) [ket (s1 s2)][bra (s1' s2')], any dtype converted to FP64.
// hs: n_terms x d^2 x d^2 FP64 device, coup: n_terms.  e_bond[t] = Tr(rho h)/Tr(rho),
// *e_site = sum_t coup_t e_t / n_sites.  drho (FP64, optional) gets dE/drho.
void energy_terms(const double* rho, const double* hs, const double* coup, int n_terms, int d2, double inv_sites,
                  double* e_bond, double* e_site, double* drho, int* status, cudaStream_t st);

// Eq. Mag1: rho = n_sites one-site RDMs (2 x 2, [ket][bra]); m[site] = (<Sx>, <Sy>, <Sz>) with
// <Sy> = 0 for real tensors; *M = mean over sites of |m|.
void site_magnetization(const double* rho, int n_sites, double* m, double* M, int* status, cudaStream_t st);
// Eq. Mag2: *Mp = |sum_{k < na} e[idx[k]] - sum_{k < nb} e[idx[na + k]]| / 4 (idx on the device)
void plaquette_order(const double* e_terms, const int* idx_dev, int na, int nb, double* Mp, cudaStream_t st);

// spectrum change between two sets of normalised spectra (batch x kept), result max into *out (atomic max)
void spectrum_delta(const double* lam, const double* lam_prev, int batch, int r, int kept, double* out,
                    cudaStream_t st);

}  // namespace ctm
