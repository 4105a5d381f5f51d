/*
 * libctm -- nested single-layer CTMRG energy and gradient on one GB300 GPU.
 *
 * C ABI.  Plain pointers and sizes only.  Every entry point returns an int
 * status: CTM_OK (0) or one of the CTM_ERR_* codes below.  No C++ exception
 * crosses this boundary.  A failed call leaves the handle valid; the next
 * ctm_init clears its error state.
 *
 * The method (arXiv:2512.14414, Sec. SLF):
 *   E(X) = <Psi|H|Psi> / <Psi|Psi>                                   (Eq. ExpH)
 * evaluated on the nested single-layer network in which ket A and bra A* are
 * separate sites, joined by the crossing tensors X and Y (Eq. XY), contracted
 * by multisite CTMRG (Fig. 3) with projectors from QR + SVD (Eqs. PQ, QRSVD);
 * the gradient dE/dX is reverse mode through every CTMRG iteration (Eq. AD),
 * or, at a converged environment, the fixed-point gradient that the
 * Discussion section proposes (ctm_grad_fixed_point).
 *
 * Layouts (all row-major, C order):
 *   site tensors   A: (Lx*Ly) x [d][D][D][D][D]  = A[s][l][u][r][d];
 *                  PEPS site (x, y) at index y*Lx + x.
 *   environment    per nested site (row-major over the 2Ly x 2Lx nested cell),
 *                  8 tensors in the order C_ul, T_u, C_ur, T_r, C_dr, T_d,
 *                  C_dl, T_l, each in the ring convention (legs listed
 *                  clockwise around the site): C = [prev][next],
 *                  T = [prev][in][next], with
 *                    C_ul [down][right]   T_u [left][in][right]
 *                    C_ur [left][down]    T_r [up][in][down]
 *                    C_dr [up][left]      T_d [right][in][left]
 *                    C_dl [right][up]     T_l [down][in][up].
 *                  "in" is the leg of the site on that side; its size is D,
 *                  or D*d (index k*d + s) for the ket's right leg, the
 *                  bra's up leg and Y's left and down legs.
 *   bond operator  h: d^2 x d^2, row (s1 s2), column (s1' s2'), host memory.
 *
 * Ownership: the caller owns every pointer it passes; the library copies
 * what it needs at the call and never frees caller memory.  Device pointers
 * must be device memory of the current device; all work is enqueued on the
 * given stream, and results written to device pointers are valid when that
 * stream reaches the point after the call.  Host output pointers (delta,
 * iteration counts, energies marked host) are valid on return (the call
 * synchronises the stream for them).
 *
 * Threads: one handle per host thread.  Handles share no problem state; the
 * library caches small device work buffers (barrier words of the cooperative
 * kernels, split-K partial tiles, the sketch test matrix) per host thread,
 * device and stream, so work enqueued on different streams never shares them.
 */
#ifndef CTM_H
#define CTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ctm_handle ctm_handle;

enum {
  CTM_OK = 0,
  CTM_ERR_INVALID_ARG = 1,  /* bad size, null pointer, unsupported combination */
  CTM_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  CTM_ERR_OOM = 3,          /* device allocation failed */
  CTM_ERR_NONFINITE = 4,    /* NaN or Inf in a spectrum or in the energy */
  CTM_ERR_SVD_NOCONV = 5,   /* Jacobi SVD hit its sweep limit */
  CTM_ERR_DEGENERATE = 6,   /* all singular values of a bond density matrix are zero */
  CTM_ERR_TIMEOUT = 7,      /* a bounded device-side wait ran out */
  CTM_ERR_STATE = 8,        /* call out of order (e.g. ctm_step before ctm_init) */
  CTM_ERR_DIVERGED = 9      /* the fixed-point gradient's series grew instead of converging */
};

/* Arithmetic of the contractions.  QR, SVD, projectors, their adjoints and
 * the final trace/normalisation of the energy are FP64 in every mode. */
typedef enum {
  CTM_FP64 = 0,    /* FP64 everywhere */
  CTM_TF32 = 1,    /* contractions TF32 x TF32 -> FP32 on the tensor cores */
  CTM_BF16 = 2,    /* contractions BF16 x BF16 -> FP32 on the tensor cores */
  CTM_TF32X3 = 3,  /* error-compensated TF32 (hi*hi + hi*lo + lo*hi) */
  CTM_BF16X3 = 4   /* error-compensated BF16 (hi*hi + hi*lo + lo*hi, ~16 significant bits) */
} ctm_precision;

/* Bond kinds, relative to PEPS site (x, y):
 *   H: (x,y)-(x+1,y)   V: (x,y)-(x,y+1)
 *   DIAG_DR: (x,y)-(x+1,y+1)   DIAG_UR: (x+1,y)-(x,y+1)  (first site listed first) */
typedef enum { CTM_BOND_H = 0, CTM_BOND_V = 1, CTM_BOND_DIAG_DR = 2, CTM_BOND_DIAG_UR = 3 } ctm_bond_kind;

typedef struct {
  int x, y;              /* PEPS site of the bond, 0 <= x < Lx, 0 <= y < Ly */
  int kind;              /* ctm_bond_kind */
  double coupling;       /* J of this term */
  const double* h;       /* d^2 x d^2 bond operator, host memory, copied at ctm_create */
} ctm_term;

typedef struct {
  int Lx, Ly;            /* PEPS unit cell; nested cell is 2Ly x 2Lx */
  int d, D, chi;         /* physical, bond and environment dimensions */
  int precision;         /* ctm_precision */
  int n_terms;
  const ctm_term* terms; /* Hamiltonian: sum of coupling * h over the listed bonds */
  double svd_cutoff_rel; /* projector pseudo-inverse cutoff s_k <= cut*s_1 -> 0; <=0 means 1e-6 */
  double svd_adjoint_eps;/* Lorentzian broadening of 1/(s_j^2-s_i^2), relative to (s_i^2+s_j^2)^2;
                            <0 means 1e-24 */
  int max_iter;          /* upper bound on iterations stored for the gradient (sizes the factor store) */
} ctm_desc;

/* Create a handle for one problem size (Eq. PEPS cell, D, chi, terms).
 * Allocates the device state lazily on first use.  *out is set on success.
 * Limits (CTM_ERR_INVALID_ARG otherwise): all sizes >= 1, 1 <= n_terms <= 64, every term's
 * site inside the cell and kind in 0..3, chi * D * d <= 2048 (the longest projector bond). */
int ctm_create(const ctm_desc* desc, ctm_handle** out);

/* Load the site tensors and the initial environment.
 *   A        : device, FP64, layout above (Lx*Ly tensors).
 *   env0     : device, FP64, concatenation of all nested sites' 8 tensors
 *              (layout above); NULL keeps the environment already in the
 *              handle (e.g. from ctm_set_env).
 * Resets the iteration counter and the stored projector factors. */
int ctm_init(ctm_handle* h, const double* A, const double* env0, void* stream);

/* Run n_iter CTMRG iterations (left, right, up, down moves; Sec. SLF) from
 * the current environment.  Records the projector factors so that a
 * following ctm_grad can differentiate them.  If delta_host is non-NULL it
 * receives the spectrum change of the last iteration:
 * max over projector pairs of ||s~/|s~|_1 - s~_prev/|s~_prev|_1||_inf. */
int ctm_step(ctm_handle* h, int n_iter, double* delta_host, void* stream);

/* Energy per PEPS site of the current environment (Eq. ExpH with the
 * impurity reduced density matrices).  e_site_dev: device, 1 double.
 * e_bonds_dev: device, n_terms doubles (per-term Tr(rho h)/Tr(rho)), or NULL. */
int ctm_energy(ctm_handle* h, double* e_site_dev, double* e_bonds_dev, void* stream);

/* Energy and its gradient with respect to A (Eq. AD): re-initialises from the
 * environment given at ctm_init, runs n_iter iterations, evaluates the
 * energy, then back-propagates through the energy and every iteration
 * (recomputing each iteration from its stored environment).
 *   e_site_dev : device, 1 double.   dA_dev : device, FP64, layout of A. */
int ctm_grad(ctm_handle* h, int n_iter, double* e_site_dev, double* dA_dev, void* stream);

/* Fixed-point (implicit) gradient at the handle's current environment, which
 * the caller has converged with ctm_step (the gradient from a converged
 * environment proposed in the Discussion section, instead of the unrolled
 * chain of Eq. AD).  With f one CTMRG iteration and e the energy (Eq. ExpH),
 * at env* = f(A, env*):
 *     dE/dA = de/dA + sum_{k>=0} [de/denv (df/denv)^k] df/dA,
 * accumulated by repeated vector-Jacobian products through the one iteration
 * recorded at env* (its projector factors computed once).  The series stops
 * when a term adds less than tol relative to the running sum (tol <= 0 means
 * 1e-10) or after max_terms terms (>= 1).
 *   e_site_dev : device, 1 double: the energy at env*.
 *   dA_dev     : device, FP64, layout of A.
 *   info_host  : host, 2 doubles, or NULL: [0] terms taken, [1] fixed-point
 *                residual ||f(A, env*) - env*|| / ||env*|| (how far the
 *                environment is from a fixed point; the result is only as
 *                good as this is small).
 * Requires a prior ctm_init (CTM_ERR_STATE otherwise); the handle keeps env*.
 * The series also stops when its terms have reached a rounding floor (no new
 * smallest term for 10 terms, each below 1e-4 of the sum).
 * CTM_ERR_DIVERGED when a term grows past 10x the first term (the series
 * diverges: env* is not an attracting fixed point, e.g. the iteration has
 * not converged or cycles); info_host is filled in either case.
 * Needs memory for one iteration's tape, not one per iteration. */
int ctm_grad_fixed_point(ctm_handle* h, int max_terms, double tol, double* e_site_dev, double* dA_dev,
                         double* info_host, void* stream);

/* Order parameters of the current environment (Sec. Results).
 * ctm_magnetization: Eq. Mag1 for spin 1/2 (d = 2).  m_dev: device, Lx*Ly x 3 doubles, the
 *   expectation values (<S_x>, <S_y>, <S_z>) of every PEPS site of the cell (index y*Lx + x) from its
 *   one-site reduced density matrix (the nested block [A Y; X A*] with Y's physical line cut open);
 *   with real tensors <S_y> = 0.  M_dev: device, 1 double, M = (1/N) sum_i |m_i| over the N = Lx*Ly
 *   sites.  For a sublattice-rotated ansatz the rotation flips S_x and S_z of one sublattice, which
 *   leaves |m_i| and M unchanged.  CTM_ERR_INVALID_ARG unless d == 2 and Lx*Ly <= 64.
 * ctm_plaquette_order: Eq. Mag2, M_p = |sum_{a in A} e_a - sum_{b in B} e_b| / 4, where e_t =
 *   Tr(rho_t h_t) / Tr(rho_t) of term t (the bond value ctm_energy reports; <S_i.S_j> when h_t is
 *   the Heisenberg bond) and terms_a / terms_b (host, na / nb term indices in the order given to
 *   ctm_create) list the nearest-neighbour bonds of the two inequivalent empty plaquettes.
 *   Mp_dev: device, 1 double.
 * Both enqueue on the stream and synchronise it (status check); no allocation outside the handle. */
int ctm_magnetization(ctm_handle* h, double* m_dev, double* M_dev, void* stream);
int ctm_plaquette_order(ctm_handle* h, const int* terms_a, int na, const int* terms_b, int nb, double* Mp_dev,
                        void* stream);

/* Copy the current environment out / in (FP64, layout above). */
int ctm_get_env(ctm_handle* h, double* env_dev, void* stream);
int ctm_set_env(ctm_handle* h, const double* env_dev, void* stream);

/* Number of doubles of the environment buffer (sum over nested sites and slots). */
int64_t ctm_env_numel(const ctm_handle* h);

/* Launch counters (kernels enqueued by this handle since creation). */
int64_t ctm_kernel_launches(const ctm_handle* h);

/* Limits of the iterative device kernels of this handle.
 *   max_sweeps : sweeps of the one-sided Jacobi SVD before it gives up with
 *                CTM_ERR_SVD_NOCONV (default 60; <= 0 restores the default).
 *   spin_limit : polls of every bounded device-side wait (the grid barriers of
 *                the cooperative QR / Jacobi kernels) before the kernel records
 *                CTM_ERR_TIMEOUT, tells the other blocks to stop and returns
 *                (default 2^22, a few seconds; <= 0 restores the default).
 * A call that runs into either limit returns the error; the handle stays valid
 * and the next ctm_init clears it.  Host memory only, no device work. */
int ctm_set_limits(ctm_handle* h, int max_sweeps, int64_t spin_limit);

/* Per-kernel-class device timing.  ctm_profile(h, 1) clears the record and
 * starts recording a CUDA event pair (on the launching stream) around every
 * launch of the classes below; ctm_profile(h, 0) stops.  ctm_profile_read
 * synchronises the last stream used and returns, for one class, the summed
 * event time (ms), the number of recorded launches and the algorithmic flops
 * and bytes of those launches (flops of the Jacobi SVD are counted on the
 * device: 6r per column-pair test and 12r per rotation).
 * Classes: 0 FP32 GEMM (CUDA cores), 1 permutation, 2 Jacobi SVD,
 * 3 Householder QR, 4 other, 5 tensor-core GEMM, 6 FP64 GEMM (CUDA cores). */
int ctm_profile(ctm_handle* h, int enable);
int ctm_profile_read(ctm_handle* h, int cls, double* ms, int64_t* launches, double* flops, double* bytes);

/* Batched SVD M_b = U_b diag(s_b) V_b^t of square r x r FP64 matrices by the
 * one-sided Jacobi kernels of the projector step (Eq. QRSVD; Hestenes' method).
 *   M : device, batch x r x r, row-major (read only).
 *   U, V : device, batch x r x r, row-major; column k is the k-th singular vector.
 *   s : device, batch x r, descending.
 * Singular values at the rounding floor (below 1e-16 ||M_b||_F) come out as
 * numerical noise with unnormalised U columns.  Allocates its working copies on
 * the device (cudaMalloc) and frees them before returning (a few barrier and
 * flag words are cached per host thread); synchronises the stream. */
int ctm_svd(const double* M, int batch, int r, double* U, double* s, double* V, void* stream);

/* ctm_svd without any device allocation, for callers that cannot call
 * cudaMalloc (memory handed out by a caller-owned pool, allocators that
 * forbid new device allocations while they run).  The paper has no
 * counterpart: this is a service of the library, not a step of the method.
 * Same arguments, layouts and results as ctm_svd; batch*r*r must not exceed
 * 1,048,576 and batch must not exceed 1024, otherwise CTM_ERR_INVALID_ARG is
 * returned before any work is enqueued.  The workspace is one fixed ~16 MiB
 * device array compiled into the library: every GPU that loads the library
 * holds it until the process exits.  Every call looks up the array's device
 * address on the current device (cudaGetSymbolAddress, no allocation); the
 * first call on a device loads the module there, so make that first call
 * before any stream capture.  All calls share the array and every call clears the
 * parts that must start at zero, so calls whose work overlaps on the GPU (two
 * streams, two host threads) race with each other: serialise them.
 * Synchronises the stream to read the status. */
int ctm_svd_noalloc(const double* M, int batch, int r, double* U, double* s, double* V, void* stream);

/* Singular values of the bond density matrix rho = N S^t of every projector pair of iteration
 * `iter` (0-based) of the run since the last ctm_init -- the spectra that define the projectors of
 * Eqs. PQ, QRSVD and whose change is the convergence measure of ctm_step.  Descending, FP64, in
 * execution order (left, right, up, down moves; columns in order; rows in order).
 *   out_host : host, max_pairs x max_vals, zero-filled beyond each pair's stored values (values
 *              below 1e-14 s_1 are not stored).
 *   *n_pairs : the number of pairs of the iteration.
 * CTM_ERR_STATE if that iteration has not run.  Synchronises the stream of the last call. */
int ctm_get_spectra(ctm_handle* h, int iter, double* out_host, int max_pairs, int max_vals, int* n_pairs);

/* Forward pass of the warm-start network: an MLP that maps the flattened site tensors to an
 * initial environment, so that the CTMRG iterations of Sec. SLF (step ii) start near their
 * fixed point.  The paper has no counterpart (it starts from a fixed environment); the network
 * and its training live in paper_2512_14414_gb300/warmstart.py.
 *   x    : device, FP32, batch x dims[0] (row-major).
 *   W[k] : device, FP32, dims[k+1] x dims[k] row-major (torch.nn.Linear layout), k < n_layers;
 *          W itself is a HOST array of device pointers.
 *   b[k] : device, FP32, dims[k+1] entries, or b == NULL (no biases).
 *   work : device, FP32, at least 2 * batch * max(dims[1..n_layers-1]) floats (caller-owned).
 *   y    : device, FP32, batch x dims[n_layers].
 * Hidden layers apply GELU (exact, erf form) after the bias; the last layer is linear.
 * 1 <= n_layers <= 16.  Enqueued on the stream; no allocation. */
int ctm_mlp_forward(const float* x, int batch, int n_layers, const int* dims, const float* const* W,
                    const float* const* b, float* work, float* y, void* stream);

/* Work size (FP32 elements) that ctm_mlp_backward needs for this network and batch; -1 on bad
 * arguments (same limits as ctm_mlp_forward). */
int64_t ctm_mlp_work_floats(int batch, int n_layers, const int* dims);

/* Gradient of the warm-start network's training loss, the mean-squared error
 *     L = sum (y - target)^2 / (batch * dims[n_layers]),  y = the forward pass of ctm_mlp_forward,
 * by the chain rule layer by layer: the forward pass is recomputed keeping each hidden layer's
 * pre-activation z_k, then dL/dz_L = 2 (y - target) / (batch * n_out), dW_k = (dL/dz_k)^t h_k,
 * db_k = sum over the batch of dL/dz_k, dL/dh_k = dL/dz_k W_k and
 * dL/dz_{k-1} = dL/dh_k * GELU'(z_{k-1}) with GELU'(z) = Phi(z) + z phi(z) (exact GELU).
 *   x, target : device, FP32, batch x dims[0] and batch x dims[n_layers] (row-major).
 *   W, b      : as ctm_mlp_forward (b == NULL: no biases).
 *   dW[k]     : device, FP32, the shape of W[k] (overwritten); dW is a HOST array of pointers.
 *   db[k]     : device, FP32, dims[k+1] entries (overwritten), or db == NULL; HOST array.
 *   work      : device, FP32, ctm_mlp_work_floats(batch, n_layers, dims) elements (caller-owned).
 *   loss_dev  : device, 1 float receiving L, or NULL.
 * Enqueued on the stream; no allocation.  Training is an offline step: the energy and gradient
 * path never calls it. */
int ctm_mlp_backward(const float* x, const float* target, int batch, int n_layers, const int* dims,
                     const float* const* W, const float* const* b, float* const* dW, float* const* db, float* work,
                     float* loss_dev, void* stream);

/* One Adam step (Kingma & Ba 2015) on n FP32 parameters, all device arrays updated in place:
 *   m = beta1 m + (1 - beta1) g;  v = beta2 v + (1 - beta2) g^2;
 *   p -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * t >= 1 is the step count; 0 <= beta1, beta2 < 1. */
int ctm_adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                  float eps, int t, void* stream);

int ctm_destroy(ctm_handle* h);
const char* ctm_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* CTM_H */
