// The nested single-layer CTMRG of arXiv:2512.14414 (Sec. SLF) on the engine of engine.h,
// and the C ABI of include/ctm.h.
//
// Network.  Per PEPS site the nested cell is [A  Y; X  A*] (ket at even row /
// even column, Y at even/odd, X at odd/even, bra at odd/odd; Fig. 2(c)).  The
// crossing tensors X and Y (Eq. XY) are never stored: they only identify
// labels.  X passes its left label to its right and its up label to its
// down; Y passes (i, s) on its left to i on its right and s down, and its up
// label k to its down leg (k, s).  So the ket's right leg is (r, s) and the
// bra's up leg is (u, s), the two D*d bonds of the paper's footnote on bond
// dimensions; every contraction below is a pairwise labelled contraction
// (permute + batched GEMM) over the stored tensors A and the environment.
//
// CTMRG (Fig. 3).  Every nested site owns 4 corners and 4 edges.  A left move
// runs over the columns j in order: for every row i the 2x2 cluster of sites
// (i..i+1, j..j+1) with their environments gives the upper half N (rows: the
// open right cut, columns: the left cut where P Q^t is inserted) and the lower
// half S; the projectors of all rows come first (Eqs. PQ, QRSVD), then every
// row absorbs column j into the left corner, edge and corner of (i, j+1).  The
// right, up and down moves are left moves in the frame rotated by 180, 90 and
// 270 degrees (counterclockwise); a rotation by q maps frame leg f to actual
// leg (f + q) mod 4 (order left, up, right, down) and frame slot k to actual
// slot (k + 2q) mod 8 (ring order C_ul, T_u, C_ur, T_r, C_dr, T_d, C_dl, T_l).
//
// Projectors.  With rho = N S^t, QR + SVD give P = S^t V' L~^{-1/2} and
// Q = N^t U' L~^{-1/2} where U' L V'^t is the thin SVD of rho: for a tall N
// (more right-cut rows than left-cut columns) U' = Q_n U, V' = Q_s V with
// R_n R_s^t = U L V^t (Householder QR); otherwise Q_n is square and the SVD
// is taken of rho itself, which is the same matrix up to that rotation.
// L~^{-1/2} := 0 below cutoff * L_1.  The reverse mode is the adjoint of the
// thin SVD of rho over its numerically non-zero singular values with the
// Lorentzian-broadened 1/(s_j^2 - s_i^2) (no inverse of R is ever formed).
//
// Gradient.  Forward iterations keep no tape: they store the environment at
// the start of every iteration and the factors U', V', L of every projector
// pair.  The backward pass recomputes one iteration at a time from its stored
// environment, taking P and Q from the stored factors (bit-identical to the
// forward), and back-propagates through it (Eq. AD).
#include <array>
#include <cmath>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "engine.h"

namespace ctm {
namespace {

enum Kind { KET = 0, YS = 1, XS = 2, BRA = 3 };
inline int kind_of(int i, int j) { return (i % 2 == 0) ? ((j % 2 == 0) ? KET : YS) : ((j % 2 == 0) ? XS : BRA); }

// ------------------------------------------------------------------ labels with identification
struct Net {
  std::vector<int> par;
  std::vector<int64_t> dim;
  int make(int64_t d) {
    par.push_back((int)par.size());
    dim.push_back(d);
    return (int)par.size() - 1;
  }
  int find(int x) {
    while (par[x] != x) x = par[x] = par[par[x]];
    return x;
  }
  void unify(int a, int b) {
    a = find(a);
    b = find(b);
    CTM_CHECK(dim[a] == dim[b], CTM_ERR_INVALID_ARG, "bond dimension mismatch in network");
    if (a != b) par[b] = a;
  }
  Labels res(const Labels& l) {
    Labels r;
    for (int x : l) r.push_back(find(x));
    return r;
  }
};

// A nested site placed in a network: its four legs (actual order L, U, R, D) as label lists.
struct Pos {
  int site = 0, kind = 0, peps = 0, q = 0;
  std::array<Labels, 4> leg;
  Labels tl;          // labels of the stored tensor A[s][l][u][r][d] (ket/bra only)
  int s_ket = -1, s_bra = -1;  // open physical labels of an impurity Y
  const Labels& frame(int f) const { return leg[(f + q) % 4]; }
};

struct Item {
  Tensor t;
  Labels l;
};

}  // namespace
}  // namespace ctm

// ==================================================================== handle
struct ctm_handle {
  ctm_desc d{};
  struct TermH {
    int x, y, kind;
    double coup;
    std::vector<double> h;
  };
  std::vector<TermH> terms;
  int R = 0, C = 0, nsites = 0;
  ctm::DType edt = ctm::F64;
  double cut = 1e-6, eps = 1e-24;
  double rank_tol = 1e-13;  // triplets below rank_tol * s_1 are left out of the adjoint's core
  int64_t launches = 0;
  cudaStream_t st = nullptr;
  std::unique_ptr<ctm::Arena> persist, tape, store;
  std::unique_ptr<ctm::Engine> eng;
  bool dev_ready = false, inited = false;
  // persistent device state
  ctm::Tensor A64, Amode;                          // site tensors
  std::vector<std::array<ctm::Tensor, 8>> slots;   // environment slot buffers (edt)
  std::vector<std::array<ctm::Tensor, 8>> env;     // current environment values
  std::vector<std::array<ctm::Tensor, 8>> denv;    // environment cotangents (edt)
  double* env0 = nullptr;                          // FP64 copy of the initial environment
  std::vector<std::vector<std::array<ctm::Tensor, 8>>> ckpt;  // environment at the start of each iteration
  struct Fac {
    double *U = nullptr, *V = nullptr, *lam = nullptr;  // U, V: n_r x rs row-major; lam: rs
    int64_t n_r = 0;
    int r = 0;   // min(n_r, n_l): rank bound of rho
    int rs = 0;  // singular triplets stored (r, or the sketch width l)
  };
  std::vector<std::vector<Fac>> fac;  // [iteration][projector pair]
  std::vector<int> rank_hint;         // [projector pair] numerical rank of rho in the previous iteration (0: unknown)
  // Side streams for the independent rows of a column step (fork from / join into st).
  static constexpr int kRowStreams = 4;
  cudaStream_t row_st[kRowStreams] = {};
  cudaEvent_t row_ev[kRowStreams] = {};
  cudaEvent_t fork_ev = nullptr;
  int iters_done = 0;
  int* dstatus = nullptr;
  int* dsweeps = nullptr;
  double* dscal = nullptr;  // [0] delta
  double *hs = nullptr, *coup = nullptr;
  std::string last_error;
  ctm::Profiler prof;
  ctm::Limits limits;  // sweep and spin limits of the iterative kernels (ctm_set_limits)
  // replay state of the current iteration (backward recompute)
  bool replay = false;
  int cur_iter = 0, cur_pair = 0;
  bool debug_sweeps = getenv("CTM_DEBUG_SWEEPS") != nullptr;
};

namespace ctm {
namespace {

// ------------------------------------------------------------------ geometry helpers
inline void to_actual(int q, int R, int C, int fi, int fj, int& i, int& j) {
  switch (q & 3) {
    case 0: i = fi; j = fj; break;
    case 1: i = fj; j = C - 1 - fi; break;
    case 2: i = R - 1 - fi; j = C - 1 - fj; break;
    default: i = R - 1 - fj; j = fi; break;
  }
}

inline int mod(int a, int n) { return ((a % n) + n) % n; }

struct Frame {
  ctm_handle* h;
  int q, FR, FC;
  Frame(ctm_handle* hh, int qq) : h(hh), q(qq) {
    FR = (q % 2 == 0) ? h->R : h->C;
    FC = (q % 2 == 0) ? h->C : h->R;
  }
  int site(int fi, int fj) const {
    int i, j;
    to_actual(q, h->R, h->C, mod(fi, FR), mod(fj, FC), i, j);
    return i * h->C + j;
  }
  int slot(int fk) const { return (fk + 2 * q) % 8; }
  Tensor& env(int s, int fk) const { return h->env[s][slot(fk)]; }
};

// elementary dims of the actual legs of a nested site
std::array<std::vector<int64_t>, 4> leg_dims(int kind, int64_t D, int64_t d) {
  std::array<std::vector<int64_t>, 4> r;
  for (auto& x : r) x = {D};
  if (kind == KET) r[2] = {D, d};
  if (kind == YS) r[0] = {D, d}, r[3] = {D, d};
  if (kind == BRA) r[1] = {D, d};
  return r;
}

Pos make_pos(ctm_handle* h, Net& net, int site, int q, bool impurity) {
  Pos p;
  p.site = site;
  p.q = q;
  int i = site / h->C, j = site % h->C;
  p.kind = kind_of(i, j);
  p.peps = (i / 2) * h->d.Lx + (j / 2);
  const int64_t D = h->d.D, d = h->d.d;
  switch (p.kind) {
    case KET: {
      int s = net.make(d), a = net.make(D), b = net.make(D), c = net.make(D), e = net.make(D);
      p.leg = {Labels{a}, Labels{b}, Labels{c, s}, Labels{e}};
      p.tl = {s, a, b, c, e};
      break;
    }
    case BRA: {
      int s = net.make(d), a = net.make(D), b = net.make(D), c = net.make(D), e = net.make(D);
      p.leg = {Labels{a}, Labels{b, s}, Labels{c}, Labels{e}};
      p.tl = {s, a, b, c, e};
      break;
    }
    case XS: {
      int a = net.make(D), b = net.make(D);
      p.leg = {Labels{a}, Labels{b}, Labels{a}, Labels{b}};
      break;
    }
    default: {
      int a = net.make(D), b = net.make(D);
      if (impurity) {
        int s1 = net.make(d), s2 = net.make(d);
        p.leg = {Labels{a, s1}, Labels{b}, Labels{a}, Labels{b, s2}};
        p.s_ket = s1;
        p.s_bra = s2;
      } else {
        int s = net.make(d);
        p.leg = {Labels{a, s}, Labels{b}, Labels{a}, Labels{b, s}};
      }
    }
  }
  return p;
}

// identify the frame leg fa of A with the frame leg fb of B
void bond(Net& net, const Pos& A, int fa, const Pos& B, int fb) {
  const Labels& x = A.frame(fa);
  const Labels& y = B.frame(fb);
  CTM_CHECK(x.size() == y.size(), CTM_ERR_INVALID_ARG, "bond structure mismatch");
  for (size_t k = 0; k < x.size(); ++k) net.unify(x[k], y[k]);
}

enum { FL = 0, FU = 1, FR = 2, FD = 3 };
enum { S_CUL = 0, S_TU = 1, S_CUR = 2, S_TR = 3, S_CDR = 4, S_TD = 5, S_CDL = 6, S_TL = 7 };

Labels cat(std::initializer_list<Labels> ls) {
  Labels r;
  for (auto& l : ls) r.insert(r.end(), l.begin(), l.end());
  return r;
}

Labels natural_out(const Labels& a, const Labels& b) {
  Labels r;
  for (int x : a)
    if (std::find(b.begin(), b.end(), x) == b.end()) r.push_back(x);
  for (int x : b)
    if (std::find(a.begin(), a.end(), x) == a.end()) r.push_back(x);
  return r;
}

int64_t numel_of(const Labels& l, Net& net) {
  int64_t n = 1;
  for (int x : l) n *= net.dim[x];
  return n;
}

// Greedy pairwise contraction: always the connected pair with the smallest result.
Item contract_greedy(Engine& E, Net& net, std::vector<Item> items, const Labels* out = nullptr) {
  CTM_CHECK(!items.empty(), CTM_ERR_INVALID_ARG, "empty contraction");
  while (items.size() > 1) {
    int bp = -1, bq = -1;
    int64_t bsize = 0, bcost = 0;
    for (size_t p = 0; p < items.size(); ++p)
      for (size_t q = p + 1; q < items.size(); ++q) {
        Labels o = natural_out(items[p].l, items[q].l);
        size_t shared = items[p].l.size() + items[q].l.size() - o.size();
        if (shared == 0) continue;
        int64_t size = numel_of(o, net);
        int64_t cost = size;
        for (int x : items[p].l)
          if (std::find(items[q].l.begin(), items[q].l.end(), x) != items[q].l.end()) cost *= net.dim[x];
        if (bp < 0 || size < bsize || (size == bsize && cost < bcost)) {
          bp = (int)p;
          bq = (int)q;
          bsize = size;
          bcost = cost;
        }
      }
    if (bp < 0) {  // no connected pair left: outer product of the first two
      bp = 0;
      bq = 1;
    }
    Labels o = natural_out(items[bp].l, items[bq].l);
    if (items.size() == 2 && out) o = *out;
    Item r{E.einsum(items[bp].t, items[bp].l, items[bq].t, items[bq].l, o), o};
    std::vector<Item> nx;
    for (size_t k = 0; k < items.size(); ++k)
      if ((int)k != bp && (int)k != bq) nx.push_back(items[k]);
    nx.push_back(r);
    items.swap(nx);
  }
  if (out && items[0].l != *out) {
    // single item whose order differs: permute
    std::vector<int> perm;
    for (int x : *out) perm.push_back((int)(std::find(items[0].l.begin(), items[0].l.end(), x) - items[0].l.begin()));
    items[0].t = E.permute(items[0].t, perm);
    items[0].l = *out;
  }
  return items[0];
}

void sync_status(ctm_handle* h) {
  int s = 0;
  CTM_CUDA(cudaMemcpyAsync(&s, h->dstatus, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CTM_CUDA(cudaStreamSynchronize(h->st));
  if (s) {
    CTM_CUDA(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
    if (s & DEV_TIMEOUT) throw Error(CTM_ERR_TIMEOUT, "device wait timed out");
    if (s & DEV_SVD_NOCONV) throw Error(CTM_ERR_SVD_NOCONV, "Jacobi SVD did not converge");
    if (s & DEV_NONFINITE) throw Error(CTM_ERR_NONFINITE, "non-finite value in spectrum or energy");
    if (s & DEV_DEGENERATE) throw Error(CTM_ERR_DEGENERATE, "all singular values zero");
  }
}

}  // namespace
}  // namespace ctm

using namespace ctm;

// ==================================================================== per-site tensors of A
// Amode is one buffer of Lx*Ly site tensors; a leaf per site lets einsum accumulate each
// site's gradient into its own sub-buffer.
namespace ctm {
namespace {

struct SiteLeaves {
  std::vector<Tensor> t;  // one per PEPS site (views into Amode)
};

SiteLeaves site_views(ctm_handle* h, bool leaves) {
  SiteLeaves s;
  int64_t per = (int64_t)h->d.d * h->d.D * h->d.D * h->d.D * h->d.D;
  for (int p = 0; p < h->d.Lx * h->d.Ly; ++p) {
    Tensor a;
    a.dt = h->Amode.dt;
    a.p = (char*)h->Amode.p + per * p * dtype_size(a.dt);
    a.dims = {h->d.d, h->d.D, h->d.D, h->d.D, h->d.D};
    s.t.push_back(leaves ? h->eng->leaf(a) : a);
  }
  return s;
}

thread_local SiteLeaves* g_sites = nullptr;

void push_site(std::vector<Item>& v, Net& net, const Pos& p) {
  if (p.kind == KET || p.kind == BRA) v.push_back({g_sites->t[p.peps], net.res(p.tl)});
}

Item env_item(const Frame& F, Net& net, int s, int fk, const Labels& prev, const Labels& in, const Labels& next) {
  Tensor t = F.env(s, fk);
  return {t, net.res(cat({prev, in, next}))};
}

// ------------------------------------------------------------------ projector op
struct PairIn {
  Tensor N, S;          // edt, [right cut..., left cut...]
  int64_t n_r, n_l;
  std::vector<int64_t> pdims, qdims;  // dims of P and Q tensors [chi, b..., chi]
};

// Full factorisation of rho = N S^t for every pair of the batch (svd_product_full): Householder
// QR of S (tall pairs) and of X = N S^t Q_s, one-sided Jacobi on the rows of the triangular factor.
// Stores all r singular triplets.
void projectors_full(ctm_handle* h, const std::vector<PairIn>& in, const std::vector<Tensor>& N64,
                     const std::vector<Tensor>& S64, std::vector<ctm_handle::Fac*>& F, int r) {
  Engine& E = *h->eng;
  cudaStream_t st = h->st;
  const int nb = (int)in.size();
  std::vector<const double*> Np(nb), Sp(nb);
  std::vector<double*> Up(nb), Vp(nb);
  std::vector<int> nrs(nb), nls(nb);
  int nrmax = 0, nlmax = 0;
  for (int b = 0; b < nb; ++b) {
    Np[b] = (const double*)N64[b].p;
    Sp[b] = (const double*)S64[b].p;
    nrs[b] = (int)in[b].n_r;
    nls[b] = (int)in[b].n_l;
    nrmax = std::max(nrmax, nrs[b]);
    nlmax = std::max(nlmax, nls[b]);
    Up[b] = F[b]->U;
    Vp[b] = F[b]->V;
  }
  double* ws = (double*)E.arena().alloc(svd_product_full_ws(nb, nrmax, nlmax, r));
  double* lam = (double*)E.arena().alloc(sizeof(double) * nb * r);
  std::vector<int> rk;
  svd_product_full(Np.data(), Sp.data(), nrs.data(), nls.data(), nb, r, ws, lam, Up.data(), Vp.data(), h->dstatus,
                   h->dsweeps, rk, st);
  auto& hint = h->rank_hint;
  for (int b = 0; b < nb; ++b) {
    F[b]->rs = r;
    CTM_CUDA(cudaMemcpyAsync(F[b]->lam, lam + (int64_t)b * r, sizeof(double) * r, cudaMemcpyDeviceToDevice, st));
    hint[h->cur_pair + b] = std::max(rk[b], 1);
  }
}

void projectors(ctm_handle* h, std::vector<PairIn>& in, std::vector<Tensor>& P, std::vector<Tensor>& Q) {
  Engine& E = *h->eng;
  cudaStream_t st = h->st;
  const int chi = h->d.chi;
  const int nb = (int)in.size();
  P.assign(nb, Tensor());
  Q.assign(nb, Tensor());
  // per-row FP64 operands
  std::vector<Tensor> N64(nb), S64(nb);
  for (int b = 0; b < nb; ++b) {
    Tensor n2 = in[b].N, s2 = in[b].S;
    n2.dims = {in[b].n_r, in[b].n_l};
    s2.dims = {in[b].n_r, in[b].n_l};
    N64[b] = (n2.dt == F64) ? n2 : E.cast(n2, F64);
    S64[b] = (s2.dt == F64) ? s2 : E.cast(s2, F64);
    N64[b].id = S64[b].id = -1;  // gradients are routed by hand below
  }
  int r = (int)std::min(in[0].n_r, in[0].n_l);
  for (auto& x : in) CTM_CHECK(std::min(x.n_r, x.n_l) == r, CTM_ERR_INVALID_ARG, "projector rank size differs");
  const int kept = std::min(chi, r);
  auto& fac = h->fac[h->cur_iter];
  if ((int)fac.size() < h->cur_pair + nb) fac.resize(h->cur_pair + nb);
  std::vector<ctm_handle::Fac*> F(nb);
  for (int b = 0; b < nb; ++b) {
    F[b] = &fac[h->cur_pair + b];
    if (!F[b]->U) {
      F[b]->n_r = in[b].n_r;
      F[b]->r = r;
      F[b]->U = (double*)h->store->alloc(sizeof(double) * in[b].n_r * r);
      F[b]->V = (double*)h->store->alloc(sizeof(double) * in[b].n_r * r);
      F[b]->lam = (double*)h->store->alloc(sizeof(double) * r);
    }
  }
  if (!h->replay) {
    // Truncated SVD through a sketch of width l (Sec. Outlook: partial / randomised
    // decompositions in Eq. QRSVD) taken directly on the product rho = N S^t; exact whenever
    // the numerical rank of rho is below l, which is checked per matrix -- otherwise the full
    // QR + Jacobi factorisation runs for the whole batch.
    // Width: the pair's numerical rank in the previous iteration plus a margin (chi + 16 when
    // unknown); doubled once when the sketch misses the floor.
    auto& hint = h->rank_hint;
    if ((int)hint.size() < h->cur_pair + nb) hint.resize(h->cur_pair + nb, 0);
    int l = std::min(r, std::max(chi + 16, 32));
    bool sketched = false;
    if (h->debug_sweeps) CTM_CUDA(cudaMemsetAsync(h->dsweeps, 0, sizeof(int), st));
    // all pairs of the column step in one batch (different n_r are padded inside the sketch)
    {
      int hmax = 0, nrmax = 0;
      bool known = true;
      std::vector<int> nrs(nb), nls(nb);
      for (int b = 0; b < nb; ++b) {
        hmax = std::max(hmax, hint[h->cur_pair + b]);
        known = known && hint[h->cur_pair + b] > 0;
        nrs[b] = (int)in[b].n_r;
        nls[b] = (int)in[b].n_l;
        nrmax = std::max(nrmax, nrs[b]);
      }
      int nlmax = *std::max_element(nls.begin(), nls.end());
      l = known ? std::min(r, std::max(16, (hmax + 12 + 7) / 8 * 8)) : std::min(r, std::max(chi + 16, 32));
      std::vector<const double*> Np(nb), Sp(nb);
      for (int b = 0; b < nb; ++b) Np[b] = (const double*)N64[b].p, Sp[b] = (const double*)S64[b].p;
      // The test matrix is random: a sketch started from the previous iteration's singular vectors
      // can carry numerically null directions of the new rho (old tail vectors) whose tiny Ritz
      // values would pass the exactness test below although the sketch misses part of the range.
      std::vector<const double*> Wp(nb, nullptr);
      const int kw = 0, ldw = 0;
      bool ok = false;
      for (int attempt = 0; attempt < 2 && !ok && 2 * l <= r; ++attempt) {
        double* ws = (double*)E.arena().alloc(svd_sketch_product_ws(nb, nrmax, nlmax, l));
        double* lam = (double*)E.arena().alloc(sizeof(double) * nb * l);
        double* Uo = (double*)E.arena().alloc(sizeof(double) * nb * (int64_t)nrmax * l);
        double* Vo = (double*)E.arena().alloc(sizeof(double) * nb * (int64_t)nrmax * l);
        std::vector<int> inc, rk;
        const int kwa = std::min(kw, l - 8);
        svd_sketch_product(Np.data(), Sp.data(), nrs.data(), nls.data(), nb, l, kwa > 0 ? Wp.data() : nullptr, ldw,
                           std::max(kwa, 0), ws, lam, Uo, Vo, h->dstatus, h->dsweeps, inc, rk, st);
        // exact when the sketch's smallest Ritz value is at the rounding floor and at least 8 of the
        // l directions are numerically null (the range of rho fits with room to spare)
        ok = true;
        for (int x : inc) ok = ok && x == 0;
        for (int x : rk) ok = ok && x <= l - 8;
        if (!ok) {
          l *= 2;
          continue;
        }
        for (int b = 0; b < nb; ++b) {
          ctm_handle::Fac* f = F[b];
          f->rs = l;
          hint[h->cur_pair + b] = rk[b];
          const size_t nb_uv = sizeof(double) * (size_t)nrs[b] * l;  // the first n_r rows of the padded block
          CTM_CUDA(cudaMemcpyAsync(f->lam, lam + (int64_t)b * l, sizeof(double) * l, cudaMemcpyDeviceToDevice, st));
          CTM_CUDA(cudaMemcpyAsync(f->U, Uo + (int64_t)b * nrmax * l, nb_uv, cudaMemcpyDeviceToDevice, st));
          CTM_CUDA(cudaMemcpyAsync(f->V, Vo + (int64_t)b * nrmax * l, nb_uv, cudaMemcpyDeviceToDevice, st));
        }
      }
      sketched = ok;
    }
    if (!sketched) projectors_full(h, in, N64, S64, F, r);
    if (h->debug_sweeps) {
      int sw = 0;
      CTM_CUDA(cudaMemcpyAsync(&sw, h->dsweeps, sizeof(int), cudaMemcpyDeviceToHost, st));
      CTM_CUDA(cudaStreamSynchronize(st));
      int rk_floor = 0, rk_cut = 0;  // largest numerical rank (1e-14) and kept count (cutoff) of the batch
      std::string kept_list;
      for (int b = 0; b < nb; ++b) {
        std::vector<double> lh(F[b]->rs);
        CTM_CUDA(cudaMemcpy(lh.data(), F[b]->lam, sizeof(double) * lh.size(), cudaMemcpyDeviceToHost));
        int a = 0, c = 0;
        for (double v : lh) a += v > 1e-14 * lh[0], c += v > h->cut * lh[0];
        rk_floor = std::max(rk_floor, a);
        rk_cut = std::max(rk_cut, c);
        kept_list += " " + std::to_string(c);
        // distance of the nearest singular value to the cutoff, in units of the cutoff
        double near = 1e300;
        for (double v : lh) near = std::min(near, std::fabs(v / lh[0] / h->cut - 1.0));
        kept_list += "(" + std::to_string(near).substr(0, 6) + ")";
      }
      fprintf(stderr, "libctm: iteration %d pairs %d..%d r=%d %s l=%d Jacobi sweeps %d rank %d above cutoff %d kept%s\n",
              h->cur_iter, h->cur_pair, h->cur_pair + nb - 1, r, sketched ? "sketch" : "full", l, sw, rk_floor, rk_cut,
              kept_list.c_str());
    }
    // Sign gauge of the singular triplets.  With the previous iteration's factors of the same pair at
    // hand, each kept right vector takes the sign of its overlap with the previous one, so that a
    // converged environment is reproduced entry by entry (the fixed point that ctm_grad_fixed_point
    // differentiates); otherwise the entry of largest magnitude is made positive.  Both rules are
    // locally constant, so the derivative ignores them.
    for (int b = 0; b < nb; ++b) {
      sign_fix(F[b]->U, F[b]->V, 1, in[b].n_r, F[b]->rs, st);
      if (h->cur_iter >= 1 && (int)h->fac[h->cur_iter - 1].size() > h->cur_pair + b) {
        const ctm_handle::Fac& pv = h->fac[h->cur_iter - 1][h->cur_pair + b];
        if (pv.V && pv.n_r == in[b].n_r)
          sign_align(F[b]->U, F[b]->V, F[b]->rs, pv.V, pv.rs, in[b].n_r,
                     std::min<int>((int)chi, std::min(F[b]->rs, pv.rs)), st);
      }
    }
  }
  // P = S^t V' L^-1/2, Q = N^t U' L^-1/2 (identical in forward and replay)
  struct Saved {
    double *inv, *sinv, *Wp, *Zp;
  };
  std::vector<Saved> sv(nb);
  for (int b = 0; b < nb; ++b) {
    const int64_t nr = in[b].n_r, nl = in[b].n_l;
    Saved& s = sv[b];
    const int rs = F[b]->rs;
    const int kb = std::min(kept, rs);  // triplets beyond the stored ones are below the rank floor
    s.inv = (double*)E.arena().alloc(sizeof(double) * kb);
    s.sinv = (double*)E.arena().alloc(sizeof(double) * rs);
    s.Wp = (double*)E.arena().alloc(sizeof(double) * nr * kb);
    s.Zp = (double*)E.arena().alloc(sizeof(double) * nr * kb);
    proj_prepare(F[b]->lam, F[b]->U, F[b]->V, s.inv, s.sinv, 1, nr, rs, kb, h->cut, h->rank_tol, h->dstatus, st);
    scale_cols(F[b]->V, rs, 0, s.inv, 0, s.Wp, 1, nr, kb, st);
    scale_cols(F[b]->U, rs, 0, s.inv, 0, s.Zp, 1, nr, kb, st);
    Tensor P64 = E.zeros(F64, {nl, (int64_t)chi});
    Tensor Q64 = E.zeros(F64, {nl, (int64_t)chi});
    GemmSpec g;
    g.M = nl; g.N = kb; g.K = nr; g.transA = true; g.lda = nl; g.transB = false; g.ldb = kb; g.ldc = chi;
    gemm_f64((const double*)S64[b].p, s.Wp, (double*)P64.p, g, st);
    gemm_f64((const double*)N64[b].p, s.Zp, (double*)Q64.p, g, st);
    P64.dims = in[b].pdims;
    Q64.dims = in[b].qdims;
    P[b] = (h->edt == F64) ? P64 : E.cast(P64, h->edt);
    Q[b] = (h->edt == F64) ? Q64 : E.cast(Q64, h->edt);
    P[b].id = Q[b].id = -1;
  }
  h->cur_pair += nb;
  if (!E.recording()) return;
  // ---- reverse mode of (N, S) -> (P, Q)
  bool any = false;
  for (auto& x : in) any = any || x.N.id >= 0 || x.S.id >= 0;
  if (!any) return;
  std::vector<int> pid(nb), qid(nb);
  for (int b = 0; b < nb; ++b) {
    P[b].id = pid[b] = E.new_id(P[b]);
    Q[b].id = qid[b] = E.new_id(Q[b]);
  }
  std::vector<ctm_handle::Fac> Fc(nb);
  for (int b = 0; b < nb; ++b) Fc[b] = *F[b];
  std::vector<PairIn> inc = in;
  std::vector<Tensor> Pc = P, Qc = Q;
  const double eps = h->eps, rank_tol = h->rank_tol;
  const DType edt = h->edt;
  ctm_handle* hh = h;
  E.push([hh, &E, inc, N64, S64, Fc, sv, Pc, Qc, kept, chi, eps, rank_tol, edt, st]() {
    for (size_t b = 0; b < inc.size(); ++b) {
      void* gP = E.grad(Pc[b], false);
      void* gQ = E.grad(Qc[b], false);
      if (!gP && !gQ) continue;
      const int64_t nr = inc[b].n_r, nl = inc[b].n_l;
      const int rs = Fc[b].rs;
      const int kb = std::min(kept, rs);
      auto A64 = [&](int64_t n) { return (double*)E.arena().alloc(sizeof(double) * std::max<int64_t>(n, 1)); };
      double* dP = A64(nl * chi);
      double* dQ = A64(nl * chi);
      if (gP) cast(gP, edt, dP, F64, nl * chi, false, st); else fill(dP, F64, nl * chi, 0.0, st);
      if (gQ) cast(gQ, edt, dQ, F64, nl * chi, false, st); else fill(dQ, F64, nl * chi, 0.0, st);
      const double* N = (const double*)N64[b].p;
      const double* S = (const double*)S64[b].p;
      const double* U = Fc[b].U;
      const double* V = Fc[b].V;
      const double* lam = Fc[b].lam;
      double* dN = A64(nr * nl);
      double* dS = A64(nr * nl);
      double* dW = A64(nr * kb);
      double* dZ = A64(nr * kb);
      GemmSpec g;
      // dS = W dP^t, dN = Z dQ^t  (n_r x n_l, K = kb; dP has leading dimension chi)
      g.M = nr; g.N = nl; g.K = kb; g.transA = false; g.lda = kb; g.transB = true; g.ldb = chi; g.ldc = nl;
      gemm_f64(sv[b].Wp, dP, dS, g, st);
      gemm_f64(sv[b].Zp, dQ, dN, g, st);
      // dW = S dP, dZ = N dQ (n_r x kb)
      g = GemmSpec();
      g.M = nr; g.N = kb; g.K = nl; g.transA = false; g.lda = nl; g.transB = false; g.ldb = chi; g.ldc = kb;
      gemm_f64(S, dP, dW, g, st);
      gemm_f64(N, dQ, dZ, g, st);
      double* dUk = A64(nr * kb);
      double* dVk = A64(nr * kb);
      double* dl = A64(kb);
      scale_cols(dZ, kb, 0, sv[b].inv, 0, dUk, 1, nr, kb, st);
      scale_cols(dW, kb, 0, sv[b].inv, 0, dVk, 1, nr, kb, st);
      proj_dlam(dZ, U, dW, V, sv[b].inv, dl, 1, nr, rs, kb, st);
      double* Aa = A64((int64_t)rs * kb);
      double* Bb = A64((int64_t)rs * kb);
      g = GemmSpec();
      g.M = rs; g.N = kb; g.K = nr; g.transA = true; g.lda = rs; g.transB = false; g.ldb = kb; g.ldc = kb;
      gemm_f64(U, dUk, Aa, g, st);
      gemm_f64(V, dVk, Bb, g, st);
      double* core = A64((int64_t)rs * rs);
      proj_core(Aa, Bb, lam, dl, core, 1, rs, kb, rank_tol, eps, st);
      double* Xu = A64(nr * kb);
      double* Xv = A64(nr * kb);
      g = GemmSpec();
      g.M = nr; g.N = kb; g.K = rs; g.lda = rs; g.ldb = kb; g.ldc = kb;
      gemm_f64(U, Aa, Xu, g, st);
      gemm_f64(V, Bb, Xv, g, st);
      double* Eu = A64(nr * kb);
      double* Ev = A64(nr * kb);
      proj_resid(dUk, Xu, sv[b].sinv, Eu, 1, nr, rs, kb, st);
      proj_resid(dVk, Xv, sv[b].sinv, Ev, 1, nr, rs, kb, st);
      // drho = U core V^t + Eu V_k^t + U_k Ev^t is never formed (n_r x n_r).  core vanishes
      // outside its first kb rows and columns (only kept triplets carry a cotangent), so
      //   U core V^t = U_k Y0^t + Z0 V_k^t,  Y0 = V core[:kb, :]^t,  Z0 = U core[:, :kb] - U_k core[:kb, :kb],
      // and with Y = Y0 + Ev, Z = Z0 + Eu (n_r x kb) drho = U_k Y^t + Z V_k^t has rank <= 2 kb:
      //   dN += drho S   = U_k (Y^t S) + Z (V_k^t S)
      //   dS += drho^t N = Y (U_k^t N) + V_k (Z^t N)
      double* Y = Ev;
      double* Z = Eu;
      g = GemmSpec();
      g.M = nr; g.N = kb; g.K = rs; g.lda = rs; g.transB = true; g.ldb = rs; g.ldc = kb; g.beta = 1.0;
      gemm_f64(V, core, Y, g, st);
      g = GemmSpec();
      g.M = nr; g.N = kb; g.K = rs; g.lda = rs; g.ldb = rs; g.ldc = kb; g.beta = 1.0;
      gemm_f64(U, core, Z, g, st);
      g.K = kb; g.alpha = -1.0;
      gemm_f64(U, core, Z, g, st);
      double* YtS = A64((int64_t)kb * nl);
      double* VtS = A64((int64_t)kb * nl);
      double* UtN = A64((int64_t)kb * nl);
      double* ZtN = A64((int64_t)kb * nl);
      g = GemmSpec();
      g.M = kb; g.N = nl; g.K = nr; g.transA = true; g.lda = kb; g.ldb = nl; g.ldc = nl;
      gemm_f64(Y, S, YtS, g, st);
      gemm_f64(Z, N, ZtN, g, st);
      g.lda = rs;
      gemm_f64(V, S, VtS, g, st);
      gemm_f64(U, N, UtN, g, st);
      g = GemmSpec();
      g.M = nr; g.N = nl; g.K = kb; g.ldb = nl; g.ldc = nl; g.beta = 1.0;
      g.lda = rs;
      gemm_f64(U, YtS, dN, g, st);
      gemm_f64(V, ZtN, dS, g, st);
      g.lda = kb;
      gemm_f64(Z, VtS, dN, g, st);
      gemm_f64(Y, UtN, dS, g, st);
      if (inc[b].N.id >= 0) cast(dN, F64, E.grad(inc[b].N), edt, nr * nl, true, st);
      if (inc[b].S.id >= 0) cast(dS, F64, E.grad(inc[b].S), edt, nr * nl, true, st);
    }
  });
}

// ------------------------------------------------------------------ row streams
// The rows of one column step contract independent networks: each runs on its own side stream,
// forked from the main stream (side streams wait for all work enqueued so far) and joined back
// (the main stream waits for all of them) before anything reads their results.  While forked,
// the engine keeps the temporaries of each contraction (the arena is shared by the streams);
// they are recycled with the column step.  CTM_ROW_STREAMS=0 keeps every row on the main stream.
static bool row_streams_on() {
  static const bool on = []() {
    const char* e = getenv("CTM_ROW_STREAMS");
    return !(e && e[0] == '0');
  }();
  return on;
}

void fork_rows(ctm_handle* h) {
  if (!row_streams_on()) return;
  CTM_CUDA(cudaEventRecord(h->fork_ev, h->st));
  for (int k = 0; k < ctm_handle::kRowStreams; ++k) CTM_CUDA(cudaStreamWaitEvent(h->row_st[k], h->fork_ev, 0));
  h->eng->set_defer_release(true);
}

void use_row_stream(ctm_handle* h, int i) {
  if (row_streams_on()) h->eng->set_stream(h->row_st[i % ctm_handle::kRowStreams]);
}

void join_rows(ctm_handle* h) {
  if (!row_streams_on()) return;
  for (int k = 0; k < ctm_handle::kRowStreams; ++k) {
    CTM_CUDA(cudaEventRecord(h->row_ev[k], h->row_st[k]));
    CTM_CUDA(cudaStreamWaitEvent(h->st, h->row_ev[k], 0));
  }
  h->eng->set_stream(h->st);
  h->eng->set_defer_release(false);
}

// ------------------------------------------------------------------ one left move (in frame q)
void left_move(ctm_handle* h, int q) {
  Engine& E = *h->eng;
  Frame F(h, q);
  const int64_t chi = h->d.chi;
  for (int j = 0; j < F.FC; ++j) {
    auto mark = h->tape->mark();
    std::vector<PairIn> pin(F.FR);
    fork_rows(h);
    for (int i = 0; i < F.FR; ++i) {
      use_row_stream(h, i);
      Net net;
      int s00 = F.site(i, j), s01 = F.site(i, j + 1), s10 = F.site(i + 1, j), s11 = F.site(i + 1, j + 1);
      Pos p00 = make_pos(h, net, s00, q, false), p01 = make_pos(h, net, s01, q, false);
      Pos p10 = make_pos(h, net, s10, q, false), p11 = make_pos(h, net, s11, q, false);
      bond(net, p00, FR, p01, FL);
      bond(net, p10, FR, p11, FL);
      bond(net, p01, FD, p11, FU);
      int x1 = net.make(chi), x2 = net.make(chi), x3 = net.make(chi), x4 = net.make(chi), x5 = net.make(chi);
      int cu = net.make(chi), cl = net.make(chi), cr = net.make(chi);
      int y1 = net.make(chi), y2 = net.make(chi), y3 = net.make(chi), y4 = net.make(chi), y5 = net.make(chi);
      std::vector<Item> gul, gur, gdl, gdr;
      gul.push_back(env_item(F, net, s00, S_CUL, {x1}, {}, {x2}));
      gul.push_back(env_item(F, net, s00, S_TU, {x2}, p00.frame(FU), {x3}));
      gul.push_back(env_item(F, net, s00, S_TL, {cu}, p00.frame(FL), {x1}));
      push_site(gul, net, p00);
      gur.push_back(env_item(F, net, s01, S_TU, {x3}, p01.frame(FU), {x4}));
      gur.push_back(env_item(F, net, s01, S_CUR, {x4}, {}, {x5}));
      gur.push_back(env_item(F, net, s01, S_TR, {x5}, p01.frame(FR), {cr}));
      push_site(gur, net, p01);
      gdl.push_back(env_item(F, net, s10, S_TL, {y1}, p10.frame(FL), {cl}));
      gdl.push_back(env_item(F, net, s10, S_CDL, {y2}, {}, {y1}));
      gdl.push_back(env_item(F, net, s10, S_TD, {y3}, p10.frame(FD), {y2}));
      push_site(gdl, net, p10);
      gdr.push_back(env_item(F, net, s11, S_TD, {y4}, p11.frame(FD), {y3}));
      gdr.push_back(env_item(F, net, s11, S_CDR, {y5}, {}, {y4}));
      gdr.push_back(env_item(F, net, s11, S_TR, {cr}, p11.frame(FR), {y5}));
      push_site(gdr, net, p11);
      Labels rcut = net.res(cat({p01.frame(FD), {cr}}));
      Labels lcutN = net.res(cat({{cu}, p00.frame(FD)}));
      Labels lcutS = net.res(cat({{cl}, p10.frame(FU)}));
      Labels outN = cat({rcut, lcutN}), outS = cat({rcut, lcutS});
      Item Gul = contract_greedy(E, net, gul), Gur = contract_greedy(E, net, gur);
      Item Nn = contract_greedy(E, net, {Gul, Gur}, &outN);
      Item Gdl = contract_greedy(E, net, gdl), Gdr = contract_greedy(E, net, gdr);
      Item Ss = contract_greedy(E, net, {Gdl, Gdr}, &outS);
      PairIn& pi = pin[i];
      pi.N = Nn.t;
      pi.S = Ss.t;
      pi.n_r = numel_of(rcut, net);
      pi.n_l = numel_of(lcutN, net);
      CTM_CHECK(pi.n_l == numel_of(lcutS, net), CTM_ERR_INVALID_ARG, "left cut sizes differ");
      pi.pdims.clear();
      for (int x : lcutN) pi.pdims.push_back(net.dim[x]);
      pi.pdims.push_back(chi);
      pi.qdims.clear();
      for (int x : lcutS) pi.qdims.push_back(net.dim[x]);
      pi.qdims.push_back(chi);
    }
    join_rows(h);
    std::vector<Tensor> P, Q;
    projectors(h, pin, P, Q);
    // absorb column j into the left environment of column j + 1
    std::vector<std::array<Tensor, 3>> nw(F.FR);
    fork_rows(h);
    for (int i = 0; i < F.FR; ++i) {
      use_row_stream(h, i);
      const int im = mod(i - 1, F.FR);
      const int s = F.site(i, j);
      Net net;
      Pos p = make_pos(h, net, s, q, false);
      const Labels U = p.frame(FU), D = p.frame(FD), L = p.frame(FL), Rr = p.frame(FR);
      {  // C_ul' = C_ul T_u P_{i-1}  -> ring [down, right]
        int pc = net.make(chi), r1 = net.make(chi), rr = net.make(chi), kn = net.make(chi);
        std::vector<Item> v;
        v.push_back(env_item(F, net, s, S_CUL, {pc}, {}, {r1}));
        v.push_back(env_item(F, net, s, S_TU, {r1}, U, {rr}));
        v.push_back({P[im], net.res(cat({{pc}, U, {kn}}))});
        Labels o = net.res({kn, rr});
        nw[i][0] = E.normalize(contract_greedy(E, net, v, &o).t);
      }
      {  // T_l' = Q_{i-1} T_l a P_i  -> ring [down, in, up]
        int c1 = net.make(chi), c2 = net.make(chi), up = net.make(chi), dn = net.make(chi);
        std::vector<Item> v;
        v.push_back(env_item(F, net, s, S_TL, {c1}, L, {c2}));
        push_site(v, net, p);
        v.push_back({Q[im], net.res(cat({{c2}, U, {up}}))});
        v.push_back({P[i], net.res(cat({{c1}, D, {dn}}))});
        Labels o = net.res(cat({{dn}, Rr, {up}}));
        nw[i][1] = E.normalize(contract_greedy(E, net, v, &o).t);
      }
      {  // C_dl' = C_dl T_d Q_i -> ring [right, up]
        int c3 = net.make(chi), c4 = net.make(chi), c5 = net.make(chi), un = net.make(chi);
        std::vector<Item> v;
        v.push_back(env_item(F, net, s, S_CDL, {c3}, {}, {c4}));
        v.push_back(env_item(F, net, s, S_TD, {c5}, D, {c3}));
        v.push_back({Q[i], net.res(cat({{c4}, D, {un}}))});
        Labels o = net.res({c5, un});
        nw[i][2] = E.normalize(contract_greedy(E, net, v, &o).t);
      }
    }
    join_rows(h);
    for (int i = 0; i < F.FR; ++i) {
      const int t = F.site(i, j + 1);
      const int ks[3] = {F.slot(S_CUL), F.slot(S_TL), F.slot(S_CDL)};
      for (int k = 0; k < 3; ++k) {
        Tensor v = nw[i][k];
        Tensor& slot = h->slots[t][ks[k]];
        CTM_CHECK(v.numel() == slot.numel(), CTM_ERR_INVALID_ARG, "environment shape changed");
        if (E.recording()) {
          v.dims = slot.dims;
          h->env[t][ks[k]] = v;
        } else {
          CTM_CUDA(cudaMemcpyAsync(slot.p, v.p, v.bytes(), cudaMemcpyDeviceToDevice, h->st));
          h->env[t][ks[k]] = slot;
        }
      }
    }
    if (!E.recording()) h->tape->release(mark);
  }
}

void one_iteration(ctm_handle* h) {
  h->cur_pair = 0;
  for (int q : {0, 2, 1, 3}) left_move(h, q);  // left, right, up, down
}

// ------------------------------------------------------------------ energy
// Blocks (rows x cols of nested sites at (2y, 2x)) and the positions of the two open Y's.
struct BlockSpec {
  int h, w, a1, b1, a2, b2;
};
BlockSpec block_of(int kind) {
  switch (kind) {
    case CTM_BOND_H: return {2, 4, 0, 1, 0, 3};
    case CTM_BOND_V: return {4, 2, 0, 1, 2, 1};
    case CTM_BOND_DIAG_DR: return {4, 4, 0, 1, 2, 3};
    default: return {4, 4, 0, 3, 2, 1};
  }
}

// Reduced density matrix of a bh x bw block of nested sites whose upper-left site is (i0, j0),
// closed by the environment, with the physical line of the Y at every position of `imps` cut
// open (impurity Y's).  Legs of the result: the ket indices of the impurities in order, then
// their bra indices.
Tensor block_rdm(ctm_handle* h, int i0, int j0, int bh, int bw, const std::vector<std::pair<int, int>>& imps) {
  Engine& E = *h->eng;
  Frame F(h, 0);
  const int64_t chi = h->d.chi;
  Net net;
  std::vector<Pos> pos(bh * bw);
  for (int a = 0; a < bh; ++a)
    for (int b = 0; b < bw; ++b) {
      bool imp = false;
      for (auto& x : imps) imp = imp || (x.first == a && x.second == b);
      pos[a * bw + b] = make_pos(h, net, F.site(i0 + a, j0 + b), 0, imp);
    }
  for (int a = 0; a < bh; ++a)
    for (int b = 0; b < bw; ++b) {
      if (b + 1 < bw) bond(net, pos[a * bw + b], FR, pos[a * bw + b + 1], FL);
      if (a + 1 < bh) bond(net, pos[a * bw + b], FD, pos[(a + 1) * bw + b], FU);
    }
  std::vector<int> TU(bw + 1), TD(bw + 1), TL(bh + 1), TR(bh + 1);
  for (auto* v : {&TU, &TD})
    for (auto& x : *v) x = net.make(chi);
  for (auto* v : {&TL, &TR})
    for (auto& x : *v) x = net.make(chi);
  std::map<int, std::vector<Item>> groups;
  auto G = [&](int a, int b) { return (a / 2) * 16 + (b / 2); };
  auto P = [&](int a, int b) -> Pos& { return pos[a * bw + b]; };
  for (int a = 0; a < bh; ++a)
    for (int b = 0; b < bw; ++b) push_site(groups[G(a, b)], net, P(a, b));
  const int H = bh - 1, W = bw - 1;
  groups[G(0, 0)].push_back(env_item(F, net, P(0, 0).site, S_CUL, {TL[0]}, {}, {TU[0]}));
  groups[G(0, W)].push_back(env_item(F, net, P(0, W).site, S_CUR, {TU[bw]}, {}, {TR[0]}));
  groups[G(H, W)].push_back(env_item(F, net, P(H, W).site, S_CDR, {TR[bh]}, {}, {TD[bw]}));
  groups[G(H, 0)].push_back(env_item(F, net, P(H, 0).site, S_CDL, {TD[0]}, {}, {TL[bh]}));
  for (int b = 0; b < bw; ++b) {
    groups[G(0, b)].push_back(env_item(F, net, P(0, b).site, S_TU, {TU[b]}, P(0, b).frame(FU), {TU[b + 1]}));
    groups[G(H, b)].push_back(env_item(F, net, P(H, b).site, S_TD, {TD[b + 1]}, P(H, b).frame(FD), {TD[b]}));
  }
  for (int a = 0; a < bh; ++a) {
    groups[G(a, 0)].push_back(env_item(F, net, P(a, 0).site, S_TL, {TL[a + 1]}, P(a, 0).frame(FL), {TL[a]}));
    groups[G(a, W)].push_back(env_item(F, net, P(a, W).site, S_TR, {TR[a]}, P(a, W).frame(FR), {TR[a + 1]}));
  }
  std::vector<Item> parts;
  for (auto& g : groups) parts.push_back(contract_greedy(E, net, g.second));
  Labels out;
  for (auto& x : imps) out.push_back(P(x.first, x.second).s_ket);
  for (auto& x : imps) out.push_back(P(x.first, x.second).s_bra);
  out = net.res(out);
  return contract_greedy(E, net, parts, &out).t;
}

// two-site RDM of a bond term (Eq. ExpH): rows (ket s1, ket s2), columns (bra s1, bra s2)
Tensor bond_rdm(ctm_handle* h, const ctm_handle::TermH& t) {
  BlockSpec bs = block_of(t.kind);
  return block_rdm(h, 2 * t.y, 2 * t.x, bs.h, bs.w, {{bs.a1, bs.b1}, {bs.a2, bs.b2}});
}

// one-site RDM of PEPS site (x, y): the 2 x 2 nested block [A Y; X A*] with its Y opened
Tensor site_rdm(ctm_handle* h, int x, int y) { return block_rdm(h, 2 * y, 2 * x, 2, 2, {{0, 1}}); }

// energy of the current environment; optionally seeds dE = 1 into the RDM gradients.
void energy_op(ctm_handle* h, double* e_site, double* e_bonds, bool backward_seed) {
  Engine& E = *h->eng;
  const int nt = (int)h->terms.size();
  const int d2 = h->d.d * h->d.d;
  std::vector<Tensor> rho(nt);
  double* rho64 = (double*)E.arena().alloc(sizeof(double) * nt * d2 * d2);
  for (int t = 0; t < nt; ++t) {
    rho[t] = bond_rdm(h, h->terms[t]);
    cast(rho[t].p, rho[t].dt, rho64 + (int64_t)t * d2 * d2, F64, (int64_t)d2 * d2, false, h->st);
  }
  double* drho = backward_seed ? (double*)E.arena().alloc(sizeof(double) * nt * d2 * d2) : nullptr;
  energy_terms(rho64, h->hs, h->coup, nt, d2, 1.0 / (h->d.Lx * h->d.Ly), e_bonds, e_site, drho, h->dstatus, h->st);
  if (backward_seed)
    for (int t = 0; t < nt; ++t)
      if (rho[t].id >= 0) E.seed_grad(rho[t], drho + (int64_t)t * d2 * d2, F64);
}

// ------------------------------------------------------------------ device state
void ensure_device(ctm_handle* h) {
  if (h->dev_ready) return;
  for (int k = 0; k < ctm_handle::kRowStreams; ++k) {
    CTM_CUDA(cudaStreamCreateWithFlags(&h->row_st[k], cudaStreamNonBlocking));
    CTM_CUDA(cudaEventCreateWithFlags(&h->row_ev[k], cudaEventDisableTiming));
  }
  CTM_CUDA(cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming));
  h->persist.reset(new Arena(size_t(64) << 20));
  h->tape.reset(new Arena(size_t(256) << 20));
  h->store.reset(new Arena(size_t(256) << 20));
  h->eng.reset(new Engine(h->st, h->tape.get()));
  const int64_t chi = h->d.chi, D = h->d.D, d = h->d.d;
  h->slots.resize(h->nsites);
  h->env.resize(h->nsites);
  h->denv.resize(h->nsites);
  for (int s = 0; s < h->nsites; ++s) {
    int i = s / h->C, j = s % h->C;
    auto ld = leg_dims(kind_of(i, j), D, d);
    for (int k = 0; k < 8; ++k) {
      std::vector<int64_t> dims;
      if (k % 2 == 0) {
        dims = {chi, chi};
      } else {
        int leg = ((k - 1) / 2 + 1) % 4;
        dims = {chi};
        for (auto x : ld[leg]) dims.push_back(x);
        dims.push_back(chi);
      }
      Tensor t;
      t.dt = h->edt;
      t.dims = dims;
      t.p = h->persist->alloc(t.bytes());
      h->slots[s][k] = t;
      h->env[s][k] = t;
      Tensor g = t;
      g.p = h->persist->alloc(t.bytes());
      h->denv[s][k] = g;
    }
  }
  int64_t n = (int64_t)h->d.Lx * h->d.Ly * d * D * D * D * D;
  h->A64.dt = F64;
  h->A64.dims = {n};
  h->A64.p = h->persist->alloc(n * 8);
  h->Amode = h->A64;
  if (h->edt != F64) {
    h->Amode.dt = h->edt;
    h->Amode.p = h->persist->alloc(n * dtype_size(h->edt));
  }
  int64_t en = ctm_env_numel(h);
  h->env0 = (double*)h->persist->alloc(en * 8);
  h->dstatus = (int*)h->persist->alloc(64);
  h->dsweeps = (int*)h->persist->alloc(64);
  h->dscal = (double*)h->persist->alloc(64);
  const int nt = (int)h->terms.size(), d2 = (int)(d * d);
  h->hs = (double*)h->persist->alloc(sizeof(double) * nt * d2 * d2);
  h->coup = (double*)h->persist->alloc(sizeof(double) * nt);
  std::vector<double> hh, cc;
  for (auto& t : h->terms) {
    hh.insert(hh.end(), t.h.begin(), t.h.end());
    cc.push_back(t.coup);
  }
  CTM_CUDA(cudaMemcpy(h->hs, hh.data(), sizeof(double) * hh.size(), cudaMemcpyHostToDevice));
  CTM_CUDA(cudaMemcpy(h->coup, cc.data(), sizeof(double) * cc.size(), cudaMemcpyHostToDevice));
  CTM_CUDA(cudaMemset(h->dstatus, 0, 64));
  h->dev_ready = true;
}

// copy a FP64 ring-layout environment into the slots (dtype of the mode)
void load_env(ctm_handle* h, const double* src) {
  int64_t off = 0;
  for (int s = 0; s < h->nsites; ++s)
    for (int k = 0; k < 8; ++k) {
      Tensor& t = h->slots[s][k];
      cast(src + off, F64, t.p, t.dt, t.numel(), false, h->st);
      h->env[s][k] = t;
      off += t.numel();
    }
}

void save_env(ctm_handle* h, double* dst) {
  int64_t off = 0;
  for (int s = 0; s < h->nsites; ++s)
    for (int k = 0; k < 8; ++k) {
      Tensor& t = h->env[s][k];
      cast(t.p, t.dt, dst + off, F64, t.numel(), false, h->st);
      off += t.numel();
    }
}

void checkpoint(ctm_handle* h, int it) {
  if ((int)h->ckpt.size() <= it) h->ckpt.resize(it + 1);
  auto& c = h->ckpt[it];
  if (c.empty()) {
    c.resize(h->nsites);
    for (int s = 0; s < h->nsites; ++s)
      for (int k = 0; k < 8; ++k) {
        c[s][k] = h->slots[s][k];
        c[s][k].p = h->store->alloc(h->slots[s][k].bytes());
      }
  }
  for (int s = 0; s < h->nsites; ++s)
    for (int k = 0; k < 8; ++k)
      CTM_CUDA(cudaMemcpyAsync(c[s][k].p, h->env[s][k].p, c[s][k].bytes(), cudaMemcpyDeviceToDevice, h->st));
}

void forward_iters(ctm_handle* h, int n_iter, double* delta_host) {
  Engine& E = *h->eng;
  E.stop_tape();
  h->replay = false;
  SiteLeaves sl = site_views(h, false);
  SiteLeaves* saved = g_sites;
  g_sites = &sl;
  for (int k = 0; k < n_iter; ++k) {
    int it = h->iters_done;
    checkpoint(h, it);
    if ((int)h->fac.size() <= it) h->fac.resize(it + 1);
    h->cur_iter = it;
    one_iteration(h);
    h->iters_done++;
  }
  g_sites = saved;
  if (delta_host) {
    *delta_host = -1.0;
    int it = h->iters_done - 1;
    if (it >= 1) {
      CTM_CUDA(cudaMemsetAsync(h->dscal, 0, sizeof(double), h->st));
      auto& a = h->fac[it];
      auto& b = h->fac[it - 1];
      for (size_t p = 0; p < a.size() && p < b.size(); ++p)
        spectrum_delta(a[p].lam, b[p].lam, 1, std::min(a[p].rs, b[p].rs), std::min(h->d.chi, std::min(a[p].rs, b[p].rs)),
                       h->dscal, h->st);
      CTM_CUDA(cudaMemcpyAsync(delta_host, h->dscal, sizeof(double), cudaMemcpyDeviceToHost, h->st));
    }
  }
  sync_status(h);
}

}  // namespace
}  // namespace ctm

// ==================================================================== C ABI
namespace {
int guard(ctm_handle* h, const std::function<void()>& fn) {
  try {
    if (h) {
      ctm::g_launch_counter = &h->launches;
      ctm::g_prof = &h->prof;
      ctm::g_limits = &h->limits;
    }
    fn();
    ctm::g_launch_counter = nullptr;
    ctm::g_prof = nullptr;
    ctm::g_limits = nullptr;
    return CTM_OK;
  } catch (const ctm::Error& e) {
    ctm::g_launch_counter = nullptr;
    ctm::g_prof = nullptr;
    ctm::g_limits = nullptr;
    if (h) h->last_error = e.what();
    fprintf(stderr, "libctm: %s\n", e.what());
    return e.status;
  } catch (const std::exception& e) {
    ctm::g_launch_counter = nullptr;
    ctm::g_prof = nullptr;
    ctm::g_limits = nullptr;
    if (h) h->last_error = e.what();
    fprintf(stderr, "libctm: %s\n", e.what());
    return CTM_ERR_INVALID_ARG;
  }
}
}  // namespace

extern "C" {

int ctm_create(const ctm_desc* desc, ctm_handle** out) {
  if (!desc || !out) return CTM_ERR_INVALID_ARG;
  const ctm_desc& d = *desc;
  if (d.Lx < 1 || d.Ly < 1 || d.d < 1 || d.D < 1 || d.chi < 1 || d.n_terms < 1 || d.n_terms > 64 || !d.terms)
    return CTM_ERR_INVALID_ARG;
  if (d.precision < CTM_FP64 || d.precision > CTM_BF16X3) return CTM_ERR_INVALID_ARG;
  // the Jacobi kernels keep a column of the projector's bond matrix (chi * D * d rows) in registers
  if ((int64_t)d.chi * d.D * d.d > 2048) return CTM_ERR_INVALID_ARG;
  for (int t = 0; t < d.n_terms; ++t) {
    const ctm_term& tt = d.terms[t];
    if (!tt.h || tt.x < 0 || tt.x >= d.Lx || tt.y < 0 || tt.y >= d.Ly || tt.kind < 0 || tt.kind > 3)
      return CTM_ERR_INVALID_ARG;
  }
  auto* h = new ctm_handle();
  h->d = d;
  h->d.terms = nullptr;
  h->R = 2 * d.Ly;
  h->C = 2 * d.Lx;
  h->nsites = h->R * h->C;
  h->edt = d.precision == CTM_FP64 ? ctm::F64 : ctm::F32;
  h->cut = d.svd_cutoff_rel > 0 ? d.svd_cutoff_rel : 1e-6;
  h->eps = d.svd_adjoint_eps >= 0 ? d.svd_adjoint_eps : 1e-24;
  int d2 = d.d * d.d;
  for (int t = 0; t < d.n_terms; ++t) {
    const ctm_term& tt = d.terms[t];
    h->terms.push_back({tt.x, tt.y, tt.kind, tt.coupling, std::vector<double>(tt.h, tt.h + d2 * d2)});
  }
  *out = h;
  return CTM_OK;
}

int ctm_init(ctm_handle* h, const double* A, const double* env0, void* stream) {
  if (!h || !A) return CTM_ERR_INVALID_ARG;
  return guard(h, [&]() {
    h->st = (cudaStream_t)stream;
    ctm::ensure_device(h);
    h->eng->set_stream(h->st);
    const int tcm = h->d.precision == CTM_TF32     ? 1
                    : h->d.precision == CTM_BF16   ? 2
                    : h->d.precision == CTM_TF32X3 ? 3
                    : h->d.precision == CTM_BF16X3 ? 4
                                                   : 0;
    // CTM_TC_MIN_MNK (read at every ctm_init) moves the size threshold of the tensor-core route
    const char* tmin = getenv("CTM_TC_MIN_MNK");
    h->eng->set_tc(tcm, h->dstatus, tmin && *tmin ? (int64_t)atoll(tmin) : (int64_t(1) << 26));
    // CTM_STRIDED_GEMM=1 (read at every ctm_init): CUDA-core contractions address their operands
    // through group maps instead of permuted copies
    const char* sg = getenv("CTM_STRIDED_GEMM");
    h->eng->set_strided(sg && sg[0] == '1');
    int64_t n = h->A64.numel();
    CTM_CUDA(cudaMemcpyAsync(h->A64.p, A, n * 8, cudaMemcpyDeviceToDevice, h->st));
    if (h->edt != ctm::F64) ctm::cast(h->A64.p, ctm::F64, h->Amode.p, h->edt, n, false, h->st);
    if (env0) {
      CTM_CUDA(cudaMemcpyAsync(h->env0, env0, ctm_env_numel(h) * 8, cudaMemcpyDeviceToDevice, h->st));
    } else {
      ctm::save_env(h, h->env0);
    }
    ctm::load_env(h, h->env0);
    h->iters_done = 0;
    h->rank_hint.clear();
    h->fac.clear();
    h->ckpt.clear();
    h->store->release({0, 0});
    CTM_CUDA(cudaMemsetAsync(h->dstatus, 0, sizeof(int), h->st));
    h->inited = true;
    CTM_CUDA(cudaStreamSynchronize(h->st));
  });
}

int ctm_step(ctm_handle* h, int n_iter, double* delta_host, void* stream) {
  if (!h || n_iter < 0) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    h->st = (cudaStream_t)stream;
    h->eng->set_stream(h->st);
    ctm::forward_iters(h, n_iter, delta_host);
  });
}

int ctm_energy(ctm_handle* h, double* e_site_dev, double* e_bonds_dev, void* stream) {
  if (!h || !e_site_dev) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    h->st = (cudaStream_t)stream;
    h->eng->set_stream(h->st);
    h->eng->stop_tape();
    auto mark = h->tape->mark();
    ctm::SiteLeaves sl = ctm::site_views(h, false);
    ctm::g_sites = &sl;
    ctm::energy_op(h, e_site_dev, e_bonds_dev, false);
    ctm::g_sites = nullptr;
    h->tape->release(mark);
    ctm::sync_status(h);
  });
}

int ctm_grad(ctm_handle* h, int n_iter, double* e_site_dev, double* dA_dev, void* stream) {
  if (!h || !e_site_dev || !dA_dev || n_iter < 0) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    using namespace ctm;
    h->st = (cudaStream_t)stream;
    Engine& E = *h->eng;
    E.set_stream(h->st);
    // forward from the initial environment
    load_env(h, h->env0);
    h->iters_done = 0;
    h->rank_hint.clear();
    forward_iters(h, n_iter, nullptr);
    const int64_t nA = h->A64.numel();
    CTM_CUDA(cudaMemsetAsync(dA_dev, 0, nA * 8, h->st));
    // energy with its tape
    auto mark = h->tape->mark();
    E.start_tape();
    SiteLeaves sl = site_views(h, true);
    g_sites = &sl;
    for (int s = 0; s < h->nsites; ++s)
      for (int k = 0; k < 8; ++k) h->env[s][k] = E.leaf(h->env[s][k]);
    energy_op(h, e_site_dev, nullptr, true);
    E.backward();
    auto collect = [&](bool zero_missing) {
      int64_t per = (int64_t)h->d.d * h->d.D * h->d.D * h->d.D * h->d.D;
      for (int p = 0; p < (int)sl.t.size(); ++p) {
        void* g = E.grad(sl.t[p], false);
        if (g) cast(g, h->edt, dA_dev + per * p, F64, per, true, h->st);
      }
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) {
          void* g = E.grad(h->env[s][k], false);
          Tensor& dst = h->denv[s][k];
          if (g)
            CTM_CUDA(cudaMemcpyAsync(dst.p, g, dst.bytes(), cudaMemcpyDeviceToDevice, h->st));
          else if (zero_missing)
            CTM_CUDA(cudaMemsetAsync(dst.p, 0, dst.bytes(), h->st));
        }
    };
    collect(true);
    h->tape->release(mark);
    // iterations in reverse, each recomputed from its checkpoint with stored projector factors
    for (int it = n_iter - 1; it >= 0; --it) {
      auto m2 = h->tape->mark();
      E.start_tape();
      SiteLeaves sl2 = site_views(h, true);
      g_sites = &sl2;
      std::vector<std::array<Tensor, 8>> leaves(h->nsites);
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) leaves[s][k] = h->env[s][k] = E.leaf(h->ckpt[it][s][k]);
      h->replay = true;
      h->cur_iter = it;
      one_iteration(h);
      h->replay = false;
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) E.seed_grad(h->env[s][k], h->denv[s][k].p, h->edt);
      E.backward();
      int64_t per = (int64_t)h->d.d * h->d.D * h->d.D * h->d.D * h->d.D;
      for (int p = 0; p < (int)sl2.t.size(); ++p) {
        void* g = E.grad(sl2.t[p], false);
        if (g) cast(g, h->edt, dA_dev + per * p, F64, per, true, h->st);
      }
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) {
          void* g = E.grad(leaves[s][k], false);
          Tensor& dst = h->denv[s][k];
          if (g)
            CTM_CUDA(cudaMemcpyAsync(dst.p, g, dst.bytes(), cudaMemcpyDeviceToDevice, h->st));
          else
            CTM_CUDA(cudaMemsetAsync(dst.p, 0, dst.bytes(), h->st));
        }
      h->tape->release(m2);
    }
    g_sites = nullptr;
    // leave the handle holding the final environment
    for (int s = 0; s < h->nsites; ++s)
      for (int k = 0; k < 8; ++k) h->env[s][k] = h->slots[s][k];
    sync_status(h);
  });
}

int ctm_grad_fixed_point(ctm_handle* h, int max_terms, double tol, double* e_site_dev, double* dA_dev,
                         double* info_host, void* stream) {
  if (!h || !e_site_dev || !dA_dev || max_terms < 1) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  if (!(tol > 0.0)) tol = 1e-10;
  return guard(h, [&]() {
    using namespace ctm;
    h->st = (cudaStream_t)stream;
    Engine& E = *h->eng;
    E.set_stream(h->st);
    const int64_t nA = h->A64.numel();
    const int64_t nenv = ctm_env_numel(h);
    const int64_t per = (int64_t)h->d.d * h->d.D * h->d.D * h->d.D * h->d.D;
    auto base = h->tape->mark();
    // scratch: FP64 environment (for the residual), one series term of dA, norms, reduction work
    double* envd = (double*)h->tape->alloc(sizeof(double) * nenv);
    double* term = (double*)h->tape->alloc(sizeof(double) * nA);
    double* nrm = (double*)h->tape->alloc(sizeof(double) * 8);
    double* work = (double*)h->tape->alloc(sizeof(double) * 1024);
    // one more iteration from env*, numbered after those already run so that its singular vectors
    // take their signs from the previous iteration's: ckpt[it0] = env*, fac[it0] its factors
    const int it0 = h->iters_done;
    forward_iters(h, 1, nullptr);
    // residual ||f(env*) - env*|| / ||env*||
    for (int s = 0; s < h->nsites; ++s)
      for (int k = 0; k < 8; ++k) h->env[s][k] = h->ckpt[it0][s][k];
    save_env(h, envd);
    sumsq(envd, F64, nenv, nrm + 3, work, h->st);
    {
      int64_t off = 0;
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) {
          const Tensor& t = h->slots[s][k];
          PermSpec ps;  // envd -= f(env*), tensor by tensor
          ps.rank = 1;
          ps.out_dims[0] = t.numel();
          ps.in_stride[0] = 1;
          permute(t.p, t.dt, envd + off, F64, ps, true, -1.0, h->st);
          off += t.numel();
        }
    }
    sumsq(envd, F64, nenv, nrm + 2, work, h->st);
    // energy at env*: de/dA into dA, de/denv into denv
    CTM_CUDA(cudaMemsetAsync(dA_dev, 0, nA * 8, h->st));
    {
      auto mark = h->tape->mark();
      E.start_tape();
      SiteLeaves sl = site_views(h, true);
      g_sites = &sl;
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) h->env[s][k] = E.leaf(h->ckpt[it0][s][k]);
      energy_op(h, e_site_dev, nullptr, true);
      E.backward();
      for (int p = 0; p < (int)sl.t.size(); ++p) {
        void* g = E.grad(sl.t[p], false);
        if (g) cast(g, h->edt, dA_dev + per * p, F64, per, true, h->st);
      }
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) {
          void* g = E.grad(h->env[s][k], false);
          Tensor& dst = h->denv[s][k];
          if (g)
            CTM_CUDA(cudaMemcpyAsync(dst.p, g, dst.bytes(), cudaMemcpyDeviceToDevice, h->st));
          else
            CTM_CUDA(cudaMemsetAsync(dst.p, 0, dst.bytes(), h->st));
        }
      h->tape->release(mark);
    }
    // the series: each term replays iteration it0 from env* with its stored factors and pulls the
    // environment cotangent back through it once
    int terms = 0;
    double hn[4] = {0.0, 0.0, 0.0, 0.0};
    double first = -1.0, smallest = -1.0;
    int stalled = 0;
    bool diverged = false;
    for (int n = 1; n <= max_terms; ++n) {
      auto m2 = h->tape->mark();
      E.start_tape();
      SiteLeaves sl2 = site_views(h, true);
      g_sites = &sl2;
      std::vector<std::array<Tensor, 8>> leaves(h->nsites);
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) leaves[s][k] = h->env[s][k] = E.leaf(h->ckpt[it0][s][k]);
      h->replay = true;
      h->cur_iter = it0;
      one_iteration(h);
      h->replay = false;
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) E.seed_grad(h->env[s][k], h->denv[s][k].p, h->edt);
      E.backward();
      CTM_CUDA(cudaMemsetAsync(term, 0, nA * 8, h->st));
      for (int p = 0; p < (int)sl2.t.size(); ++p) {
        void* g = E.grad(sl2.t[p], false);
        if (g) cast(g, h->edt, term + per * p, F64, per, true, h->st);
      }
      cast(term, F64, dA_dev, F64, nA, true, h->st);
      for (int s = 0; s < h->nsites; ++s)
        for (int k = 0; k < 8; ++k) {
          void* g = E.grad(leaves[s][k], false);
          Tensor& dst = h->denv[s][k];
          if (g)
            CTM_CUDA(cudaMemcpyAsync(dst.p, g, dst.bytes(), cudaMemcpyDeviceToDevice, h->st));
          else
            CTM_CUDA(cudaMemsetAsync(dst.p, 0, dst.bytes(), h->st));
        }
      h->tape->release(m2);
      terms = n;
      sumsq(term, F64, nA, nrm + 0, work, h->st);
      sumsq(dA_dev, F64, nA, nrm + 1, work, h->st);
      CTM_CUDA(cudaMemcpyAsync(hn, nrm, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      CTM_CUDA(cudaStreamSynchronize(h->st));
      if (!std::isfinite(hn[0]) || !std::isfinite(hn[1])) {
        diverged = true;
        break;
      }
      if (hn[0] <= tol * tol * hn[1]) break;
      if (first < 0.0) first = hn[0];
      if (hn[0] > 100.0 * first) {  // |term| > 10 x |first term|: the series grows
        diverged = true;
        break;
      }
      // rounding floor: no new smallest term for 10 terms while the terms are already 1e-4 of the
      // sum (the mixed modes converge the environment only to FP32 rounding)
      if (smallest < 0.0 || hn[0] < smallest) {
        smallest = hn[0];
        stalled = 0;
      } else if (++stalled >= 10 && hn[0] <= 1e-8 * hn[1]) {
        break;
      }
    }
    g_sites = nullptr;
    // leave the handle holding env*
    for (int s = 0; s < h->nsites; ++s)
      for (int k = 0; k < 8; ++k) {
        Tensor& t = h->slots[s][k];
        CTM_CUDA(cudaMemcpyAsync(t.p, h->ckpt[it0][s][k].p, t.bytes(), cudaMemcpyDeviceToDevice, h->st));
        h->env[s][k] = t;
      }
    if (info_host) {
      info_host[0] = terms;
      info_host[1] = hn[3] > 0.0 ? std::sqrt(hn[2] / hn[3]) : 0.0;
    }
    h->tape->release(base);
    sync_status(h);
    if (diverged) throw Error(CTM_ERR_DIVERGED, "fixed-point gradient series diverged");
  });
}

int ctm_get_env(ctm_handle* h, double* env_dev, void* stream) {
  if (!h || !env_dev) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    h->st = (cudaStream_t)stream;
    ctm::save_env(h, env_dev);
    CTM_CUDA(cudaStreamSynchronize(h->st));
  });
}

int ctm_set_env(ctm_handle* h, const double* env_dev, void* stream) {
  if (!h || !env_dev) return CTM_ERR_INVALID_ARG;
  return guard(h, [&]() {
    h->st = (cudaStream_t)stream;
    ctm::ensure_device(h);
    ctm::load_env(h, env_dev);
    CTM_CUDA(cudaStreamSynchronize(h->st));
  });
}

int64_t ctm_env_numel(const ctm_handle* h) {
  if (!h) return -1;
  const int64_t chi = h->d.chi, D = h->d.D, d = h->d.d;
  int64_t n = 0;
  for (int s = 0; s < h->nsites; ++s) {
    auto ld = ctm::leg_dims(ctm::kind_of(s / h->C, s % h->C), D, d);
    for (int k = 0; k < 8; ++k) {
      if (k % 2 == 0) {
        n += chi * chi;
      } else {
        int64_t b = 1;
        for (auto x : ld[((k - 1) / 2 + 1) % 4]) b *= x;
        n += chi * b * chi;
      }
    }
  }
  return n;
}

int ctm_magnetization(ctm_handle* h, double* m_dev, double* M_dev, void* stream) {
  if (!h || !m_dev || !M_dev) return CTM_ERR_INVALID_ARG;
  if (h->d.d != 2 || h->d.Lx * h->d.Ly > 64) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    using namespace ctm;
    h->st = (cudaStream_t)stream;
    h->eng->set_stream(h->st);
    h->eng->stop_tape();
    auto mark = h->tape->mark();
    SiteLeaves sl = site_views(h, false);
    g_sites = &sl;
    const int ns = h->d.Lx * h->d.Ly;
    double* rho = (double*)h->eng->arena().alloc(sizeof(double) * 4 * ns);
    for (int y = 0; y < h->d.Ly; ++y)
      for (int x = 0; x < h->d.Lx; ++x) {
        Tensor r = site_rdm(h, x, y);
        cast(r.p, r.dt, rho + 4 * (y * h->d.Lx + x), F64, 4, false, h->st);
      }
    site_magnetization(rho, ns, m_dev, M_dev, h->dstatus, h->st);
    g_sites = nullptr;
    sync_status(h);
    h->tape->release(mark);
  });
}

int ctm_plaquette_order(ctm_handle* h, const int* terms_a, int na, const int* terms_b, int nb, double* Mp_dev,
                        void* stream) {
  if (!h || !Mp_dev || na < 1 || nb < 1 || !terms_a || !terms_b) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k < na; ++k)
    if (terms_a[k] < 0 || terms_a[k] >= (int)h->terms.size()) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k < nb; ++k)
    if (terms_b[k] < 0 || terms_b[k] >= (int)h->terms.size()) return CTM_ERR_INVALID_ARG;
  if (!h->inited) return CTM_ERR_STATE;
  return guard(h, [&]() {
    using namespace ctm;
    h->st = (cudaStream_t)stream;
    h->eng->set_stream(h->st);
    h->eng->stop_tape();
    auto mark = h->tape->mark();
    SiteLeaves sl = site_views(h, false);
    g_sites = &sl;
    const int nt = (int)h->terms.size();
    double* eb = (double*)h->eng->arena().alloc(sizeof(double) * (nt + 1));
    energy_op(h, eb + nt, eb, false);
    std::vector<int> idx(terms_a, terms_a + na);
    idx.insert(idx.end(), terms_b, terms_b + nb);
    int* idx_dev = (int*)h->eng->arena().alloc(sizeof(int) * idx.size());
    CTM_CUDA(cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, h->st));
    plaquette_order(eb, idx_dev, na, nb, Mp_dev, h->st);
    g_sites = nullptr;
    sync_status(h);
    h->tape->release(mark);
  });
}

int64_t ctm_kernel_launches(const ctm_handle* h) { return h ? h->launches : -1; }

int ctm_set_limits(ctm_handle* h, int max_sweeps, int64_t spin_limit) {
  if (!h) return CTM_ERR_INVALID_ARG;
  h->limits.max_sweeps = max_sweeps > 0 ? max_sweeps : ctm::Limits().max_sweeps;
  h->limits.spin_limit = spin_limit > 0 ? spin_limit : ctm::Limits().spin_limit;
  return CTM_OK;
}

int ctm_profile(ctm_handle* h, int enable) {
  if (!h) return CTM_ERR_INVALID_ARG;
  return guard(h, [&]() {
    if (enable) {
      if (h->st || h->dev_ready) CTM_CUDA(cudaStreamSynchronize(h->st));
      h->prof.clear();
      const char* dump = getenv("CTM_PROF_DUMP");
      if (dump && *dump && !h->prof.dump) h->prof.dump = fopen(dump, "w");
      ctm::jacobi_flops_read_reset(h->st);
    }
    h->prof.on = enable != 0;
  });
}

int ctm_profile_read(ctm_handle* h, int cls, double* ms, int64_t* launches, double* flops, double* bytes) {
  if (!h || cls < 0 || cls >= ctm::PROF_NCLASS) return CTM_ERR_INVALID_ARG;
  return guard(h, [&]() {
    CTM_CUDA(cudaStreamSynchronize(h->st));
    auto& P = h->prof;
    P.fold();
    P.fl[ctm::PROF_SVD] += ctm::jacobi_flops_read_reset(h->st);
    if (ms) *ms = P.ms[cls];
    if (launches) *launches = P.n[cls];
    if (flops) *flops = P.fl[cls];
    if (bytes) *bytes = P.by[cls];
  });
}

int ctm_get_spectra(ctm_handle* h, int iter, double* out_host, int max_pairs, int max_vals, int* n_pairs) {
  if (!h || !out_host || !n_pairs || iter < 0 || max_pairs < 1 || max_vals < 1) return CTM_ERR_INVALID_ARG;
  if (!h->inited || iter >= (int)h->fac.size() || iter >= h->iters_done) return CTM_ERR_STATE;
  return guard(h, [&]() {
    CTM_CUDA(cudaStreamSynchronize(h->st));
    const auto& fac = h->fac[iter];
    *n_pairs = (int)fac.size();
    for (int p = 0; p < max_pairs; ++p) {
      double* row = out_host + (int64_t)p * max_vals;
      std::fill(row, row + max_vals, 0.0);
      if (p < (int)fac.size() && fac[p].lam) {
        const int n = std::min(max_vals, fac[p].rs);
        CTM_CUDA(cudaMemcpy(row, fac[p].lam, sizeof(double) * n, cudaMemcpyDeviceToHost));
      }
    }
  });
}

int ctm_mlp_forward(const float* x, int batch, int n_layers, const int* dims, const float* const* W,
                    const float* const* b, float* work, float* y, void* stream) {
  if (!x || !y || !dims || !W || !work || batch < 1 || n_layers < 1 || n_layers > 16) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k <= n_layers; ++k)
    if (dims[k] < 1) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k < n_layers; ++k)
    if (!W[k]) return CTM_ERR_INVALID_ARG;
  return guard(nullptr, [&]() { ctm::mlp_forward(x, batch, n_layers, dims, W, b, work, y, (cudaStream_t)stream); });
}

int64_t ctm_mlp_work_floats(int batch, int n_layers, const int* dims) {
  if (!dims || batch < 1 || n_layers < 1 || n_layers > 16) return -1;
  for (int k = 0; k <= n_layers; ++k)
    if (dims[k] < 1) return -1;
  return ctm::mlp_work_floats(batch, n_layers, dims);
}

int ctm_mlp_backward(const float* x, const float* target, int batch, int n_layers, const int* dims,
                     const float* const* W, const float* const* b, float* const* dW, float* const* db, float* work,
                     float* loss_dev, void* stream) {
  if (!x || !target || !dims || !W || !dW || !work || batch < 1 || n_layers < 1 || n_layers > 16)
    return CTM_ERR_INVALID_ARG;
  for (int k = 0; k <= n_layers; ++k)
    if (dims[k] < 1) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k < n_layers; ++k)
    if (!W[k] || !dW[k] || (b && db && b[k] && !db[k])) return CTM_ERR_INVALID_ARG;
  return guard(nullptr, [&]() {
    ctm::mlp_backward(x, target, batch, n_layers, dims, W, b, dW, b ? db : nullptr, work, loss_dev,
                      (cudaStream_t)stream);
  });
}

int ctm_adam_step(float* p, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                  float eps, int t, void* stream) {
  if (!p || !g || !m || !v || n < 1 || t < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
    return CTM_ERR_INVALID_ARG;
  return guard(nullptr, [&]() { ctm::adam_step(p, g, m, v, n, lr, beta1, beta2, eps, t, (cudaStream_t)stream); });
}

int ctm_svd(const double* M, int batch, int r, double* U, double* s, double* V, void* stream) {
  if (!M || !U || !s || !V || batch < 1 || r < 1 || r > 4096) return CTM_ERR_INVALID_ARG;
  return guard(nullptr, [&]() {
    using namespace ctm;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t rr = (int64_t)r * r;
    double *W = nullptr, *Vw = nullptr;
    int* status = nullptr;
    CTM_CUDA(cudaMalloc(&W, sizeof(double) * rr * batch));
    CTM_CUDA(cudaMalloc(&Vw, sizeof(double) * rr * batch));
    CTM_CUDA(cudaMalloc(&status, 2 * sizeof(int)));
    CTM_CUDA(cudaMemsetAsync(status, 0, 2 * sizeof(int), st));
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
    svd_jacobi(W, Vw, s, U, V, batch, r, lim_sweeps(), status, status + 1, st);
    int hs[2] = {0, 0};
    CTM_CUDA(cudaMemcpyAsync(hs, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CTM_CUDA(cudaStreamSynchronize(st));
    if (getenv("CTM_DEBUG_SWEEPS")) fprintf(stderr, "libctm: ctm_svd batch %d r %d Jacobi sweeps %d\n", batch, r, hs[1]);
    cudaFree(W);
    cudaFree(Vw);
    cudaFree(status);
    if (hs[0] & DEV_TIMEOUT) throw Error(CTM_ERR_TIMEOUT, "device wait timed out");
    if (hs[0] & DEV_SVD_NOCONV) throw Error(CTM_ERR_SVD_NOCONV, "Jacobi SVD did not converge");
    if (hs[0] & DEV_NONFINITE) throw Error(CTM_ERR_NONFINITE, "non-finite singular value");
  });
}

int ctm_destroy(ctm_handle* h) {
  if (!h) return CTM_ERR_INVALID_ARG;
  for (int k = 0; k < ctm_handle::kRowStreams; ++k) {
    if (h->row_st[k]) {
      cudaStreamSynchronize(h->row_st[k]);
      cudaStreamDestroy(h->row_st[k]);
    }
    if (h->row_ev[k]) cudaEventDestroy(h->row_ev[k]);
  }
  if (h->fork_ev) cudaEventDestroy(h->fork_ev);
  h->eng.reset();
  h->persist.reset();
  h->tape.reset();
  h->store.reset();
  delete h;
  return CTM_OK;
}

const char* ctm_error_string(int s) {
  switch (s) {
    case CTM_OK: return "ok";
    case CTM_ERR_INVALID_ARG: return "invalid argument";
    case CTM_ERR_CUDA: return "CUDA runtime error";
    case CTM_ERR_OOM: return "out of device memory";
    case CTM_ERR_NONFINITE: return "non-finite value";
    case CTM_ERR_SVD_NOCONV: return "SVD did not converge";
    case CTM_ERR_DEGENERATE: return "degenerate spectrum";
    case CTM_ERR_TIMEOUT: return "device wait timed out";
    case CTM_ERR_STATE: return "call out of order";
    case CTM_ERR_DIVERGED: return "fixed-point gradient series diverged";
    default: return "unknown status";
  }
}

}  // extern "C"
