// Arena, tape and labelled contraction of libctm.
//
// A pairwise contraction C[lc] = sum A[la] B[lb] is lowered to one batched
// GEMM: labels shared by A, B and C form the batch, labels shared by A and B
// only are summed (K), the rest are the free rows (M, from A) and columns
// (N, from B).  Operands are used in place when their memory order already
// reads as [batch | M | K] or [batch | K | M] (and likewise for B); otherwise
// they are permuted into that form first.  Among the layouts that work, the
// one that moves the fewest elements is taken.  The backward pass of a
// contraction is two more contractions (dA = dC . B, dB = A . dC).
#include "engine.h"

#include <cstdlib>

#include <algorithm>
#include <cstring>
#include <numeric>

namespace ctm {



// ================================================================== Arena
Arena::~Arena() {
  for (auto& c : chunks_) cudaFree(c.p);
}

void* Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  while (true) {
    if (cur_ < chunks_.size()) {
      Chunk& c = chunks_[cur_];
      if (c.used + bytes <= c.cap) {
        void* p = c.p + c.used;
        c.used += bytes;
        live_ += bytes;
        account();
        return p;
      }
      if (cur_ + 1 < chunks_.size()) {
        ++cur_;
        chunks_[cur_].used = 0;
        continue;
      }
    }
    size_t cap = std::max(bytes, chunk_);
    char* p = nullptr;
    CTM_CUDA(cudaMalloc(&p, cap));
    chunks_.push_back({p, cap, 0});
    cur_ = chunks_.size() - 1;
  }
}

void Arena::release(const Mark& m) {
  if (chunks_.empty()) return;
  cur_ = m.chunk;
  chunks_[cur_].used = m.used;
  for (size_t k = cur_ + 1; k < chunks_.size(); ++k) chunks_[k].used = 0;
  live_ = 0;
  for (size_t k = 0; k <= cur_; ++k) live_ += chunks_[k].used;
}

size_t Arena::reserved_bytes() const {
  size_t s = 0;
  for (auto& c : chunks_) s += c.cap;
  return s;
}

void Arena::account() { peak_ = std::max(peak_, live_); }

// ================================================================== Engine basics
Tensor Engine::empty(DType dt, const std::vector<int64_t>& dims) {
  Tensor t;
  t.dt = dt;
  t.dims = dims;
  t.p = arena_->alloc(t.bytes());
  return t;
}

Tensor Engine::zeros(DType dt, const std::vector<int64_t>& dims) {
  Tensor t = empty(dt, dims);
  CTM_CUDA(cudaMemsetAsync(t.p, 0, t.bytes(), st_));
  return t;
}

void Engine::start_tape() {
  record_ = true;
  tape_.clear();
  grads_.clear();
  gshape_.clear();
  next_id_ = 0;
}

int Engine::new_id(const Tensor& like) {
  grads_.push_back(nullptr);
  Tensor s;
  s.dt = like.dt;
  s.dims = like.dims;
  gshape_.push_back(s);
  return next_id_++;
}

Tensor Engine::leaf(const Tensor& t) {
  Tensor r = t;
  r.id = record_ ? new_id(t) : -1;
  return r;
}

void* Engine::grad(const Tensor& t, bool create) {
  if (t.id < 0) return nullptr;
  void*& g = grads_[t.id];
  if (!g && create) {
    g = arena_->alloc(gshape_[t.id].bytes());
    CTM_CUDA(cudaMemsetAsync(g, 0, gshape_[t.id].bytes(), st_));
  }
  return g;
}

void Engine::seed_grad(const Tensor& t, const void* g, DType gdt) {
  void* d = grad(t, true);
  ctm::cast(g, gdt, d, t.dt, t.numel(), true, st_);
}

void Engine::backward() {
  record_ = false;
  for (auto it = tape_.rbegin(); it != tape_.rend(); ++it) (*it)();
  tape_.clear();
}

void Engine::gemm(DType dt, const void* A, const void* B, void* C, const GemmSpec& g) {
  gemm_flops_ += 2 * g.batch * g.M * g.N * g.K;
  if (dt == F64)
    gemm_f64((const double*)A, (const double*)B, (double*)C, g, st_);
  else if (dt == F32)
    gemm_f32((const float*)A, (const float*)B, (float*)C, g, st_);
  else
    throw Error(CTM_ERR_INVALID_ARG, "gemm dtype");
}

// ================================================================== contraction planning
namespace {

Labels subseq(const Labels& l, const Labels& keep) {
  Labels r;
  for (int x : l)
    if (std::find(keep.begin(), keep.end(), x) != keep.end()) r.push_back(x);
  return r;
}

bool has(const Labels& l, int x) { return std::find(l.begin(), l.end(), x) != l.end(); }

Labels cat(std::initializer_list<const Labels*> ls) {
  Labels r;
  for (auto* l : ls) r.insert(r.end(), l->begin(), l->end());
  return r;
}

int64_t prod(const Labels& l, const std::map<int, int64_t>& d) {
  int64_t p = 1;
  for (int x : l) p *= d.at(x);
  return p;
}

// permute `src` (labels ls, dims from map) into the label order `target`
PermSpec perm_spec(const Labels& ls, const Labels& target, const std::map<int, int64_t>& dims) {
  std::vector<int64_t> str(ls.size());
  int64_t s = 1;
  for (int k = (int)ls.size() - 1; k >= 0; --k) {
    str[k] = s;
    s *= dims.at(ls[k]);
  }
  PermSpec p;
  CTM_CHECK(target.size() <= 8, CTM_ERR_INVALID_ARG, "rank > 8");
  p.rank = (int)target.size();
  for (size_t k = 0; k < target.size(); ++k) {
    auto it = std::find(ls.begin(), ls.end(), target[k]);
    p.out_dims[k] = dims.at(target[k]);
    p.in_stride[k] = str[it - ls.begin()];
  }
  return p;
}

}  // namespace

void Engine::einsum_into(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc,
                         void* out, bool accumulate) {
  CTM_CHECK(A.dt == B.dt, CTM_ERR_INVALID_ARG, "einsum dtype mismatch");
  CTM_CHECK(la.size() == A.dims.size() && lb.size() == B.dims.size(), CTM_ERR_INVALID_ARG, "einsum label count");
  std::map<int, int64_t> dims;
  for (size_t k = 0; k < la.size(); ++k) dims[la[k]] = A.dims[k];
  for (size_t k = 0; k < lb.size(); ++k) {
    auto it = dims.find(lb[k]);
    CTM_CHECK(it == dims.end() || it->second == B.dims[k], CTM_ERR_INVALID_ARG, "einsum dim mismatch");
    dims[lb[k]] = B.dims[k];
  }
  Labels batch, K, M, N;
  for (int x : la) {
    bool inb = has(lb, x), inc = has(lc, x);
    CTM_CHECK(inb || inc, CTM_ERR_INVALID_ARG, "label only in A");
    if (inb && inc) batch.push_back(x);
    else if (inb) K.push_back(x);
    else M.push_back(x);
  }
  for (int x : lb) {
    bool ina = has(la, x), inc = has(lc, x);
    CTM_CHECK(ina || inc, CTM_ERR_INVALID_ARG, "label only in B");
    if (!ina) N.push_back(x);
  }
  for (int x : lc) CTM_CHECK(dims.count(x), CTM_ERR_INVALID_ARG, "output label unknown");
  const int64_t nA = A.numel(), nB = B.numel();
  int64_t nC = 1;
  for (int x : lc) nC *= dims[x];

  const Labels Mla = M, Mlc = subseq(lc, M), Nlb = N, Nlc = subseq(lc, N), Kla = K, Klb = subseq(lb, K);
  const Labels bla = batch;
  // tensor-core route for FP32 contractions: both operands K-major ([batch|M|K] and [batch|N|K])
  const int64_t KK0 = prod(K, dims), MM0 = prod(M, dims), NN0 = prod(N, dims), nb0 = prod(batch, dims);
  // Small products stay on the CUDA cores: below tc_min_mnk_ multiply-adds (or with an output
  // side shorter than 32) a tcgen05 tile's fixed cost (TMEM allocation, barrier set-up, pipeline
  // fill) exceeds the whole FP32 product, and with fewer than 8 output tiles a long K runs on a
  // handful of SMs where the CUDA-core path splits it.
  const int64_t tiles0 = nb0 * ((MM0 + 127) / 128) * ((NN0 + 127) / 128);
  const bool tc = A.dt == F32 && tc_mode_ != 0 && KK0 >= 8 && nb0 <= 65535 &&
                  nb0 * MM0 * NN0 * KK0 >= tc_min_mnk_ && MM0 >= 32 && NN0 >= 32 &&
                  (tiles0 >= 8 || tc_min_mnk_ == 0) &&
                  (KK0 * (tc_mode_ == 2 || tc_mode_ == 4 ? 2 : 4)) % 16 == 0;  // 1 tf32, 2 bf16, 3 tf32x3, 4 bf16x3
  if (tc) {
    einsum_tc(A, la, B, lb, lc, out, accumulate, dims, batch, M, N, K, Mlc, Nlc, Klb, nC);
    return;
  }
  struct Cand {
    Labels Mo, No, Ko;
    bool swap;
    int64_t cost;
    int aLay, bLay;  // 0 = normal in place, 1 = transposed in place, 2 = permute to normal
    bool permC;
  };
  Cand best;
  best.cost = -1;
  for (const Labels* Mo : {&Mla, &Mlc})
    for (const Labels* No : {&Nlb, &Nlc})
      for (const Labels* Ko : {&Kla, &Klb})
        for (bool swap : {false, true}) {
          Cand c{*Mo, *No, *Ko, swap, 0, 2, 2, false};
          if (la == cat({&bla, Mo, Ko})) c.aLay = 0;
          else if (la == cat({&bla, Ko, Mo})) c.aLay = 1;
          else c.cost += nA;
          if (lb == cat({&bla, Ko, No})) c.bLay = 0;
          else if (lb == cat({&bla, No, Ko})) c.bLay = 1;
          else c.cost += nB;
          Labels nat = swap ? cat({&bla, No, Mo}) : cat({&bla, Mo, No});
          c.permC = (nat != lc);
          if (c.permC) c.cost += 2 * nC;
          c.cost = c.cost * 4 + (swap ? 1 : 0);
          if (best.cost < 0 || c.cost < best.cost) best = c;
        }
  const int64_t nb = prod(batch, dims), MM = prod(best.Mo, dims), NN = prod(best.No, dims), KK = prod(best.Ko, dims);
  const size_t es = dtype_size(A.dt);
  if (strided_ && KK > 0 && (A.dt == F32 || A.dt == F64) && (best.aLay == 2 || best.bLay == 2 || best.permC)) {
    // The planner's choice (M, N, K orders and swap) is kept; only the permuted copies go: the
    // GEMM reads A, B and writes C where they are.
    auto sz = [&](int l) { return dims.at(l); };
    StridedGemm sm;
    bool ok = true;
    const Tensor& GA = best.swap ? B : A;  // the GEMM's first operand
    const Tensor& GB = best.swap ? A : B;
    const Labels& lGA = best.swap ? lb : la;
    const Labels& lGB = best.swap ? la : lb;
    const Labels& gM = best.swap ? best.No : best.Mo;
    const Labels& gN = best.swap ? best.Mo : best.No;
    ok = ok && build_group_map(lGA, bla, sz, sm.aB) && build_group_map(lGA, gM, sz, sm.aM) &&
         build_group_map(lGA, best.Ko, sz, sm.aK);
    ok = ok && build_group_map(lGB, bla, sz, sm.bB) && build_group_map(lGB, best.Ko, sz, sm.bK) &&
         build_group_map(lGB, gN, sz, sm.bN);
    ok = ok && build_group_map(lc, bla, sz, sm.cB) && build_group_map(lc, gM, sz, sm.cM) &&
         build_group_map(lc, gN, sz, sm.cN);
    if (ok) {
      GemmSpec g;
      g.batch = nb;
      g.M = best.swap ? NN : MM;
      g.N = best.swap ? MM : NN;
      g.K = KK;
      g.alpha = 1.0;
      g.beta = accumulate ? 1.0 : 0.0;
      // neighbouring threads along the index whose innermost stride is 1 (coalesced loads)
      auto inner = [](const GroupMap& m) { return m.n ? m.stride[m.n - 1] : 0; };
      g.transA = inner(sm.aM) == 1 && inner(sm.aK) != 1;
      g.transB = inner(sm.bK) == 1 && inner(sm.bN) != 1;
      gemm_flops_ += 2 * nb * MM * NN * KK;
      if (A.dt == F64)
        gemm_strided_f64((const double*)GA.p, (const double*)GB.p, (double*)out, g, sm, st_);
      else
        gemm_strided_f32((const float*)GA.p, (const float*)GB.p, (float*)out, g, sm, st_);
      return;
    }
  }
  auto mark = arena_->mark();
  const void* Ap = A.p;
  const void* Bp = B.p;
  if (best.aLay == 2) {
    Labels tgt = cat({&bla, &best.Mo, &best.Ko});
    void* t = arena_->alloc(nA * es);
    ctm::permute(A.p, A.dt, t, A.dt, perm_spec(la, tgt, dims), false, 1.0, st_);
    perm_bytes_ += 2 * nA * es;
    Ap = t;
  }
  if (best.bLay == 2) {
    Labels tgt = cat({&bla, &best.Ko, &best.No});
    void* t = arena_->alloc(nB * es);
    ctm::permute(B.p, B.dt, t, B.dt, perm_spec(lb, tgt, dims), false, 1.0, st_);
    perm_bytes_ += 2 * nB * es;
    Bp = t;
  }
  const bool aT = best.aLay == 1, bT = best.bLay == 1;  // [K|M] resp. [N|K] in memory
  void* Cp = out;
  if (best.permC) Cp = arena_->alloc(nC * es);
  GemmSpec g;
  g.batch = nb;
  g.K = KK;
  g.alpha = 1.0;
  g.beta = (!best.permC && accumulate) ? 1.0 : 0.0;
  if (!best.swap) {
    g.M = MM;
    g.N = NN;
    g.transA = aT;
    g.lda = aT ? MM : KK;
    g.transB = bT;
    g.ldb = bT ? KK : NN;
    g.ldc = NN;
    g.strideA = MM * KK;
    g.strideB = KK * NN;
    g.strideC = MM * NN;
    gemm(A.dt, Ap, Bp, Cp, g);
  } else {
    // C^T[n][m] = sum_k B(k,n) A(m,k)
    g.M = NN;
    g.N = MM;
    g.transA = !bT;  // B stored [K|N]: (n,k) at k*NN+n
    g.lda = bT ? KK : NN;
    g.transB = !aT;  // A stored [M|K]: (k,m) at m*KK+k
    g.ldb = aT ? MM : KK;
    g.ldc = MM;
    g.strideA = KK * NN;
    g.strideB = MM * KK;
    g.strideC = MM * NN;
    gemm(A.dt, Bp, Ap, Cp, g);
  }
  if (best.permC) {
    Labels nat = best.swap ? cat({&bla, &best.No, &best.Mo}) : cat({&bla, &best.Mo, &best.No});
    ctm::permute(Cp, A.dt, out, A.dt, perm_spec(nat, lc, dims), accumulate, 1.0, st_);
    perm_bytes_ += (accumulate ? 3 : 2) * nC * es;
  }
  // temporaries are dead once the kernels above are enqueued in stream order (not while several
  // streams draw on the arena: then the next contraction may run concurrently on another stream)
  if (!defer_release_) arena_->release(mark);
}

void Engine::einsum_tc(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc,
                       void* out, bool accumulate, const std::map<int, int64_t>& dims, const Labels& bla,
                       const Labels& Mla, const Labels& Nlb, const Labels& Kla, const Labels& Mlc,
                       const Labels& Nlc, const Labels& Klb, int64_t nC) {
  const bool bf16 = tc_mode_ == 2;
  const DType odt = bf16 ? BF16 : F32;
  const int64_t nA = A.numel(), nB = B.numel();
  struct Cand {
    Labels Mo, No, Ko;
    bool swap, aok, bok, permC;
    int64_t cost;
  } best;
  best.cost = -1;
  for (const Labels* Mo : {&Mla, &Mlc})
    for (const Labels* No : {&Nlb, &Nlc})
      for (const Labels* Ko : {&Kla, &Klb})
        for (bool swap : {false, true}) {
          Cand c{*Mo, *No, *Ko, swap, la == cat({&bla, Mo, Ko}), lb == cat({&bla, No, Ko}), false, 0};
          if (c.aok && (uintptr_t)A.p % 16) c.aok = false;
          if (c.bok && (uintptr_t)B.p % 16) c.bok = false;
          Labels nat = swap ? cat({&bla, No, Mo}) : cat({&bla, Mo, No});
          c.permC = nat != lc;
          c.cost = (c.aok ? 0 : nA) + (c.bok ? 0 : nB) + (c.permC ? 2 * nC : 0);
          c.cost = c.cost * 4 + (swap ? 1 : 0);
          if (best.cost < 0 || c.cost < best.cost) best = c;
        }
  const int64_t nb = prod(bla, dims), MM = prod(best.Mo, dims), NN = prod(best.No, dims), KK = prod(best.Ko, dims);
  auto mark = arena_->mark();
  const void* Ap = A.p;
  const void* Bp = B.p;
  if (!best.aok || bf16) {
    void* t = arena_->alloc(nA * dtype_size(odt));
    ctm::permute(A.p, A.dt, t, odt, perm_spec(la, cat({&bla, &best.Mo, &best.Ko}), dims), false, 1.0, st_);
    perm_bytes_ += nA * (4 + dtype_size(odt));
    Ap = t;
  }
  if (!best.bok || bf16) {
    void* t = arena_->alloc(nB * dtype_size(odt));
    ctm::permute(B.p, B.dt, t, odt, perm_spec(lb, cat({&bla, &best.No, &best.Ko}), dims), false, 1.0, st_);
    perm_bytes_ += nB * (4 + dtype_size(odt));
    Bp = t;
  }
  void* Cp = best.permC ? arena_->alloc(nC * 4) : out;
  const double beta = (!best.permC && accumulate) ? 1.0 : 0.0;
  gemm_flops_ += 2 * nb * MM * NN * KK;
  if (tc_mode_ == 4) {
    void* Ah = arena_->alloc(nA * 2);
    void* Al = arena_->alloc(nA * 2);
    void* Bh = arena_->alloc(nB * 2);
    void* Bl = arena_->alloc(nB * 2);
    split_bf16((const float*)Ap, Ah, Al, nA, st_);
    split_bf16((const float*)Bp, Bh, Bl, nB, st_);
    if (!best.swap)
      gemm_tc_x3_bf16(Ah, Al, Bh, Bl, (float*)Cp, MM, NN, KK, nb, beta, tc_status_, st_);
    else
      gemm_tc_x3_bf16(Bh, Bl, Ah, Al, (float*)Cp, NN, MM, KK, nb, beta, tc_status_, st_);
  } else if (tc_mode_ == 3) {
    float* Ah = (float*)arena_->alloc(nA * 4);
    float* Al = (float*)arena_->alloc(nA * 4);
    float* Bh = (float*)arena_->alloc(nB * 4);
    float* Bl = (float*)arena_->alloc(nB * 4);
    split_tf32((const float*)Ap, Ah, Al, nA, st_);
    split_tf32((const float*)Bp, Bh, Bl, nB, st_);
    if (!best.swap)
      gemm_tc_x3(Ah, Al, Bh, Bl, (float*)Cp, MM, NN, KK, nb, beta, tc_status_, st_);
    else
      gemm_tc_x3(Bh, Bl, Ah, Al, (float*)Cp, NN, MM, KK, nb, beta, tc_status_, st_);
  } else if (!best.swap) {
    gemm_tc(Ap, Bp, (float*)Cp, MM, NN, KK, nb, bf16, beta, tc_status_, st_);
  } else {
    gemm_tc(Bp, Ap, (float*)Cp, NN, MM, KK, nb, bf16, beta, tc_status_, st_);
  }
  if (best.permC) {
    Labels nat = best.swap ? cat({&bla, &best.No, &best.Mo}) : cat({&bla, &best.Mo, &best.No});
    ctm::permute(Cp, F32, out, F32, perm_spec(nat, lc, dims), accumulate, 1.0, st_);
    perm_bytes_ += (accumulate ? 3 : 2) * nC * 4;
  }
  if (!defer_release_) arena_->release(mark);
}

Tensor Engine::einsum(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc) {
  std::map<int, int64_t> dims;
  for (size_t k = 0; k < la.size(); ++k) dims[la[k]] = A.dims[k];
  for (size_t k = 0; k < lb.size(); ++k) dims[lb[k]] = B.dims[k];
  std::vector<int64_t> cd;
  for (int x : lc) cd.push_back(dims.at(x));
  Tensor C = empty(A.dt, cd);
  einsum_into(A, la, B, lb, lc, C.p, false);
  if (needs_grad({&A, &B})) {
    C.id = new_id(C);
    Tensor Ac = A, Bc = B;
    Labels a = la, b = lb, c = lc;
    int cid = C.id;
    Tensor Cshape = C;
    push([this, Ac, Bc, a, b, c, cid, Cshape]() {
      void* gc = grads_[cid];
      if (!gc) return;
      Tensor dC = Cshape;
      dC.p = gc;
      dC.id = -1;
      if (Ac.id >= 0) einsum_into(dC, c, Bc, b, a, grad(Ac), true);
      if (Bc.id >= 0) einsum_into(Ac, a, dC, c, b, grad(Bc), true);
    });
  }
  return C;
}

Tensor Engine::normalize(const Tensor& x) {
  Tensor y = empty(x.dt, x.dims);
  double* sc = (double*)arena_->alloc(2 * sizeof(double));
  double* work = (double*)arena_->alloc(1024 * sizeof(double));
  sumsq(x.p, x.dt, x.numel(), sc, work, st_);
  scale_rsqrt(x.p, x.dt, x.numel(), sc, y.p, sc + 1, st_);
  if (needs_grad({&x})) {
    y.id = new_id(y);
    Tensor xc = x;
    int yid = y.id;
    double* inv = sc + 1;
    push([this, xc, yid, inv]() {
      void* gy = grads_[yid];
      if (!gy) return;
      scale_by(gy, xc.dt, xc.numel(), inv, grad(xc), true, st_);
    });
  }
  return y;
}

Tensor Engine::cast(const Tensor& x, DType to) {
  Tensor y = empty(to, x.dims);
  ctm::cast(x.p, x.dt, y.p, to, x.numel(), false, st_);
  if (needs_grad({&x})) {
    y.id = new_id(y);
    Tensor xc = x;
    int yid = y.id;
    DType yt = to;
    push([this, xc, yid, yt]() {
      void* gy = grads_[yid];
      if (!gy) return;
      ctm::cast(gy, yt, grad(xc), xc.dt, xc.numel(), true, st_);
    });
  }
  return y;
}

Tensor Engine::permute(const Tensor& x, const std::vector<int>& perm) {
  std::vector<int64_t> od;
  for (int k : perm) od.push_back(x.dims[k]);
  Tensor y = empty(x.dt, od);
  Labels ls(x.dims.size());
  std::iota(ls.begin(), ls.end(), 0);
  std::map<int, int64_t> dims;
  for (size_t k = 0; k < ls.size(); ++k) dims[(int)k] = x.dims[k];
  Labels tgt(perm.begin(), perm.end());
  ctm::permute(x.p, x.dt, y.p, x.dt, perm_spec(ls, tgt, dims), false, 1.0, st_);
  perm_bytes_ += 2 * x.bytes();
  if (needs_grad({&x})) {
    y.id = new_id(y);
    Tensor xc = x;
    int yid = y.id;
    push([this, xc, yid, tgt, ls, dims]() {
      void* gy = grads_[yid];
      if (!gy) return;
      ctm::permute(gy, xc.dt, grad(xc), xc.dt, perm_spec(tgt, ls, dims), true, 1.0, st_);
    });
  }
  return y;
}

}  // namespace ctm
