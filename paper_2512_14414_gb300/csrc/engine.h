// Host-side engine of libctm: device arena, tensors, the reverse-mode tape and the
// labelled pairwise contraction (einsum) that lowers to permute + batched GEMM.
#pragma once
#include <functional>
#include <map>
#include <vector>

#include "kernels.h"

namespace ctm {

// Chunked bump allocator over cudaMalloc'd slabs; mark/release recycles memory
// without ever returning it to the driver until destruction.
class Arena {
 public:
  explicit Arena(size_t chunk_bytes = size_t(256) << 20) : chunk_(chunk_bytes) {}
  ~Arena();
  void* alloc(size_t bytes);
  struct Mark {
    size_t chunk, used;
  };
  Mark mark() const { return {cur_, chunks_.empty() ? 0 : chunks_[cur_].used}; }
  void release(const Mark& m);
  size_t peak_bytes() const { return peak_; }
  size_t reserved_bytes() const;

 private:
  struct Chunk {
    char* p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks_;
  size_t cur_ = 0, chunk_, live_ = 0, peak_ = 0;
  void account();
};

struct Tensor {
  void* p = nullptr;
  DType dt = F64;
  std::vector<int64_t> dims;
  int id = -1;  // tape value id when it carries a gradient
  int64_t numel() const {
    int64_t n = 1;
    for (auto d : dims) n *= d;
    return n;
  }
  size_t bytes() const { return (size_t)numel() * dtype_size(dt); }
};

using Labels = std::vector<int>;

class Engine {
 public:
  Engine(cudaStream_t st, Arena* arena) : st_(st), arena_(arena) {}
  cudaStream_t stream() const { return st_; }
  void set_stream(cudaStream_t s) { st_ = s; }
  // While on, contractions keep their temporaries (the caller releases them later): set when
  // work is spread over several streams that share the arena.
  void set_defer_release(bool on) { defer_release_ = on; }
  // CUDA-core contractions read and write their operands in place through group maps instead of
  // permuting them first (the same products in the same order).  Off by default: on GB300 at
  // D=6, chi=64 it removes 13-17 % of the launches but its index-computed, partly uncoalesced
  // loads make an evaluation 2-6 % slower.
  void set_strided(bool on) { strided_ = on; }
  Arena& arena() { return *arena_; }

  Tensor empty(DType dt, const std::vector<int64_t>& dims);
  Tensor zeros(DType dt, const std::vector<int64_t>& dims);

  // ---- tape
  bool recording() const { return record_; }
  void start_tape();   // clears the tape and gradients
  void stop_tape() { record_ = false; }
  Tensor leaf(const Tensor& t);  // value that receives a gradient
  void* grad(const Tensor& t, bool create = true);  // gradient buffer (zero-initialised), same dtype
  void seed_grad(const Tensor& t, const void* g, DType gdt);  // grad(t) += g
  void backward();  // run the tape in reverse
  int new_id(const Tensor& like);
  void push(std::function<void()> fn) {
    if (record_) tape_.push_back(std::move(fn));
  }
  bool needs_grad(std::initializer_list<const Tensor*> ts) const {
    if (!record_) return false;
    for (auto* t : ts)
      if (t->id >= 0) return true;
    return false;
  }

  // ---- operations
  // C[lc] = sum over labels shared by A and B (and absent from lc) of A[la] * B[lb].
  Tensor einsum(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc);
  // out[lc] (+)= einsum(...) into an existing buffer (used by the backward pass).
  void einsum_into(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc, void* out,
                   bool accumulate);
  // y = x / ||x||_F, the norm held constant under differentiation.
  Tensor normalize(const Tensor& x);
  Tensor cast(const Tensor& x, DType to);
  Tensor permute(const Tensor& x, const std::vector<int>& perm);  // out dim k = in dim perm[k]

  // Tensor-core mode of FP32 contractions: 0 SIMT FP32, 1 TF32 (tcgen05 kind::tf32),
  // 2 BF16 operands (tcgen05 kind::f16), 3 error-compensated TF32 (three products),
  // 4 error-compensated BF16.  `status` receives device-side error bits.
  // Products of fewer than min_mnk multiply-adds (batch * M * N * K) stay on the CUDA cores.
  void set_tc(int mode, int* status, int64_t min_mnk) {
    tc_mode_ = mode;
    tc_status_ = status;
    tc_min_mnk_ = min_mnk;
  }
  int64_t gemm_flops() const { return gemm_flops_; }
  int64_t perm_bytes() const { return perm_bytes_; }
  void reset_counters() { gemm_flops_ = perm_bytes_ = 0; }

 private:
  void gemm(DType dt, const void* A, const void* B, void* C, const GemmSpec& g);
  void einsum_tc(const Tensor& A, const Labels& la, const Tensor& B, const Labels& lb, const Labels& lc, void* out,
                 bool accumulate, const std::map<int, int64_t>& dims, const Labels& bla, const Labels& Mla,
                 const Labels& Nlb, const Labels& Kla, const Labels& Mlc, const Labels& Nlc, const Labels& Klb,
                 int64_t nC);
  cudaStream_t st_;
  Arena* arena_;
  bool record_ = false;
  int tc_mode_ = 0;
  int* tc_status_ = nullptr;
  int64_t tc_min_mnk_ = int64_t(1) << 26;
  bool defer_release_ = false;
  bool strided_ = false;
  int next_id_ = 0;
  std::vector<std::function<void()>> tape_;
  std::vector<void*> grads_;
  std::vector<Tensor> gshape_;
  int64_t gemm_flops_ = 0, perm_bytes_ = 0;
};

}  // namespace ctm
