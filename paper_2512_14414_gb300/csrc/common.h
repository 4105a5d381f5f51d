// Shared host/device helpers of libctm: dtypes, error status, launch accounting.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>
#include "../../include/ctm.h"

namespace ctm {

enum DType : int { F64 = 0, F32 = 1, BF16 = 2 };

inline size_t dtype_size(DType t) { return t == F64 ? 8 : (t == F32 ? 4 : 2); }

// Error carried inside the library as an exception, converted to a status at the ABI.
struct Error : std::runtime_error {
  int status;
  Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define CTM_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::ctm::Error(e_ == cudaErrorMemoryAllocation ? CTM_ERR_OOM : CTM_ERR_CUDA,    \
                         std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

#define CTM_CHECK(cond, status, msg)                 \
  do {                                               \
    if (!(cond)) throw ::ctm::Error(status, msg);    \
  } while (0)

// Every kernel launch goes through this counter (reported by ctm_kernel_launches).
extern thread_local int64_t* g_launch_counter;
inline void count_launch() {
  if (g_launch_counter) ++*g_launch_counter;
}

#define CTM_LAUNCHED()                    \
  do {                                    \
    ::ctm::count_launch();                \
    CTM_CUDA(cudaGetLastError());         \
  } while (0)

// Limits of the iterative device kernels (ctm_set_limits): the sweep limit of the Jacobi SVD and
// the spin limit of every bounded device-side wait.  The ABI entry points point g_limits at the
// handle's values for the duration of a call; without a handle the defaults apply.
struct Limits {
  int max_sweeps = 60;
  int64_t spin_limit = int64_t(1) << 22;
};
extern thread_local const Limits* g_limits;
inline int lim_sweeps() { return g_limits ? g_limits->max_sweeps : Limits().max_sweeps; }
inline int64_t lim_spins() { return g_limits ? g_limits->spin_limit : Limits().spin_limit; }

// Per-class device timing with CUDA events (enabled by ctm_profile).  A scope records an
// event pair around the launches it encloses, on the launching stream.
enum ProfClass : int { PROF_GEMM = 0, PROF_PERMUTE = 1, PROF_SVD = 2, PROF_QR = 3, PROF_MISC = 4, PROF_TC = 5,
                       PROF_GEMM64 = 6, PROF_NCLASS = 7 };
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs, recycled once folded
  std::vector<int> cls;
  std::vector<double> flops, bytes;
  std::vector<std::string> tags;  // per launch, only when dumping
  size_t used = 0;
  int depth = 0;  // nested scopes count toward the outermost one only
  double ms[PROF_NCLASS] = {0}, fl[PROF_NCLASS] = {0}, by[PROF_NCLASS] = {0};
  int64_t n[PROF_NCLASS] = {0};
  FILE* dump = nullptr;  // per-launch records (CTM_PROF_DUMP=<path>): class, tag, ms
  void begin(int c, cudaStream_t st, double f, double b, const char* tag);
  void end(cudaStream_t st);
  void fold();   // waits for the recorded events and adds them to the class totals
  void clear();  // totals to zero
  ~Profiler();
};
extern thread_local Profiler* g_prof;
inline bool prof_dumping() { return g_prof && g_prof->on && g_prof->dump; }
// Shape tag of a launch for the per-launch dump ("" unless dumping).
inline const char* prof_tag(const char* kind, int64_t b, int64_t m, int64_t n, int64_t k, int x = 0) {
  static thread_local char buf[128];
  if (!prof_dumping()) return nullptr;
  snprintf(buf, sizeof buf, "%s b=%lld M=%lld N=%lld K=%lld x=%d", kind, (long long)b, (long long)m, (long long)n,
           (long long)k, x);
  return buf;
}
struct ProfScope {
  bool active;
  cudaStream_t st;
  ProfScope(int c, cudaStream_t s, double f = 0, double b = 0, const char* tag = nullptr)
      : active(g_prof && g_prof->on), st(s) {
    if (active) g_prof->begin(c, s, f, b, tag);
  }
  ~ProfScope() {
    if (active) g_prof->end(st);
  }
};

// Device status word bits (written by kernels, read by the host at sync points).
enum : int { DEV_SVD_NOCONV = 1, DEV_TIMEOUT = 2, DEV_NONFINITE = 4, DEV_DEGENERATE = 8 };

}  // namespace ctm
