// Shared host/device helpers of libctm: dtypes, error status, launch accounting.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
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

// Device status word bits (written by kernels, read by the host at sync points).
enum : int { DEV_SVD_NOCONV = 1, DEV_TIMEOUT = 2, DEV_NONFINITE = 4, DEV_DEGENERATE = 8 };

}  // namespace ctm
