// Tensor-core GEMM for sm_103a: tcgen05.mma (single CTA) with the accumulator in TMEM,
// operands staged into shared memory by TMA (128-byte swizzle) through a 4-stage
// mbarrier pipeline.
//
//   C[b][m][n] (+)= sum_k A[b][m][k] * B[b][n][k]      (both operands K-major, C row-major FP32)
//
// Operands are BF16 (tcgen05 kind::f16, BF16 inputs) or FP32 read as TF32 (kind::tf32);
// accumulation is FP32.  One CTA computes one 128 x 128 output tile:
//   warp 0 / lane 0 issues the TMA loads, warp 1 / lane 0 issues the MMAs, and all four
//   warps read the accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31).
// Every mbarrier wait is bounded; on timeout the CTA raises DEV_TIMEOUT, waits (bounded)
// for the loads it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <set>

#include "kernels.h"

namespace ctm {
namespace {

constexpr int BM = 128, BN = 128;
constexpr int TILE_BYTES = 128 * 128;          // 128 rows x 128 bytes per operand tile and stage
// plain: 2 tiles (A, B) x 4 stages; split (x3): 4 tiles (A_hi, A_lo, B_hi, B_lo) x 3 stages
__host__ __device__ constexpr int stages_of(bool x3) { return x3 ? 3 : 4; }
__host__ __device__ constexpr int smem_of(bool x3) { return (x3 ? 4 : 2) * stages_of(x3) * TILE_BYTES + 1024 + 256; }
constexpr long kWaitLimit = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on timeout or when the CTA is aborting
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_cta) {
  long n = 0;
  while (!mbar_try(bar, parity)) {
    if (*abort_cta) return false;
    if (++n > kWaitLimit) return false;
    if (n > 256) __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile with 128-byte swizzle:
// start address >> 4 in bits 0-13, leading byte offset (unused for this layout) = 1,
// stride byte offset (8 rows x 128 B = 1024 B) >> 4 in bits 32-45, descriptor version 1
// in bits 46-47, layout type 2 (128-byte swizzle) in bits 61-63.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A/B format in bits 7-9 / 10-12
// (BF16 = 1 for kind::f16, TF32 = 2 for kind::tf32), both K-major, N>>3 in bits 17-22,
// M>>4 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  if (BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// X3: error-compensated TF32 -- A = A_hi + A_lo, B = B_hi + B_lo with every part exactly a TF32
// number, and C = A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo is ~2^-22 relative).
template <bool BF16, bool X3>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const __grid_constant__ CUtensorMap mapA2, const __grid_constant__ CUtensorMap mapB2, float* C,
                   int M, int N, int K, float beta, int* status) {
  constexpr int STAGES = stages_of(X3);
  constexpr int NT = X3 ? 4 : 2;  // operand tiles per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tile area (the swizzle pattern repeats every 1024 bytes)
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* tileA = smem;
  unsigned char* tileB = smem + STAGES * TILE_BYTES;
  unsigned char* tileA2 = smem + 2 * STAGES * TILE_BYTES;  // X3 only
  unsigned char* tileB2 = smem + 3 * STAGES * TILE_BYTES;  // X3 only
  uint64_t* full = (uint64_t*)(smem + NT * STAGES * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  volatile int* abort_cta = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, b = blockIdx.z;
  constexpr int ES = BF16 ? 2 : 4;
  constexpr int BK = 128 / ES;           // K elements per stage (one 128-byte swizzle row)
  constexpr int UK = BF16 ? 16 : 8;      // K per MMA instruction (32 bytes)
  const int nk = (K + BK - 1) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *abort_cta = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // loads issued by the producer (for the drain on abort)
  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, use = kb / STAGES;
      if (!mbar_wait(&empty[s], (use & 1) ^ 1, abort_cta)) {
        atomicOr(status, DEV_TIMEOUT);
        *abort_cta = 1;
        break;
      }
      mbar_expect_tx(&full[s], NT * TILE_BYTES);
      tma_load_3d(tileA + s * TILE_BYTES, &mapA, &full[s], kb * BK, m0, b);
      tma_load_3d(tileB + s * TILE_BYTES, &mapB, &full[s], kb * BK, n0, b);
      if (X3) {
        tma_load_3d(tileA2 + s * TILE_BYTES, &mapA2, &full[s], kb * BK, m0, b);
        tma_load_3d(tileB2 + s * TILE_BYTES, &mapB2, &full[s], kb * BK, n0, b);
      }
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = instr_desc(BF16 ? 1u : 2u);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES, use = kb / STAGES;
      if (!mbar_wait(&full[s], use & 1, abort_cta)) {
        atomicOr(status, DEV_TIMEOUT);
        *abort_cta = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(tileA + s * TILE_BYTES), b0 = smem_u32(tileB + s * TILE_BYTES);
#pragma unroll
      for (int kk = 0; kk < BK / UK; ++kk) {
        const uint64_t da = sw128_desc(a0 + kk * 32), db = sw128_desc(b0 + kk * 32);
        if (X3) {  // small terms first
          const uint32_t a2 = smem_u32(tileA2 + s * TILE_BYTES), b2 = smem_u32(tileB2 + s * TILE_BYTES);
          mma<BF16>(tmem, sw128_desc(a2 + kk * 32), db, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          mma<BF16>(tmem, da, sw128_desc(b2 + kk * 32), idesc, 1u);
          mma<BF16>(tmem, da, db, idesc, 1u);
        } else {
          mma<BF16>(tmem, da, db, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  // ---- epilogue: wait for the accumulator, TMEM -> registers -> global
  bool ok = mbar_wait(done, 0, abort_cta);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = __all_sync(0xffffffffu, ok && !*abort_cta);  // tcgen05.ld below is warp-collective
  if (ok) {
    // Each warp stages its 32 rows x 32 columns through a padded shared buffer (the operand tiles
    // are no longer read once `done` has fired) so that the global stores run along rows.
    float* stage = (float*)smem + warp * (32 * 33);
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
      __syncwarp();
      const int col = n0 + c + lane;
#pragma unroll 4
      for (int r = 0; r < 32; ++r) {
        const int row = m0 + warp * 32 + r;
        if (row < M && col < N) {
          float* cp = C + ((int64_t)b * M + row) * (int64_t)N + col;
          float x = stage[r * 33 + lane];
          if (beta != 0.f) x += beta * *cp;
          *cp = x;
        }
      }
      __syncwarp();
    }
  } else {
    atomicOr(status, DEV_TIMEOUT);
  }
  // ---- drain: on abort, wait (bounded) for every issued load to land before the CTA exits
  if (warp == 0 && lane == 0 && *abort_cta) {
    for (int kb = 0; kb < issued; ++kb) {
      long n = 0;
      while (!mbar_try(&full[kb % STAGES], (kb / STAGES) & 1) && ++n < kWaitLimit) {
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, []() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  CTM_CHECK(g_encode != nullptr, CTM_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  return g_encode;
}

// 3-D map over [batch][rows][K] (K innermost), box = 128-byte row x 128 rows, 128B swizzle.
CUtensorMap make_map(const void* p, bool bf16, int64_t rows, int64_t K, int64_t batch) {
  CUtensorMap m;
  const int es = bf16 ? 2 : 4;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)(K * es), (cuuint64_t)(K * rows * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), 128u, 1u};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encoder()(&m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                         const_cast<void*>(p), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CTM_CHECK(r == CUDA_SUCCESS, CTM_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

}  // namespace

bool tc_gemm_ok(bool bf16, int64_t M, int64_t N, int64_t K, const void* A, const void* B) {
  const int es = bf16 ? 2 : 4;
  if ((K * es) % 16 != 0) return false;                        // TMA: row stride multiple of 16 bytes
  if (((uintptr_t)A % 16) || ((uintptr_t)B % 16)) return false;  // TMA: 16-byte aligned base
  if (M > (int64_t(1) << 30) || N > (int64_t(1) << 30) || K > (int64_t(1) << 30)) return false;
  return true;
}

template <bool BF16, bool X3>
void launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& ma2, const CUtensorMap& mb2, float* C,
               int64_t M, int64_t N, int64_t batch, int64_t K, float beta, int* status, cudaStream_t st) {
  // the shared-memory opt-in is a property of the kernel on each device: set it once per device
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      CTM_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<BF16, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    smem_of(X3)));
      done.insert(dev);
    }
  }
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM), (unsigned)batch);
  tc_gemm_kernel<BF16, X3><<<grid, 128, smem_of(X3), st>>>(ma, mb, ma2, mb2, C, (int)M, (int)N, (int)K, beta, status);
  CTM_LAUNCHED();
}

void gemm_tc(const void* A, const void* B, float* C, int64_t M, int64_t N, int64_t K, int64_t batch, bool bf16,
             double beta, int* status, cudaStream_t st) {
  if (M == 0 || N == 0 || batch == 0) return;
  CTM_CHECK(tc_gemm_ok(bf16, M, N, K, A, B), CTM_ERR_INVALID_ARG, "tc gemm: unsupported shape/alignment");
  CTM_CHECK(batch <= 65535, CTM_ERR_INVALID_ARG, "tc gemm: batch too large");
  ProfScope ps(PROF_TC, st, 2.0 * batch * M * N * K, (double)batch * ((bf16 ? 2 : 4) * (M * K + N * K) + 4.0 * M * N),
               prof_tag(bf16 ? "tc_bf16" : "tc_tf32", batch, M, N, K, beta != 0.0));
  CUtensorMap ma = make_map(A, bf16, M, K, batch), mb = make_map(B, bf16, N, K, batch);
  if (bf16)
    launch_tc<true, false>(ma, mb, ma, mb, C, M, N, batch, K, (float)beta, status, st);
  else
    launch_tc<false, false>(ma, mb, ma, mb, C, M, N, batch, K, (float)beta, status, st);
}

void gemm_tc_x3(const float* Ahi, const float* Alo, const float* Bhi, const float* Blo, float* C, int64_t M,
                int64_t N, int64_t K, int64_t batch, double beta, int* status, cudaStream_t st) {
  if (M == 0 || N == 0 || batch == 0) return;
  CTM_CHECK(tc_gemm_ok(false, M, N, K, Ahi, Bhi) && tc_gemm_ok(false, M, N, K, Alo, Blo), CTM_ERR_INVALID_ARG,
            "tc gemm x3: unsupported shape/alignment");
  CTM_CHECK(batch <= 65535, CTM_ERR_INVALID_ARG, "tc gemm: batch too large");
  // algorithmic flops of the product itself (the three partial products are the compensation)
  ProfScope ps(PROF_TC, st, 2.0 * batch * M * N * K, (double)batch * (8.0 * (M * K + N * K) + 4.0 * M * N),
               prof_tag("tc_x3", batch, M, N, K, beta != 0.0));
  CUtensorMap ma = make_map(Ahi, false, M, K, batch), mb = make_map(Bhi, false, N, K, batch);
  CUtensorMap ma2 = make_map(Alo, false, M, K, batch), mb2 = make_map(Blo, false, N, K, batch);
  launch_tc<false, true>(ma, mb, ma2, mb2, C, M, N, batch, K, (float)beta, status, st);
}

void gemm_tc_x3_bf16(const void* Ahi, const void* Alo, const void* Bhi, const void* Blo, float* C, int64_t M,
                     int64_t N, int64_t K, int64_t batch, double beta, int* status, cudaStream_t st) {
  if (M == 0 || N == 0 || batch == 0) return;
  CTM_CHECK(tc_gemm_ok(true, M, N, K, Ahi, Bhi) && tc_gemm_ok(true, M, N, K, Alo, Blo), CTM_ERR_INVALID_ARG,
            "tc gemm bf16 x3: unsupported shape/alignment");
  CTM_CHECK(batch <= 65535, CTM_ERR_INVALID_ARG, "tc gemm: batch too large");
  ProfScope ps(PROF_TC, st, 2.0 * batch * M * N * K, (double)batch * (4.0 * (M * K + N * K) + 4.0 * M * N),
               prof_tag("tc_bf16x3", batch, M, N, K, beta != 0.0));
  CUtensorMap ma = make_map(Ahi, true, M, K, batch), mb = make_map(Bhi, true, N, K, batch);
  CUtensorMap ma2 = make_map(Alo, true, M, K, batch), mb2 = make_map(Blo, true, N, K, batch);
  launch_tc<true, true>(ma, mb, ma2, mb2, C, M, N, batch, K, (float)beta, status, st);
}

}  // namespace ctm
