// Element-wise, permutation, SIMT GEMM, projector-helper and energy kernels of libctm.
#include <type_traits>

#include "kernels.h"

#include <algorithm>
#include <cmath>
#include <map>

namespace ctm {

thread_local int64_t* g_launch_counter = nullptr;
thread_local Profiler* g_prof = nullptr;
thread_local const Limits* g_limits = nullptr;

void Profiler::begin(int c, cudaStream_t st, double f, double b, const char* tag) {
  if (depth++ > 0) return;
  if (used + 2 > ev.size()) {
    if (ev.size() >= (size_t(1) << 16)) fold();
    if (used + 2 > ev.size()) {
      size_t old = ev.size();
      ev.resize(std::max<size_t>(4096, ev.size() * 2));
      for (size_t k = old; k < ev.size(); ++k) cudaEventCreate(&ev[k]);
    }
  }
  cls.push_back(c);
  flops.push_back(f);
  bytes.push_back(b);
  if (dump) tags.push_back(tag ? tag : "");
  cudaEventRecord(ev[used++], st);
}

void Profiler::end(cudaStream_t st) {
  if (--depth > 0) return;
  if (used % 2 == 1) cudaEventRecord(ev[used++], st);
}

void Profiler::fold() {
  if (used == 0) return;
  cudaEventSynchronize(ev[used - 1]);
  for (size_t k = 0; k + 1 < used; k += 2) {
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
    const int c = cls[k / 2];
    ms[c] += t;
    n[c] += 1;
    fl[c] += flops[k / 2];
    by[c] += bytes[k / 2];
    if (dump) fprintf(dump, "%d\t%s\t%.6f\n", c, tags[k / 2].c_str(), t);
  }
  used = 0;
  cls.clear();
  flops.clear();
  bytes.clear();
  tags.clear();
}

void Profiler::clear() {
  used = 0;
  depth = 0;
  cls.clear();
  flops.clear();
  bytes.clear();
  tags.clear();
  for (int c = 0; c < PROF_NCLASS; ++c) ms[c] = fl[c] = by[c] = 0, n[c] = 0;
}

Profiler::~Profiler() {
  for (auto e : ev) cudaEventDestroy(e);
  if (dump) fclose(dump);
}

namespace {

template <typename T>
__device__ __forceinline__ double to_d(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_d<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <typename T>
__device__ __forceinline__ T from_d(double v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }

inline int nblocks(int64_t n, int per_block, int cap = 65535 * 8) {
  int64_t b = (n + per_block - 1) / per_block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

// ------------------------------------------------------------------ permutation
struct PermDev {
  int rank;
  int64_t dims[8];
  int64_t istr[8];
  int64_t ostr[8];
};

template <typename Ti, typename To, bool ACC>
__global__ void permute_generic(const Ti* __restrict__ in, To* __restrict__ out, PermDev p, int64_t n, double scale) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = idx, src = 0;
#pragma unroll 8
    for (int k = 7; k >= 0; --k) {
      if (k < p.rank) {
        int64_t c = rem % p.dims[k];
        rem /= p.dims[k];
        src += c * p.istr[k];
      }
    }
    double v = scale * to_d(in[src]);
    if (ACC) v += to_d(out[idx]);
    out[idx] = from_d<To>(v);
  }
}

// Tiled transpose: output innermost dim `a` (in-stride sa) and the output dim `b` with input stride 1.
struct PermTile {
  int64_t Na, Nb, sa, ob;  // sizes, in-stride of a, out-stride of b
  int nrest;
  int64_t rdims[8], ristr[8], rostr[8];
  int64_t nrest_total;
};

template <typename Ti, typename To, bool ACC>
__global__ void permute_tiled(const Ti* __restrict__ in, To* __restrict__ out, PermTile p, double scale) {
  __shared__ double tile[32][33];
  const int64_t tiles_a = (p.Na + 31) / 32;
  const int64_t ta = blockIdx.x % tiles_a, tb = blockIdx.x / tiles_a;
  const int64_t a0 = ta * 32, b0 = tb * 32;
  for (int64_t rest = blockIdx.y; rest < p.nrest_total; rest += gridDim.y) {
    int64_t rem = rest, ioff = 0, ooff = 0;
    for (int k = p.nrest - 1; k >= 0; --k) {
      int64_t c = rem % p.rdims[k];
      rem /= p.rdims[k];
      ioff += c * p.ristr[k];
      ooff += c * p.rostr[k];
    }
    __syncthreads();
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
      int64_t ai = a0 + ty, bi = b0 + threadIdx.x;
      if (ai < p.Na && bi < p.Nb) tile[ty][threadIdx.x] = to_d(in[ioff + ai * p.sa + bi]);
    }
    __syncthreads();
    for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
      int64_t bi = b0 + ty, ai = a0 + threadIdx.x;
      if (ai < p.Na && bi < p.Nb) {
        int64_t o = ooff + bi * p.ob + ai;
        double v = scale * tile[threadIdx.x][ty];
        if (ACC) v += to_d(out[o]);
        out[o] = from_d<To>(v);
      }
    }
  }
}

// Row copy: the innermost output dimension is contiguous in the input as well (in-stride 1), so
// the permutation moves whole rows of `len` elements.  One warp per work item (a row, or a
// 1024-element piece of a long one); the row's source and destination offsets are decoded once
// and the piece is copied with 16-byte loads and stores where both ends are 16-byte aligned
// (`vec` elements per access).
struct PermRows {
  int nouter;         // output dimensions before the row
  int dims[7];        // their sizes
  int64_t istr[7];    // their input strides
  int64_t ostr[7];    // their output strides
  int64_t nrows;
  int len;            // row length (elements)
  int chunk;          // elements per work item (a multiple of the vector width)
  int nchunk;         // work items per row
};

template <typename Ti, typename To, bool ACC, int VEC>
__global__ void permute_rows(const Ti* __restrict__ in, To* __restrict__ out, PermRows p, double scale) {
  const int lane = threadIdx.x % 32;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
  const int64_t items = p.nrows * p.nchunk;
  for (int64_t item = gw; item < items; item += nw) {
    const int64_t row = item / p.nchunk;
    const int c0 = (int)(item % p.nchunk) * p.chunk;
    const int c1 = min(p.len, c0 + p.chunk);
    int64_t rem = row, ioff = 0, ooff = 0;
    for (int k = p.nouter - 1; k >= 0; --k) {
      const int64_t c = rem % p.dims[k];
      rem /= p.dims[k];
      ioff += c * p.istr[k];
      ooff += c * p.ostr[k];
    }
    const Ti* src = in + ioff;
    To* dst = out + ooff;
    if (VEC > 1) {
      // Ti == To here (no conversion), 16-byte vectors
      using V = typename std::conditional<sizeof(Ti) == 8, double2, float4>::type;
      const V* s4 = reinterpret_cast<const V*>(src);
      V* d4 = reinterpret_cast<V*>(dst);
      for (int i = c0 / VEC + lane; i < c1 / VEC; i += 32) {
        V v = __ldg(s4 + i);
        if (scale != 1.0 || ACC) {
          Ti* e = reinterpret_cast<Ti*>(&v);
          const Ti* o = reinterpret_cast<const Ti*>(d4 + i);
#pragma unroll
          for (int k = 0; k < VEC; ++k) e[k] = (Ti)(scale * (double)e[k] + (ACC ? (double)o[k] : 0.0));
        }
        d4[i] = v;
      }
    } else {
      for (int i = c0 + lane; i < c1; i += 32) {
        double v = scale * to_d(src[i]);
        if (ACC) v += to_d(dst[i]);
        dst[i] = from_d<To>(v);
      }
    }
  }
}

template <typename Ti, typename To>
void permute_t(const Ti* in, To* out, const PermSpec& ps, bool acc, double scale, cudaStream_t st) {
  int r = ps.rank;
  int64_t n = 1;
  for (int k = 0; k < r; ++k) n *= ps.out_dims[k];
  if (n == 0) return;
  ProfScope prof(PROF_PERMUTE, st, 0.0, (double)n * (sizeof(Ti) + sizeof(To) * (acc ? 2 : 1)),
                 prof_tag("permute", ps.rank, n, sizeof(Ti), sizeof(To), acc));
  int64_t ostr[8];
  int64_t s = 1;
  for (int k = r - 1; k >= 0; --k) {
    ostr[k] = s;
    s *= ps.out_dims[k];
  }
  int b = -1;
  for (int k = 0; k < r - 1; ++k)
    if (ps.in_stride[k] == 1 && ps.out_dims[k] > 1) b = k;
  // whole rows: the last output dimension is also contiguous in the input; merge with the
  // dimensions before it while they stay contiguous in both
  if (ps.in_stride[r - 1] == 1 && ps.out_dims[r - 1] >= 16) {
    int64_t len = ps.out_dims[r - 1];
    int k = r - 2;
    while (k >= 0 && ps.in_stride[k] == len && len * ps.out_dims[k] < (int64_t(1) << 30)) len *= ps.out_dims[k--];
    PermRows p{};
    p.nouter = k + 1;
    p.len = (int)len;
    p.nrows = 1;
    for (int q = 0; q <= k; ++q) {
      p.dims[q] = (int)ps.out_dims[q];
      p.istr[q] = ps.in_stride[q];
      p.ostr[q] = ostr[q];
      p.nrows *= ps.out_dims[q];
    }
    constexpr int vec = 16 / (int)sizeof(Ti);
    // long rows are split into work items of 1024 elements (a warp moves 32 per access)
    p.chunk = 1024;
    p.nchunk = (int)((len + p.chunk - 1) / p.chunk);
    const int64_t warps = p.nrows * p.nchunk;
    const int bl = nblocks(warps, 8);
    bool aligned = std::is_same<Ti, To>::value && sizeof(Ti) >= 4 && len % vec == 0 &&
                   ((uintptr_t)in % 16) == 0 && ((uintptr_t)out % 16) == 0;
    for (int q = 0; q <= k && aligned; ++q) aligned = (p.istr[q] % vec == 0) && (p.ostr[q] % vec == 0);
    if (aligned) {
      if (acc)
        permute_rows<Ti, To, true, vec><<<bl, 256, 0, st>>>(in, out, p, scale);
      else
        permute_rows<Ti, To, false, vec><<<bl, 256, 0, st>>>(in, out, p, scale);
    } else {
      if (acc)
        permute_rows<Ti, To, true, 1><<<bl, 256, 0, st>>>(in, out, p, scale);
      else
        permute_rows<Ti, To, false, 1><<<bl, 256, 0, st>>>(in, out, p, scale);
    }
    CTM_LAUNCHED();
    return;
  }
  bool tiled = r >= 2 && ps.in_stride[r - 1] != 1 && b >= 0 && ps.out_dims[r - 1] >= 8 && ps.out_dims[b] >= 8;
  if (tiled) {
    PermTile p{};
    p.Na = ps.out_dims[r - 1];
    p.sa = ps.in_stride[r - 1];
    p.Nb = ps.out_dims[b];
    p.ob = ostr[b];
    p.nrest = 0;
    p.nrest_total = 1;
    for (int k = 0; k < r - 1; ++k) {
      if (k == b) continue;
      p.rdims[p.nrest] = ps.out_dims[k];
      p.ristr[p.nrest] = ps.in_stride[k];
      p.rostr[p.nrest] = ostr[k];
      p.nrest_total *= ps.out_dims[k];
      p.nrest++;
    }
    dim3 grid((unsigned)(((p.Na + 31) / 32) * ((p.Nb + 31) / 32)), (unsigned)std::min<int64_t>(p.nrest_total, 65535));
    dim3 block(32, 8);
    if (acc)
      permute_tiled<Ti, To, true><<<grid, block, 0, st>>>(in, out, p, scale);
    else
      permute_tiled<Ti, To, false><<<grid, block, 0, st>>>(in, out, p, scale);
  } else {
    PermDev p{};
    p.rank = r;
    for (int k = 0; k < r; ++k) {
      p.dims[k] = ps.out_dims[k];
      p.istr[k] = ps.in_stride[k];
    }
    int bl = nblocks(n, 256);
    if (acc)
      permute_generic<Ti, To, true><<<bl, 256, 0, st>>>(in, out, p, n, scale);
    else
      permute_generic<Ti, To, false><<<bl, 256, 0, st>>>(in, out, p, n, scale);
  }
  CTM_LAUNCHED();
}

// ------------------------------------------------------------------ SIMT GEMM
// Split-K: with nsplit > 1 the (split, batch) pairs form an extended batch; each block sums its
// K chunk and writes the raw partial tile to C (a workspace [nsplit][batch][M][N], ldc = N); a
// second kernel adds the partials in split order (deterministic) and applies alpha and beta.
// 256 threads as a 16 x 16 grid, each owning TM x TN outputs: tiles BM = 16 TM by BN = 16 TN.
// Shared memory is double-buffered and the next K tile is fetched into registers while the
// current one is multiplied, so one global-load latency is hidden per K step.
template <typename T, int TM, int TN, int BK>
__global__ void __launch_bounds__(256) gemm_simt(const T* __restrict__ A, const T* __restrict__ B, T* __restrict__ C,
                                                 GemmSpec g, int64_t nsplit, int64_t kchunk) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int LA = (BM * BK) / 256, LB = (BN * BK) / 256;
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t mtiles = (g.M + BM - 1) / BM;
  for (int64_t work = blockIdx.z * (int64_t)gridDim.y + blockIdx.y; work < nsplit * g.batch * mtiles;
       work += (int64_t)gridDim.z * gridDim.y) {
    const int64_t ext = work / mtiles;
    const int64_t m0 = (work % mtiles) * BM;
    const int64_t bb = ext % g.batch, sp = ext / g.batch;
    const int64_t kbeg = sp * kchunk, kend = min(g.K, kbeg + kchunk);
    const T* Ab = A + bb * g.strideA;
    const T* Bb = B + bb * g.strideB;
    T* Cb = (nsplit > 1) ? C + ext * g.M * g.N : C + bb * g.strideC;
    const int64_t ldc = (nsplit > 1) ? g.N : g.ldc;
    T ra[LA], rb[LB];
    // global -> registers for the K tile starting at k0
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int ml = g.transA ? e % BM : e / BK, kl = g.transA ? e / BM : e % BK;
        const int64_t m = m0 + ml, k = k0 + kl;
        ra[q] = (m < g.M && k < kend) ? (g.transA ? Ab[k * g.lda + m] : Ab[m * g.lda + k]) : T(0);
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int nl = g.transB ? e / BK : e % BN, kl = g.transB ? e % BK : e / BN;
        const int64_t n = n0 + nl, k = k0 + kl;
        rb[q] = (n < g.N && k < kend) ? (g.transB ? Bb[n * g.ldb + k] : Bb[k * g.ldb + n]) : T(0);
      }
    };
    // registers -> shared buffer `buf`
    auto stash = [&](int buf) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int ml = g.transA ? e % BM : e / BK, kl = g.transA ? e / BM : e % BK;
        As[buf][kl][ml] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int nl = g.transB ? e / BK : e % BN, kl = g.transB ? e % BK : e / BN;
        Bs[buf][kl][nl] = rb[q];
      }
    };
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    __syncthreads();  // the previous work item may still read both buffers
    fetch(kbeg);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) fetch(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int64_t m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int64_t n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        if (nsplit > 1) {
          Cb[m * ldc + n] = acc[i][j];
        } else {
          T v = (T)g.alpha * acc[i][j];
          if (g.beta != 0.0) v += (T)g.beta * Cb[m * ldc + n];
          Cb[m * ldc + n] = v;
        }
      }
    }
  }
}

// The same GEMM with every operand resolved through group maps (stride_map.h): A(b, m, k) at
// A[aB(b) + aM(m) + aK(k)], B(b, k, n) at B[bB(b) + bK(k) + bN(n)], C(b, m, n) at C[cB(b) + cM(m) +
// cN(n)] (split-K partials stay dense).  Products are added in the same order as gemm_simt; transA
// and transB only choose which index runs across neighbouring threads in the loads.
template <typename T, int TM, int TN, int BK>
__global__ void __launch_bounds__(256) gemm_simt_strided(const T* __restrict__ A, const T* __restrict__ B,
                                                         T* __restrict__ C, GemmSpec g, StridedGemm sm,
                                                         int64_t nsplit, int64_t kchunk) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int LA = (BM * BK) / 256, LB = (BN * BK) / 256;
  __shared__ T As[2][BK][BM + 1];
  __shared__ T Bs[2][BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t mtiles = (g.M + BM - 1) / BM;
  for (int64_t work = blockIdx.z * (int64_t)gridDim.y + blockIdx.y; work < nsplit * g.batch * mtiles;
       work += (int64_t)gridDim.z * gridDim.y) {
    const int64_t ext = work / mtiles;
    const int64_t m0 = (work % mtiles) * BM;
    const int64_t bb = ext % g.batch, sp = ext / g.batch;
    const int64_t kbeg = sp * kchunk, kend = min(g.K, kbeg + kchunk);
    const T* Ab = A + group_offset(sm.aB, bb);
    const T* Bb = B + group_offset(sm.bB, bb);
    // the M and N parts of this thread's load offsets do not change along K
    int64_t am[LA], bn[LB];
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int64_t m = m0 + (g.transA ? e % BM : e / BK);
      am[q] = m < g.M ? group_offset(sm.aM, m) : -1;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int64_t n = n0 + (g.transB ? e / BK : e % BN);
      bn[q] = n < g.N ? group_offset(sm.bN, n) : -1;
    }
    T ra[LA], rb[LB];
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int64_t k = k0 + (g.transA ? e / BM : e % BK);
        ra[q] = (am[q] >= 0 && k < kend) ? Ab[am[q] + group_offset(sm.aK, k)] : T(0);
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int64_t k = k0 + (g.transB ? e % BK : e / BN);
        rb[q] = (bn[q] >= 0 && k < kend) ? Bb[group_offset(sm.bK, k) + bn[q]] : T(0);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int q = 0; q < LA; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int ml = g.transA ? e % BM : e / BK, kl = g.transA ? e / BM : e % BK;
        As[buf][kl][ml] = ra[q];
      }
#pragma unroll
      for (int q = 0; q < LB; ++q) {
        const int e = threadIdx.x + 256 * q;
        const int nl = g.transB ? e / BK : e % BN, kl = g.transB ? e % BK : e / BN;
        Bs[buf][kl][nl] = rb[q];
      }
    };
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    __syncthreads();
    fetch(kbeg);
    stash(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) fetch(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (more) stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
    T* Cdense = C + ext * g.M * g.N;
    T* Cb = C + group_offset(sm.cB, bb);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int64_t m = m0 + ty + 16 * i;
      if (m >= g.M) continue;
      const int64_t cm = nsplit > 1 ? 0 : group_offset(sm.cM, m);
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        int64_t n = n0 + tx + 16 * j;
        if (n >= g.N) continue;
        if (nsplit > 1) {
          Cdense[m * g.N + n] = acc[i][j];
        } else {
          T* cp = Cb + cm + group_offset(sm.cN, n);
          T v = (T)g.alpha * acc[i][j];
          if (g.beta != 0.0) v += (T)g.beta * *cp;
          *cp = v;
        }
      }
    }
  }
}

template <typename T>
__global__ void splitk_reduce_strided(const T* __restrict__ W, T* __restrict__ C, GemmSpec g, StridedGemm sm,
                                      int64_t nsplit) {
  const int64_t per = g.M * g.N, total = g.batch * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per, r = e % per, m = r / g.N, n = r % g.N;
    T acc = T(0);
    for (int64_t s = 0; s < nsplit; ++s) acc += W[(s * g.batch + b) * per + r];
    T* c = C + group_offset(sm.cB, b) + group_offset(sm.cM, m) + group_offset(sm.cN, n);
    T v = (T)g.alpha * acc;
    if (g.beta != 0.0) v += (T)g.beta * *c;
    *c = v;
  }
}

template <typename T>
__global__ void splitk_reduce(const T* __restrict__ W, T* __restrict__ C, GemmSpec g, int64_t nsplit) {
  const int64_t per = g.M * g.N, total = g.batch * per;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per, r = e % per, m = r / g.N, n = r % g.N;
    T acc = T(0);
    for (int64_t s = 0; s < nsplit; ++s) acc += W[(s * g.batch + b) * per + r];
    T* c = C + b * g.strideC + m * g.ldc + n;
    T v = (T)g.alpha * acc;
    if (g.beta != 0.0) v += (T)g.beta * *c;
    *c = v;
  }
}

// Cached workspace of the split-K partial tiles, one per (host thread, device, stream): products
// enqueued on different streams may run at the same time.
struct SplitkWs {
  void* p = nullptr;
  size_t cap = 0;
};
thread_local std::map<std::pair<int, cudaStream_t>, SplitkWs> g_splitk_ws;

void* splitk_workspace(size_t bytes, cudaStream_t st) {
  int dev = 0;
  CTM_CUDA(cudaGetDevice(&dev));
  SplitkWs& w = g_splitk_ws[{dev, st}];
  if (bytes > w.cap) {
    if (w.p) {  // launches already enqueued on st may still read the old buffer
      CTM_CUDA(cudaStreamSynchronize(st));
      CTM_CUDA(cudaFree(w.p));
    }
    w.cap = std::max(bytes, size_t(64) << 20);
    CTM_CUDA(cudaMalloc(&w.p, w.cap));
  }
  return w.p;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    CTM_CUDA(cudaGetDevice(&dev));
    CTM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

// Tile and split-K decision shared by the dense and the strided GEMM (so that both add the
// same products in the same order).
struct GemmPlan {
  int64_t BT, nsplit, kchunk;
};

template <typename T>
GemmPlan gemm_plan(const GemmSpec& g) {
  // Tile: the largest of 64, 32 and 16 whose output tiles cover the SMs (FP64 is issue-bound at
  // about 2 FMA/clk/SM, so a product must reach every SM; FP32 stops at 32, where latency rather
  // than arithmetic is the limit).  K is then split while the tiles alone cannot fill the GPU:
  // FP64 into chunks of at least 16 (when K >= 64), FP32 into chunks of at least 128 (up to 256
  // chunks for outputs of a few elements with a long K).  The FP32 chunk also sets the summation
  // order of the mixed-precision gradient, whose agreement with FP64 after many unrolled
  // iterations depends on it (chunks of 64 gave a 1.7e-2 relative difference at 50 iterations of
  // the D=6, chi=64 workload, chunks of 128 give 7e-5).
  auto ntiles = [&](int64_t bt) { return g.batch * ((g.M + bt - 1) / bt) * ((g.N + bt - 1) / bt); };
  const int64_t sms = num_sms();
  int64_t BT = 64;
  if (ntiles(64) < (sizeof(T) == 8 ? 2 : 1) * sms || g.M < 64 || g.N < 64) BT = 32;
  if (sizeof(T) == 8 && BT == 32 && (ntiles(32) < sms || g.M < 32 || g.N < 32)) BT = 16;
  const int64_t tiles = ntiles(BT);
  const int64_t min_chunk = sizeof(T) == 8 ? 16 : 128;
  const int64_t max_split = sizeof(T) == 8 ? 64 : (tiles <= 4 ? 256 : 32);
  int64_t nsplit = 1;
  if (tiles < 2 * sms && g.K >= (sizeof(T) == 8 ? 64 : 2 * min_chunk)) {
    nsplit = std::min<int64_t>({(2 * sms + tiles - 1) / tiles, g.K / min_chunk, max_split});
    // workspace bound: 256 MB of partial tiles
    nsplit = std::min<int64_t>(nsplit, std::max<int64_t>(1, (int64_t(256) << 20) / ((int64_t)sizeof(T) * g.batch * g.M * g.N)));
    if (nsplit < 2) nsplit = 1;
  }
  const int64_t kchunk = ((g.K + nsplit - 1) / nsplit + 15) / 16 * 16;
  nsplit = (g.K + kchunk - 1) / kchunk;
  return {BT, nsplit, kchunk};
}

template <typename T>
void gemm_t(const T* A, const T* B, T* C, const GemmSpec& g, cudaStream_t st) {
  if (g.M == 0 || g.N == 0 || g.batch == 0) return;
  ProfScope ps(sizeof(T) == 8 ? PROF_GEMM64 : PROF_GEMM, st, 2.0 * g.batch * g.M * g.N * g.K,
               (double)sizeof(T) * g.batch * (g.M * g.K + g.K * g.N + (g.beta != 0.0 ? 2 : 1) * g.M * g.N),
               prof_tag(sizeof(T) == 8 ? "simt64" : "simt32", g.batch, g.M, g.N, g.K, g.transA * 2 + g.transB));
  if (g.K == 0) {  // C = beta C
    CTM_CHECK(g.beta == 0.0, CTM_ERR_INVALID_ARG, "gemm with K=0 and beta!=0 unsupported");
    for (int64_t b = 0; b < g.batch; ++b)
      for (int64_t m = 0; m < g.M; ++m) CTM_CUDA(cudaMemsetAsync(C + b * g.strideC + m * g.ldc, 0, g.N * sizeof(T), st));
    return;
  }
  const GemmPlan pl = gemm_plan<T>(g);
  const int64_t BT = pl.BT, nsplit = pl.nsplit, kchunk = pl.kchunk;
  T* out = C;
  if (nsplit > 1) out = (T*)splitk_workspace(sizeof(T) * nsplit * g.batch * g.M * g.N, st);
  const int64_t work = nsplit * g.batch * ((g.M + BT - 1) / BT);
  CTM_CHECK((g.N + BT - 1) / BT < (int64_t(1) << 31), CTM_ERR_INVALID_ARG, "gemm N too large");
  dim3 grid((unsigned)((g.N + BT - 1) / BT), (unsigned)std::min<int64_t>(work, 65535),
            (unsigned)std::min<int64_t>((work + 65534) / 65535, 65535));
  if (BT == 16)
    gemm_simt<T, 1, 1, 16><<<grid, 256, 0, st>>>(A, B, out, g, nsplit, kchunk);
  else if (BT == 32)
    gemm_simt<T, 2, 2, 16><<<grid, 256, 0, st>>>(A, B, out, g, nsplit, kchunk);
  else
    gemm_simt<T, 4, 4, 16><<<grid, 256, 0, st>>>(A, B, out, g, nsplit, kchunk);
  CTM_LAUNCHED();
  if (nsplit > 1) {
    splitk_reduce<T><<<nblocks(g.batch * g.M * g.N, 256), 256, 0, st>>>(out, C, g, nsplit);
    CTM_LAUNCHED();
  }
}

template <typename T>
void gemm_strided_t(const T* A, const T* B, T* C, const GemmSpec& g, const StridedGemm& sm, cudaStream_t st) {
  if (g.M == 0 || g.N == 0 || g.batch == 0) return;
  ProfScope ps(sizeof(T) == 8 ? PROF_GEMM64 : PROF_GEMM, st, 2.0 * g.batch * g.M * g.N * g.K,
               (double)sizeof(T) * g.batch * (g.M * g.K + g.K * g.N + (g.beta != 0.0 ? 2 : 1) * g.M * g.N),
               prof_tag(sizeof(T) == 8 ? "simt64s" : "simt32s", g.batch, g.M, g.N, g.K, g.transA * 2 + g.transB));
  CTM_CHECK(g.K > 0, CTM_ERR_INVALID_ARG, "strided gemm with K=0");
  const GemmPlan pl = gemm_plan<T>(g);
  const int64_t BT = pl.BT, nsplit = pl.nsplit, kchunk = pl.kchunk;
  T* out = C;
  if (nsplit > 1) out = (T*)splitk_workspace(sizeof(T) * nsplit * g.batch * g.M * g.N, st);
  const int64_t work = nsplit * g.batch * ((g.M + BT - 1) / BT);
  CTM_CHECK((g.N + BT - 1) / BT < (int64_t(1) << 31), CTM_ERR_INVALID_ARG, "gemm N too large");
  dim3 grid((unsigned)((g.N + BT - 1) / BT), (unsigned)std::min<int64_t>(work, 65535),
            (unsigned)std::min<int64_t>((work + 65534) / 65535, 65535));
  if (BT == 16)
    gemm_simt_strided<T, 1, 1, 16><<<grid, 256, 0, st>>>(A, B, out, g, sm, nsplit, kchunk);
  else if (BT == 32)
    gemm_simt_strided<T, 2, 2, 16><<<grid, 256, 0, st>>>(A, B, out, g, sm, nsplit, kchunk);
  else
    gemm_simt_strided<T, 4, 4, 16><<<grid, 256, 0, st>>>(A, B, out, g, sm, nsplit, kchunk);
  CTM_LAUNCHED();
  if (nsplit > 1) {
    splitk_reduce_strided<T><<<nblocks(g.batch * g.M * g.N, 256), 256, 0, st>>>(out, C, g, sm, nsplit);
    CTM_LAUNCHED();
  }
}

// ------------------------------------------------------------------ element-wise
template <typename T>
__global__ void fill_k(T* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = from_d<T>(v);
}

template <typename Ti, typename To, bool ACC>
__global__ void cast_k(const Ti* in, To* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = to_d(in[i]);
    if (ACC) v += to_d(out[i]);
    out[i] = from_d<To>(v);
  }
}

template <typename T>
__global__ void sumsq_partial(const T* x, int64_t n, double* part) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = to_d(x[i]);
    s = fma(v, v, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void sum_final(const double* part, int n, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

template <typename T>
__global__ void scale_rsqrt_k(const T* x, int64_t n, const double* ss, T* y, double* inv) {
  double s = *ss;
  double f = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && inv) *inv = f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = from_d<T>(to_d(x[i]) * f);
}

template <typename T, bool ACC>
__global__ void scale_by_k(const T* dy, int64_t n, const double* inv, T* dx) {
  double f = *inv;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = to_d(dy[i]) * f;
    if (ACC) v += to_d(dx[i]);
    dx[i] = from_d<T>(v);
  }
}

// ------------------------------------------------------------------ projector helpers
__global__ void proj_prepare_k(const double* lam, double* U, double* V, double* inv, double* sinv, int64_t n_r, int r,
                               int kept, double cut, double rank_tol, int* status) {
  const int b = blockIdx.y;
  const double* l = lam + (int64_t)b * r;
  const double l0 = l[0];
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      double v = l[k];
      if (!isfinite(v)) atomicOr(status, DEV_NONFINITE);
      sinv[(int64_t)b * r + k] = (v > rank_tol * l0) ? 1.0 / v : 0.0;
      if (k < kept) inv[(int64_t)b * kept + k] = (v > cut * l0) ? 1.0 / sqrt(v) : 0.0;
    }
    if (threadIdx.x == 0 && !(l0 > 0.0)) atomicOr(status, DEV_DEGENERATE);
  }
  int64_t total = n_r * r;
  double* Ub = U + (int64_t)b * total;
  double* Vb = V + (int64_t)b * total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e % r);
    if (!(l[k] > rank_tol * l0)) {
      Ub[e] = 0.0;
      Vb[e] = 0.0;
    }
  }
}

// Sign gauge of the singular triplets: column k of V (n x r, row-major) is made to have its
// entry of largest magnitude (first one on ties) positive; U's column k follows.
__global__ void sign_fix_k(double* U, double* V, int64_t n, int r) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (k >= r) return;
  double* Ub = U + (int64_t)b * n * r;
  double* Vb = V + (int64_t)b * n * r;
  double best = -1.0, val = 0.0;
  int64_t bi = 0;
  for (int64_t i = lane; i < n; i += 32) {
    double v = Vb[i * r + k];
    if (fabs(v) > best) {
      best = fabs(v);
      val = v;
      bi = i;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    double ov = __shfl_xor_sync(0xffffffffu, val, o);
    int64_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      val = ov;
      bi = oi;
    }
  }
  if (val < 0.0)
    for (int64_t i = lane; i < n; i += 32) {
      Vb[i * r + k] = -Vb[i * r + k];
      Ub[i * r + k] = -Ub[i * r + k];
    }
}

// Sign gauge against a reference: column k of V (n x ld row-major, k < ncols) is flipped together
// with U's column k when its overlap with column k of Vref (n x ldr row-major) is negative.
__global__ void sign_align_k(double* U, double* V, int64_t ld, const double* Vref, int64_t ldr, int64_t n, int ncols) {
  const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (k >= ncols) return;
  double dot = 0.0;
  for (int64_t i = lane; i < n; i += 32) dot = fma(V[i * ld + k], Vref[i * ldr + k], dot);
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (dot < 0.0)
    for (int64_t i = lane; i < n; i += 32) {
      V[i * ld + k] = -V[i * ld + k];
      U[i * ld + k] = -U[i * ld + k];
    }
}

__global__ void scale_cols_k(const double* Y, int64_t ldy, int64_t strideY, const double* s, int64_t strideS, double* X,
                             int64_t n, int kept) {
  const int b = blockIdx.y;
  int64_t total = n * kept;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / kept;
    int k = (int)(e % kept);
    X[(int64_t)b * total + e] = Y[(int64_t)b * strideY + i * ldy + k] * s[(int64_t)b * strideS + k];
  }
}

__global__ void proj_dlam_k(const double* dZ, const double* U, const double* dW, const double* V, const double* inv,
                            double* dl, int64_t n_r, int r, int kept) {
  const int b = blockIdx.y;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int k = blockIdx.x * (blockDim.x / 32) + warp;
  if (k >= kept) return;
  const double* dZb = dZ + (int64_t)b * n_r * kept;
  const double* dWb = dW + (int64_t)b * n_r * kept;
  const double* Ub = U + (int64_t)b * n_r * r;
  const double* Vb = V + (int64_t)b * n_r * r;
  double s = 0.0;
  for (int64_t i = lane; i < n_r; i += 32) {
    s = fma(dZb[i * kept + k], Ub[i * r + k], s);
    s = fma(dWb[i * kept + k], Vb[i * r + k], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double iv = inv[(int64_t)b * kept + k];
    dl[(int64_t)b * kept + k] = -0.5 * iv * iv * iv * s;
  }
}

__global__ void proj_core_k(const double* Aa, const double* Bb, const double* lam, const double* dl, double* core, int r,
                            int kept, double rank_tol, double eps) {
  const int b = blockIdx.y;
  const double* l = lam + (int64_t)b * r;
  const double l0 = l[0];
  const double* A = Aa + (int64_t)b * r * kept;
  const double* B = Bb + (int64_t)b * r * kept;
  int64_t total = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(e / r), j = (int)(e % r);
    double li = l[i], lj = l[j];
    double v = 0.0;
    if (i == j) {
      if (i < kept) v = dl[(int64_t)b * kept + i];
    } else if (li > rank_tol * l0 && lj > rank_tol * l0) {
      // Lorentzian broadening on the pair's own scale: only numerically degenerate pairs
      // (relative gap at the rounding level) are damped
      double diff = lj * lj - li * li;
      double sc = lj * lj + li * li;
      double F = diff / (diff * diff + eps * sc * sc);
      double aij = (j < kept) ? A[(int64_t)i * kept + j] : 0.0;
      double aji = (i < kept) ? A[(int64_t)j * kept + i] : 0.0;
      double bij = (j < kept) ? B[(int64_t)i * kept + j] : 0.0;
      double bji = (i < kept) ? B[(int64_t)j * kept + i] : 0.0;
      v = F * (aij - aji) * lj + li * F * (bij - bji);
    }
    core[(int64_t)b * total + e] = v;
  }
}

__global__ void proj_resid_k(const double* dU, const double* X, const double* sinv, double* E, int64_t n_r, int r,
                             int kept) {
  const int b = blockIdx.y;
  int64_t total = n_r * kept;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e % kept);
    int64_t o = (int64_t)b * total + e;
    E[o] = (dU[o] - X[o]) * sinv[(int64_t)b * r + k];
  }
}

// ------------------------------------------------------------------ energy
__global__ void energy_k(const double* rho, const double* hs, const double* coup, int n_terms, int d2, double inv_sites,
                         double* e_bond, double* e_site, double* drho, int* status) {
  __shared__ double es[64];
  __shared__ double trs[64];
  const int t = threadIdx.x;
  if (t < n_terms) {
    const double* R = rho + (int64_t)t * d2 * d2;
    const double* H = hs + (int64_t)t * d2 * d2;
    double tr = 0.0, num = 0.0;
    for (int a = 0; a < d2; ++a) {
      tr += R[a * d2 + a];
      for (int c = 0; c < d2; ++c) num = fma(R[a * d2 + c], H[c * d2 + a], num);
    }
    double e = num / tr;
    if (!isfinite(e)) atomicOr(status, DEV_NONFINITE);
    es[t] = e;
    trs[t] = tr;
    if (e_bond) e_bond[t] = e;
  }
  __syncthreads();
  if (t == 0) {
    double E = 0.0;
    for (int k = 0; k < n_terms; ++k) E += coup[k] * es[k];
    *e_site = E * inv_sites;
  }
  if (drho && t < n_terms) {
    const double* H = hs + (int64_t)t * d2 * d2;
    double f = coup[t] * inv_sites / trs[t];
    for (int a = 0; a < d2; ++a)
      for (int c = 0; c < d2; ++c) drho[(int64_t)t * d2 * d2 + a * d2 + c] = f * (H[c * d2 + a] - (a == c ? es[t] : 0.0));
  }
}

// x = hi + lo with hi = x rounded to the nearest TF32 number (10-bit mantissa) and lo = x - hi
// (exact in FP32); lo is itself rounded to TF32 so that the tensor core reads it unchanged.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & 0xFFFFE000u;
  return __uint_as_float(u);
}

__global__ void split_tf32_k(const float* x, float* hi, float* lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = x[i];
    float h = tf32_round(v);
    hi[i] = h;
    lo[i] = tf32_round(v - h);
  }
}

// x = hi + lo with hi = x rounded to BF16 and lo = (x - hi) rounded to BF16 (about 16
// significant bits in all; the rest of x is dropped).
__global__ void split_bf16_k(const float* x, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

__global__ void embed_t_k(const double* U, int r, double* X, int64_t m) {
  int64_t total = (int64_t)r * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t k = e / m, i = e % m;
    X[e] = (i < r) ? U[i * r + k] : 0.0;
  }
}

__global__ void spectrum_delta_k(const double* lam, const double* prev, int batch, int r, int kept, double* out) {
  __shared__ double sh[256];
  double best = 0.0;
  for (int b = 0; b < batch; ++b) {
    const double* l = lam + (int64_t)b * r;
    const double* p = prev + (int64_t)b * r;
    double sl = 0.0, sp = 0.0;
    for (int k = 0; k < kept; ++k) {
      sl += l[k];
      sp += p[k];
    }
    for (int k = threadIdx.x; k < kept; k += blockDim.x) {
      double v = fabs(l[k] / sl - p[k] / sp);
      best = v > best ? v : best;
    }
  }
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = fmax(*out, sh[0]);
}

}  // namespace

// ================================================================== host wrappers
#define DISPATCH_IO(tin, tout, F)                                                                           \
  if (tin == F64 && tout == F64) { F(double, double); }                                                     \
  else if (tin == F64 && tout == F32) { F(double, float); }                                                 \
  else if (tin == F32 && tout == F64) { F(float, double); }                                                 \
  else if (tin == F32 && tout == F32) { F(float, float); }                                                  \
  else if (tin == F32 && tout == BF16) { F(float, __nv_bfloat16); }                                         \
  else if (tin == F64 && tout == BF16) { F(double, __nv_bfloat16); }                                        \
  else if (tin == BF16 && tout == F32) { F(__nv_bfloat16, float); }                                         \
  else throw Error(CTM_ERR_INVALID_ARG, "unsupported dtype pair");

void permute(const void* in, DType tin, void* out, DType tout, const PermSpec& p, bool acc, double scale,
             cudaStream_t st) {
#define F(Ti, To) permute_t<Ti, To>((const Ti*)in, (To*)out, p, acc, scale, st)
  DISPATCH_IO(tin, tout, F)
#undef F
}

void gemm_f64(const double* A, const double* B, double* C, const GemmSpec& g, cudaStream_t st) { gemm_t(A, B, C, g, st); }
void gemm_f32(const float* A, const float* B, float* C, const GemmSpec& g, cudaStream_t st) { gemm_t(A, B, C, g, st); }
void gemm_strided_f64(const double* A, const double* B, double* C, const GemmSpec& g, const StridedGemm& sm,
                      cudaStream_t st) {
  gemm_strided_t(A, B, C, g, sm, st);
}
void gemm_strided_f32(const float* A, const float* B, float* C, const GemmSpec& g, const StridedGemm& sm,
                      cudaStream_t st) {
  gemm_strided_t(A, B, C, g, sm, st);
}

void fill(void* p, DType t, int64_t n, double v, cudaStream_t st) {
  if (n == 0) return;
  int bl = nblocks(n, 256);
  if (t == F64) fill_k<double><<<bl, 256, 0, st>>>((double*)p, n, v);
  else if (t == F32) fill_k<float><<<bl, 256, 0, st>>>((float*)p, n, v);
  else fill_k<__nv_bfloat16><<<bl, 256, 0, st>>>((__nv_bfloat16*)p, n, v);
  CTM_LAUNCHED();
}

void cast(const void* in, DType tin, void* out, DType tout, int64_t n, bool acc, cudaStream_t st) {
  if (n == 0) return;
  int bl = nblocks(n, 256);
#define F(Ti, To)                                                                \
  if (acc) cast_k<Ti, To, true><<<bl, 256, 0, st>>>((const Ti*)in, (To*)out, n); \
  else cast_k<Ti, To, false><<<bl, 256, 0, st>>>((const Ti*)in, (To*)out, n);
  DISPATCH_IO(tin, tout, F)
#undef F
  CTM_LAUNCHED();
}

void sumsq(const void* x, DType t, int64_t n, double* out, double* work, cudaStream_t st) {
  int bl = (int)std::min<int64_t>(1024, std::max<int64_t>(1, (n + 1023) / 1024));
  if (t == F64) sumsq_partial<double><<<bl, 256, 0, st>>>((const double*)x, n, work);
  else sumsq_partial<float><<<bl, 256, 0, st>>>((const float*)x, n, work);
  CTM_LAUNCHED();
  sum_final<<<1, 256, 0, st>>>(work, bl, out);
  CTM_LAUNCHED();
}

void scale_rsqrt(const void* x, DType t, int64_t n, const double* ss, void* y, double* inv, cudaStream_t st) {
  int bl = nblocks(n, 256);
  if (t == F64) scale_rsqrt_k<double><<<bl, 256, 0, st>>>((const double*)x, n, ss, (double*)y, inv);
  else scale_rsqrt_k<float><<<bl, 256, 0, st>>>((const float*)x, n, ss, (float*)y, inv);
  CTM_LAUNCHED();
}

void scale_by(const void* dy, DType t, int64_t n, const double* inv, void* dx, bool acc, cudaStream_t st) {
  int bl = nblocks(n, 256);
  if (t == F64) {
    if (acc) scale_by_k<double, true><<<bl, 256, 0, st>>>((const double*)dy, n, inv, (double*)dx);
    else scale_by_k<double, false><<<bl, 256, 0, st>>>((const double*)dy, n, inv, (double*)dx);
  } else {
    if (acc) scale_by_k<float, true><<<bl, 256, 0, st>>>((const float*)dy, n, inv, (float*)dx);
    else scale_by_k<float, false><<<bl, 256, 0, st>>>((const float*)dy, n, inv, (float*)dx);
  }
  CTM_LAUNCHED();
}

void proj_prepare(const double* lam, double* U, double* V, double* inv, double* sinv, int batch, int64_t n_r, int r,
                  int kept, double cut, double rank_tol, int* status, cudaStream_t st) {
  dim3 grid(nblocks(n_r * r, 256, 4096), batch);
  proj_prepare_k<<<grid, 256, 0, st>>>(lam, U, V, inv, sinv, n_r, r, kept, cut, rank_tol, status);
  CTM_LAUNCHED();
}

void sign_fix(double* U, double* V, int batch, int64_t n, int r, cudaStream_t st) {
  dim3 grid((r + 7) / 8, batch);
  sign_fix_k<<<grid, 256, 0, st>>>(U, V, n, r);
  CTM_LAUNCHED();
}

void sign_align(double* U, double* V, int64_t ld, const double* Vref, int64_t ldr, int64_t n, int ncols,
                cudaStream_t st) {
  if (ncols <= 0) return;
  sign_align_k<<<(ncols + 7) / 8, 256, 0, st>>>(U, V, ld, Vref, ldr, n, ncols);
  CTM_LAUNCHED();
}

void scale_cols(const double* Y, int64_t ldy, int64_t strideY, const double* s, int64_t strideS, double* X, int batch,
                int64_t n, int kept, cudaStream_t st) {
  dim3 grid(nblocks(n * kept, 256, 4096), batch);
  scale_cols_k<<<grid, 256, 0, st>>>(Y, ldy, strideY, s, strideS, X, n, kept);
  CTM_LAUNCHED();
}

void proj_dlam(const double* dZ, const double* U, const double* dW, const double* V, const double* inv, double* dl,
               int batch, int64_t n_r, int r, int kept, cudaStream_t st) {
  dim3 grid((kept + 7) / 8, batch);
  proj_dlam_k<<<grid, 256, 0, st>>>(dZ, U, dW, V, inv, dl, n_r, r, kept);
  CTM_LAUNCHED();
}

void proj_core(const double* Aa, const double* Bb, const double* lam, const double* dl, double* core, int batch, int r,
               int kept, double rank_tol, double eps, cudaStream_t st) {
  dim3 grid(nblocks((int64_t)r * r, 256, 4096), batch);
  proj_core_k<<<grid, 256, 0, st>>>(Aa, Bb, lam, dl, core, r, kept, rank_tol, eps);
  CTM_LAUNCHED();
}

void proj_resid(const double* dU, const double* X, const double* sinv, double* E, int batch, int64_t n_r, int r,
                int kept, cudaStream_t st) {
  dim3 grid(nblocks(n_r * kept, 256, 4096), batch);
  proj_resid_k<<<grid, 256, 0, st>>>(dU, X, sinv, E, n_r, r, kept);
  CTM_LAUNCHED();
}

// ------------------------------------------------------------------ observables (FP64)
// Per PEPS site, rho is the 2 x 2 one-site RDM [ket s][bra s'] (basis up, down).  For spin 1/2,
// <S_x> = (rho_01 + rho_10) / (2 Tr rho), <S_z> = (rho_00 - rho_11) / (2 Tr rho); with real tensors
// Tr(rho S_y) is purely imaginary and its real part, the expectation value, is 0.
__global__ void magnetization_k(const double* rho, int n_sites, double* m, double* M, int* status) {
  __shared__ double acc[64];
  const int t = threadIdx.x;
  double len = 0.0;
  if (t < n_sites) {
    const double* r = rho + 4 * t;
    const double tr = r[0] + r[3];
    if (!(fabs(tr) > 0.0) || !isfinite(tr)) atomicOr(status, DEV_NONFINITE);
    const double sx = 0.5 * (r[1] + r[2]) / tr, sz = 0.5 * (r[0] - r[3]) / tr;
    m[3 * t + 0] = sx;
    m[3 * t + 1] = 0.0;
    m[3 * t + 2] = sz;
    len = sqrt(sx * sx + sz * sz);
  }
  acc[t] = len;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int k = 0; k < n_sites; ++k) sum += acc[k];
    *M = sum / n_sites;
  }
}

// M_p = |sum_{a in A} e_a - sum_{b in B} e_b| / 4 over the listed per-term values
__global__ void plaquette_k(const double* e, const int* idx, int na, int nb, double* Mp) {
  if (threadIdx.x != 0) return;
  double sa = 0.0, sb = 0.0;
  for (int k = 0; k < na; ++k) sa += e[idx[k]];
  for (int k = 0; k < nb; ++k) sb += e[idx[na + k]];
  *Mp = 0.25 * fabs(sa - sb);
}

void site_magnetization(const double* rho, int n_sites, double* m, double* M, int* status, cudaStream_t st) {
  CTM_CHECK(n_sites >= 1 && n_sites <= 64, CTM_ERR_INVALID_ARG, "magnetization: 1..64 sites");
  magnetization_k<<<1, 64, 0, st>>>(rho, n_sites, m, M, status);
  CTM_LAUNCHED();
}

void plaquette_order(const double* e_terms, const int* idx_dev, int na, int nb, double* Mp, cudaStream_t st) {
  plaquette_k<<<1, 32, 0, st>>>(e_terms, idx_dev, na, nb, Mp);
  CTM_LAUNCHED();
}

void energy_terms(const double* rho, const double* hs, const double* coup, int n_terms, int d2, double inv_sites,
                  double* e_bond, double* e_site, double* drho, int* status, cudaStream_t st) {
  CTM_CHECK(n_terms <= 64, CTM_ERR_INVALID_ARG, "at most 64 terms");
  energy_k<<<1, 64, 0, st>>>(rho, hs, coup, n_terms, d2, inv_sites, e_bond, e_site, drho, status);
  CTM_LAUNCHED();
}

void split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  ProfScope prof(PROF_PERMUTE, st, 0.0, 12.0 * n, prof_tag("split_tf32", 1, n, 0, 0));
  split_tf32_k<<<nblocks(n, 256), 256, 0, st>>>(x, hi, lo, n);
  CTM_LAUNCHED();
}

void split_bf16(const float* x, void* hi, void* lo, int64_t n, cudaStream_t st) {
  if (n == 0) return;
  ProfScope prof(PROF_PERMUTE, st, 0.0, 8.0 * n, prof_tag("split_bf16", 1, n, 0, 0));
  split_bf16_k<<<nblocks(n, 256), 256, 0, st>>>(x, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo, n);
  CTM_LAUNCHED();
}

void embed_transpose(const double* U, int r, double* X, int64_t m, cudaStream_t st) {
  embed_t_k<<<nblocks((int64_t)r * m, 256, 4096), 256, 0, st>>>(U, r, X, m);
  CTM_LAUNCHED();
}

void spectrum_delta(const double* lam, const double* lam_prev, int batch, int r, int kept, double* out, cudaStream_t st) {
  spectrum_delta_k<<<1, 256, 0, st>>>(lam, lam_prev, batch, r, kept, out);
  CTM_LAUNCHED();
}

}  // namespace ctm
