// Strided views of tensor operands for the GEMM lowering of a pairwise contraction.
//
// A contraction reads A as [batch | M | K] and B as [batch | K | N] and writes C as
// [batch | M | N], where batch, M, K and N are groups of tensor labels.  Instead of permuting a
// tensor into that order, a GroupMap describes one group inside the tensor's own row-major
// layout: the group's flat index (its labels in group order, last fastest) unravels into one
// index per label, and the element offset is the sum of index * stride.  Labels that are
// adjacent and contiguous in memory are merged, so most groups need one or two terms.
// Plain C++ (no CUDA types) so that the host-side construction can be tested on its own.
#pragma once
#include <cstdint>
#include <vector>

#if defined(__CUDACC__)
#define CTM_HD __host__ __device__ __forceinline__
#else
#define CTM_HD inline
#endif

namespace ctm {

struct GroupMap {
  int n = 0;             // number of (merged) dimensions; 0 = the group is empty (offset 0)
  int64_t dim[8] = {0};  // sizes, outermost first
  int64_t stride[8] = {0};
};

// Element offset of flat group index i (0 <= i < product of dim).
CTM_HD int64_t group_offset(const GroupMap& g, int64_t i) {
  int64_t off = 0;
  for (int d = g.n - 1; d >= 0; --d) {
    const int64_t q = i / g.dim[d];
    off += (i - q * g.dim[d]) * g.stride[d];
    i = q;
  }
  return off;
}

// The map of `group` (labels, in the order they are enumerated) inside a row-major tensor
// whose labels are `ls` with sizes `size_of(label)`.  Returns false if a label is missing or the
// group has more than 8 dimensions after merging.
template <typename SizeOf>
bool build_group_map(const std::vector<int>& ls, const std::vector<int>& group, SizeOf size_of, GroupMap& out) {
  std::vector<int64_t> str(ls.size());
  int64_t s = 1;
  for (int k = (int)ls.size() - 1; k >= 0; --k) {
    str[k] = s;
    s *= size_of(ls[k]);
  }
  std::vector<int64_t> dm, st;
  for (int lab : group) {
    int pos = -1;
    for (size_t k = 0; k < ls.size(); ++k)
      if (ls[k] == lab) pos = (int)k;
    if (pos < 0) return false;
    const int64_t d = size_of(lab), sd = str[pos];
    if (d == 1) continue;  // a size-1 label contributes nothing
    if (!dm.empty() && st.back() == sd * d) {  // previous label is the next-outer one in memory
      dm.back() *= d;
      st.back() = sd;
    } else {
      dm.push_back(d);
      st.push_back(sd);
    }
  }
  if (dm.size() > 8) return false;
  out = GroupMap();
  out.n = (int)dm.size();
  for (int k = 0; k < out.n; ++k) {
    out.dim[k] = dm[k];
    out.stride[k] = st[k];
  }
  return true;
}

// Strided GEMM description: C(b, m, n) (+)= sum_k A(b, m, k) B(b, k, n) with every index of
// every operand resolved through its group maps.
struct StridedGemm {
  GroupMap aB, aM, aK;  // A = GEMM's first operand
  GroupMap bB, bK, bN;  // B = GEMM's second operand
  GroupMap cB, cM, cN;  // C
};

}  // namespace ctm
