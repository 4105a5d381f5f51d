// CPU check of the GEMM group maps (paper_2512_14414_gb300/csrc/stride_map.h): for random tensors,
// label orders and (batch, M, K) groupings, the offsets from the maps equal the direct row-major
// offsets of every element, and stay inside the tensor.  Prints "ok <cases>" or the first failure.
#include <algorithm>
#include <cstdio>
#include <map>
#include <random>
#include <vector>

#include "../paper_2512_14414_gb300/csrc/stride_map.h"

int main() {
  std::mt19937 rng(20251214);
  int cases = 0;
  for (int trial = 0; trial < 3000; ++trial) {
    const int rank = 1 + rng() % 6;
    std::vector<int> ls(rank);
    std::map<int, int64_t> dim;
    for (int k = 0; k < rank; ++k) ls[k] = 10 + k, dim[10 + k] = 1 + rng() % 4;
    std::vector<int> perm = ls;
    std::shuffle(perm.begin(), perm.end(), rng);
    // split the permuted labels into three consecutive groups (any of them may be empty)
    int c1 = rng() % (rank + 1), c2 = c1 + rng() % (rank - c1 + 1);
    std::vector<int> G[3] = {std::vector<int>(perm.begin(), perm.begin() + c1),
                             std::vector<int>(perm.begin() + c1, perm.begin() + c2),
                             std::vector<int>(perm.begin() + c2, perm.end())};
    auto size_of = [&](int l) { return dim.at(l); };
    ctm::GroupMap gm[3];
    for (int q = 0; q < 3; ++q)
      if (!ctm::build_group_map(ls, G[q], size_of, gm[q])) {
        printf("build failed in trial %d\n", trial);
        return 1;
      }
    int64_t total = 1;
    for (int l : ls) total *= dim[l];
    int64_t n[3];
    for (int q = 0; q < 3; ++q) {
      n[q] = 1;
      for (int l : G[q]) n[q] *= dim[l];
    }
    for (int64_t i0 = 0; i0 < n[0]; ++i0)
      for (int64_t i1 = 0; i1 < n[1]; ++i1)
        for (int64_t i2 = 0; i2 < n[2]; ++i2) {
          // direct: unravel each group index over its labels, then the row-major offset in ls
          std::map<int, int64_t> idx;
          int64_t is[3] = {i0, i1, i2};
          for (int q = 0; q < 3; ++q) {
            int64_t r = is[q];
            for (int k = (int)G[q].size() - 1; k >= 0; --k) {
              idx[G[q][k]] = r % dim[G[q][k]];
              r /= dim[G[q][k]];
            }
          }
          int64_t direct = 0;
          for (int l : ls) direct = direct * dim[l] + idx[l];
          const int64_t mapped = ctm::group_offset(gm[0], i0) + ctm::group_offset(gm[1], i1) + ctm::group_offset(gm[2], i2);
          if (mapped != direct || mapped < 0 || mapped >= total) {
            printf("mismatch in trial %d: mapped %lld direct %lld total %lld\n", trial, (long long)mapped,
                   (long long)direct, (long long)total);
            return 1;
          }
        }
    ++cases;
  }
  printf("ok %d\n", cases);
  return 0;
}
