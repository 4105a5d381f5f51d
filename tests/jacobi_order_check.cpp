// Host check of the block-cyclic Jacobi schedule (paper_2512_14414_gb300/csrc/jacobi_order.h): for
// several matrix sizes, every pair of real columns is rotated exactly once per sweep, and the pairs
// that run at the same time (one inner round, all blocks of an outer round) share no column.
#include <cstdio>
#include <vector>

#include "../paper_2512_14414_gb300/csrc/jacobi_order.h"

static int check(int r) {
  const int G = ((r + 7) / 8) * 2;
  std::vector<int> seen((size_t)r * r, 0);
  for (int k = 0; k < G - 1; ++k) {
    std::vector<int> group_used(G, 0);
    for (int j = 0; j < G / 2; ++j) {
      const int ga = ctm::circle_group(k, j, G), gb = ctm::circle_group(k, G - 1 - j, G);
      if (ga == gb || group_used[ga]++ || group_used[gb]++) return printf("r=%d k=%d: groups overlap\n", r, k), 1;
      for (int it = 0; it < ctm::block_inner_rounds(k); ++it) {
        int slot_used[8] = {0};
        for (int w = 0; w < 4; ++w) {
          int p, q;
          ctm::block_pair(k, it, w, p, q);
          if (p < 0 || p > 7 || q < 0 || q > 7 || p == q || slot_used[p]++ || slot_used[q]++)
            return printf("r=%d k=%d it=%d: slots overlap\n", r, k, it), 1;
          const int cp = p < 4 ? ga * 4 + p : gb * 4 + p - 4;
          const int cq = q < 4 ? ga * 4 + q : gb * 4 + q - 4;
          if (cp < r && cq < r) {
            const int a = cp < cq ? cp : cq, b = cp < cq ? cq : cp;
            seen[(size_t)a * r + b]++;
          }
        }
      }
    }
  }
  for (int a = 0; a < r; ++a)
    for (int b = a + 1; b < r; ++b)
      if (seen[(size_t)a * r + b] != 1) return printf("r=%d pair (%d,%d) seen %d times\n", r, a, b, seen[(size_t)a * r + b]), 1;
  return 0;
}

int main() {
  const int sizes[] = {1, 2, 5, 8, 9, 16, 63, 64, 100, 127, 128, 129, 255, 256, 383, 384};
  for (int r : sizes)
    if (check(r)) return 1;
  printf("ok\n");
  return 0;
}
