// Pairing schedule of the block-cyclic one-sided Jacobi (jacobi_block_kernel), usable on the host
// as well so that its covering property can be checked without a GPU.
//
// The r columns form G groups of 4 (G even, columns past r are padding).  A sweep is G - 1 outer
// rounds; in outer round k the groups are paired by the circle method (position 0 fixed, the other
// G - 1 positions rotated by k), pair j = (group at position j, group at position G - 1 - j).  A
// block holding groups (a, b) stages their 8 columns in slots 0..3 (a) and 4..7 (b) and runs inner
// rounds of 4 disjoint slot pairs, one per warp: in outer round 0 first the 3 rounds inside each
// group ((0,1)(2,3), (0,2)(1,3), (0,3)(1,2)), then in every outer round the 4 cross rounds
// (a_w, b_{(w + t) mod 4}).  Every column pair then meets exactly once per sweep.
#pragma once

#ifndef __CUDACC__
#define JO_HD inline
#else
#define JO_HD __host__ __device__ __forceinline__
#endif

namespace ctm {

// Group at position p of outer round k of the circle method over G groups.
JO_HD int circle_group(int k, int p, int G) { return p == 0 ? 0 : 1 + ((p - 1 - k) % (G - 1) + (G - 1)) % (G - 1); }

// Inner rounds of outer round k.
JO_HD int block_inner_rounds(int k) { return k == 0 ? 7 : 4; }

// Slots (p, q) rotated by warp wid (0..3) in inner round it of outer round k.
JO_HD void block_pair(int k, int it, int wid, int& p, int& q) {
  if (k == 0 && it < 3) {
    const int base = (wid < 2) ? 0 : 4, w2 = wid % 2;
    p = base + (it == 0 ? 2 * w2 : w2);
    q = base + (it == 0 ? 2 * w2 + 1 : (it == 1 ? w2 + 2 : 3 - w2));
  } else {
    const int tt = (k == 0) ? it - 3 : it;
    p = wid;
    q = 4 + (wid + tt) % 4;
  }
}

}  // namespace ctm
