// Host check of the tcgen05 operand tile layout (umma_layout.h): every (row, feature) bf16 pair
// of an R-row tile gets its own 4-byte slot inside the tile, the slots tile it exactly, and
// every bf16 element sits where the K-major core-matrix layout with the descriptor's leading
// (K) and stride (M/N) byte offsets puts it. Prints "ok" or the first violation.
#include <stdio.h>

#include <vector>

#include "umma_layout.h"

using namespace mlmc::umma;

static int check(int R) {
  std::vector<int> seen((size_t)R * 32, 0);
  for (int r = 0; r < R; ++r)
    for (int f = 0; f < 8; ++f) {
      const int o = pair_offset(r, f);
      if (o < 0 || o + 4 > R * 32 || o % 4 != 0) {
        printf("R=%d: pair (%d,%d) at %d outside the tile\n", R, r, f, o);
        return 1;
      }
      for (int b = 0; b < 4; ++b)
        if (seen[o + b]++) {
          printf("R=%d: byte %d written twice\n", R, o + b);
          return 1;
        }
      for (int e = 0; e < 2; ++e) {  // k = 2 f + e: Re, Im
        const int k = 2 * f + e;
        const int canon = (r / 8) * kStrideBytes + (k / 8) * kLeadingBytes + (r % 8) * 16 + (k % 8) * 2;
        if (canon != o + 2 * e) {
          printf("R=%d: element (%d,%d) at %d, core-matrix layout %d\n", R, r, k, o + 2 * e, canon);
          return 1;
        }
      }
    }
  for (int i = 0; i < R * 32; ++i)
    if (seen[i] != 1) {
      printf("R=%d: byte %d not covered\n", R, i);
      return 1;
    }
  // a core matrix (8 rows x 8 k) is 128 contiguous bytes
  for (int rg = 0; rg < R / 8; ++rg)
    for (int kg = 0; kg < 2; ++kg) {
      int lo = 1 << 30, hi = -1;
      for (int rr = 0; rr < 8; ++rr)
        for (int f4 = 0; f4 < 4; ++f4) {
          const int o = pair_offset(rg * 8 + rr, kg * 4 + f4);
          lo = o < lo ? o : lo;
          hi = o + 4 > hi ? o + 4 : hi;
        }
      if (hi - lo != 128 || lo % 128 != 0) {
        printf("R=%d: core matrix (%d,%d) spans [%d,%d)\n", R, rg, kg, lo, hi);
        return 1;
      }
    }
  return 0;
}

int main() {
  if (check(128) || check(64) || check(16)) return 1;
  printf("ok\n");
  return 0;
}
