// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), shared by the field kernels.
#pragma once
#include <stdint.h>

namespace mlmc {

// Ten rounds of the two-multiplier S-box on the counter (c0..c3) with the Weyl key schedule.
__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                         uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t t0 = hi1 ^ c1 ^ k0, t2 = hi0 ^ c3 ^ k1;
    c0 = t0;
    c1 = lo1;
    c2 = t2;
    c3 = lo0;
  }
}

}  // namespace mlmc
