// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw, SC'11),
// written from its published round function: two 32x32-bit multiplies per round, a Weyl
// key schedule, ten rounds.  A draw's random words depend only on its counter and key.
#pragma once
#include <cstdint>

namespace mbis {

struct Philox4 {
  uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                 uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox4 o = {{c0, c1, c2, c3}};
  return o;
}

}  // namespace mbis
