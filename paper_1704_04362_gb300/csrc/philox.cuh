// Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel Random Numbers: As
// Easy as 1, 2, 3", SC'11), the counter-based generator behind every random
// draw of the library: the Bernoulli coins and with-replacement draws of the
// sampled t-product (Algorithm 2), the slice picks of t-CX / t-CUR
// (Algorithms 4-5) and the test matrix of the randomized t-SVD.  A 128-bit
// counter and a 64-bit key pass through ten rounds; each round multiplies
// words 0 and 2 by fixed 32-bit constants, keeps both halves of the products,
// XORs the high halves with the other two words and the round key, and
// permutes; the key advances by two Weyl constants between rounds.
#pragma once

#include <stdint.h>

namespace tp {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t y0 = hi1 ^ c[1] ^ k0, y2 = hi0 ^ c[3] ^ k1;
    c[0] = y0; c[1] = lo1; c[2] = y2; c[3] = lo0;
  }
}

}  // namespace tp
