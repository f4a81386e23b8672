// Device-side Philox4x32-10 counter-based generator (Salmon et al., SC'11),
// used for the random start permutations and tabu tenures of each walk.
#pragma once
#include <cstdint>

namespace qapk {

struct Philox4 {
  uint32_t v[4];
};

// Ten rounds of the Philox 4x32 bijection.  Round: with the 32x32->64
// products M0*x0 and M1*x2 split into (hi, lo) halves, the new word vector
// is (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0)); the
// key is bumped by the Weyl constants between rounds.
__device__ __forceinline__ Philox4 philox4x32_10(uint32_t x0, uint32_t x1, uint32_t x2,
                                                uint32_t x3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t hiA = __umulhi(kM0, x0), loA = kM0 * x0;
    const uint32_t hiB = __umulhi(kM1, x2), loB = kM1 * x2;
    const uint32_t y0 = hiB ^ x1 ^ k0;
    const uint32_t y2 = hiA ^ x3 ^ k1;
    x0 = y0;
    x1 = loB;
    x2 = y2;
    x3 = loA;
    k0 += kW0;
    k1 += kW1;
  }
  return Philox4{{x0, x1, x2, x3}};
}

// Draw `idx` of stream `stream` for walk id `wid`: counter block idx/4,
// word idx%4.
__device__ __forceinline__ uint32_t walk_draw(uint64_t seed, uint32_t wid, uint32_t stream,
                                              uint32_t idx) {
  const Philox4 b = philox4x32_10(wid, stream, idx >> 2, 0u, (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
  const uint32_t q = idx & 3u;
  return q == 0 ? b.v[0] : q == 1 ? b.v[1] : q == 2 ? b.v[2] : b.v[3];
}

// Uniform value in [0, m): high word of the 64-bit product x * m.
__device__ __forceinline__ uint32_t below(uint32_t x, uint32_t m) { return __umulhi(x, m); }

}  // namespace qapk
