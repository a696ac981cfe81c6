// Counter-based random numbers for the sampler's univariate draws.
//
// Sec. 3.4 of the paper gives each core its own seeded generator so parallel
// draws never collide.  On the GPU every draw is instead a pure function of
// (key = seed, counter = (index, sweep, chain, stream)) through Philox4x32-10
// (Salmon, Moraes, Dror & Shaw, SC'11): one call maps a 128-bit counter and a
// 64-bit key to four 32-bit words through ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key advanced by the Weyl increments (W0, W1) between rounds.
// Unit normals follow Box & Muller (1958) on word pairs (w0, w1) and (w2, w3),
// with U = (w + 1/2) 2^-32 so that log U is finite.
#pragma once
#include <cstdint>

namespace mg {

struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return {c0, c1, c2, c3};
}

// Box-Muller in FP64: U exactly (2w + 1) 2^-33.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double ua = (2.0 * double(wa) + 1.0) * 0x1p-33;
  const double ub = (2.0 * double(wb) + 1.0) * 0x1p-33;
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Box-Muller in FP32: (2w + 1) rounded to nearest FP32, then scaled by 2^-33.
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float ua = __ull2float_rn(2ull * wa + 1ull) * 0x1p-33f;
  const float ub = __ull2float_rn(2ull * wb + 1ull) * 0x1p-33f;
  const float r = sqrtf(-2.0f * logf(ua));
  float s, c;
  sincospif(2.0f * ub, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// Stream ids (counter word 3).
constexpr uint32_t kStreamMessenger = 0;
constexpr uint32_t kStreamModes = 1;

}  // namespace mg
