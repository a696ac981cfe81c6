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

// The FP32 path's Box-Muller on the special-function unit: U = fma(w, 2^-32,
// 2^-33); -2 ln U from the hardware base-2 logarithm; the angle 2 pi U is
// shifted by pi into (-pi, pi] so the hardware sine and cosine stay in their
// accurate range (|error| <= 2^-21.4 there).  The normals agree with the FP64
// construction to ~1e-6 absolute.
__device__ __forceinline__ float u01_fast(uint32_t w) { return fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f); }

__device__ __forceinline__ float minus2log_fast(uint32_t w) { return -1.3862943611198906f * __log2f(u01_fast(w)); }

__device__ __forceinline__ void box_muller_fast(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float r2 = minus2log_fast(wa);
  const float r = r2 > 0.f ? r2 * rsqrtf(r2) : 0.f;
  float s, c;
  __sincosf(6.28318530717958647692f * (u01_fast(wb) - 0.5f), &s, &c);
  z0 = -(r * c);
  z1 = -(r * s);
}

// Precision dispatch: FP64 uses the correctly rounded construction above, the
// FP32 path the special-function-unit one.
template <typename T>
__device__ __forceinline__ void normal_pair(uint32_t wa, uint32_t wb, T& z0, T& z1);
template <>
__device__ __forceinline__ void normal_pair<double>(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  box_muller(wa, wb, z0, z1);
}
template <>
__device__ __forceinline__ void normal_pair<float>(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  box_muller_fast(wa, wb, z0, z1);
}

// -2 ln U of one word: the squared radius of a Box-Muller pair, i.e. the sum
// of the squares of the two normals the pair yields.
template <typename T>
__device__ __forceinline__ T radius2(uint32_t w);
template <>
__device__ __forceinline__ double radius2<double>(uint32_t w) {
  return -2.0 * log((2.0 * double(w) + 1.0) * 0x1p-33);
}
template <>
__device__ __forceinline__ float radius2<float>(uint32_t w) {
  return minus2log_fast(w);
}

// Stream ids (counter word 3).
constexpr uint32_t kStreamMessenger = 0;
constexpr uint32_t kStreamModes = 1;
constexpr uint32_t kStreamStart = 2;   // over-dispersed starting powers
constexpr uint32_t kStreamMixing = 4;  // the mixing sweeps' per-shell proposals

}  // namespace mg
