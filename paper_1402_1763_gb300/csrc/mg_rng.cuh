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

#include "mg_rng_tables.h"

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

// FP64 Box-Muller with U exactly (2w + 1) 2^-33.  Both transcendental
// functions are table-driven (tables in mg_rng_tables.h, made in 40-digit
// decimal arithmetic), taking the 33-bit integer v = 2w + 1 as it comes:
//
// ln U = ln v - 33 ln 2 (Tang 1990): v = 2^k m with m in [1, 2); F = 1 + j/128
// the grid point nearest m (j from the 8 bits of m after the leading one),
// f = m - F (exact, |f| <= 1/256), r = f / F, ln m = ln F + ln(1 + r) with
// ln(1 + r) = r - r^2/2 + ... + r^7/7 - r^8/8 (|r| <= 2^-8; the first omitted
// term is below 2^-67 r).  When m rounds to 2 it is halved instead (k + 1,
// F = 1), so U just below 1 is ln(1 + r) alone, without cancellation.  The
// sum (k - 33) ln 2 + ln F + ln(1 + r) is formed with ln 2 and ln F each split
// in two, the high parts on one 2^-44 grid so that their sum is exact.
//
// sin, cos of 2 pi U: U = j/256 + t/(2 pi) with j the top 8 bits of v and
// t = 2 pi (v mod 2^25) 2^-33 in [0, 2 pi/256); sin t and cos t - 1 by their
// Taylor series to t^9 and t^8 (t < 0.0246: the omitted terms are below
// 1e-20), then the angle-addition formulas with the table's sin, cos of
// 2 pi j/256.  Accuracy is a few ulp, far inside the FP64 path's parity with
// the oracle (relative L2 1e-12).
__device__ __forceinline__ double ln_u33(uint32_t w) {
  const unsigned long long v = 2ull * w + 1ull;  // 1 <= v < 2^33
  int k = 63 - __clzll(static_cast<long long>(v));
  const int q = k >= 8 ? int((v >> (k - 8)) & 255ull) : int((v << (8 - k)) & 255ull);
  int j = (q + 1) >> 1;  // nearest grid point, 0 .. 128
  double m = double(v) * __longlong_as_double(static_cast<long long>(1023 - k) << 52);  // exact
  if (j == 128) {
    j = 0;
    k += 1;
    m *= 0.5;
  }
  const double2 tab = __ldg(&kLnTab128[j]);  // {hi(ln F), 1/F}
  const double lo = __ldg(&kLnLo128[j]);      // ln F - hi(ln F)
  const double f = m - (1.0 + double(j) * 0x1p-7);
  const double r = f * tab.y;
  double p = fma(r, -1.0 / 8.0, 1.0 / 7.0);
  p = fma(r, p, -1.0 / 6.0);
  p = fma(r, p, 1.0 / 5.0);
  p = fma(r, p, -1.0 / 4.0);
  p = fma(r, p, 1.0 / 3.0);
  p = fma(r, p, -0.5);
  p = fma(r * r, p, r);  // ln(1 + r)
  const double K = double(k - 33);
  return fma(K, kLn2Hi, tab.x) + (fma(K, kLn2Lo, lo) + p);  // the first sum is exact
}

__device__ __forceinline__ void sincos_2pi_u33(uint32_t w, double& s, double& c) {
  const unsigned long long v = 2ull * w + 1ull;
  const int j = int(v >> 25);  // 0 .. 255
  const double t = double(uint32_t(v & 0x1ffffffull)) * kTwoPi2m33;
  const double t2 = t * t;
  double ps = fma(t2, 1.0 / 362880.0, -1.0 / 5040.0);
  ps = fma(t2, ps, 1.0 / 120.0);
  ps = fma(t2, ps, -1.0 / 6.0);
  const double st = fma(t * t2, ps, t);  // sin t
  double pc = fma(t2, 1.0 / 40320.0, -1.0 / 720.0);
  pc = fma(t2, pc, 1.0 / 24.0);
  pc = fma(t2, pc, -0.5);
  const double cm1 = t2 * pc;  // cos t - 1
  const double2 tab = __ldg(&kSinCos256[j]);  // {sin, cos} of 2 pi j / 256
  s = tab.x + fma(tab.x, cm1, tab.y * st);
  c = tab.y + fma(tab.y, cm1, -(tab.x * st));
}

__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double r = sqrt(-2.0 * ln_u33(wa));
  double s, c;
  sincos_2pi_u33(wb, s, c);
  z0 = r * c;
  z1 = r * s;
}

// The FP32 path's Box-Muller on the special-function unit: U = fma(w, 2^-32,
// 2^-33); -2 ln U from the hardware base-2 logarithm; the angle 2 pi U is
// shifted by pi into (-pi, pi] so the hardware sine and cosine stay in their
// accurate range (|error| <= 2^-21.4 there); since cos(2 pi U - pi) =
// -cos(2 pi U) and sin(2 pi U - pi) = -sin(2 pi U), both products are negated.  The normals agree with the FP64
// construction to a few 1e-6 absolute, except as U_a -> 1, where U's FP32
// rounding (relative 2^-23) moves -2 ln U by up to ~2^-22 and so the radius
// by up to ~2^-22 / (2 r) (at most 5e-4, for radii below 1e-3).
__device__ __forceinline__ float u01_fast(uint32_t w) { return fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f); }

__device__ __forceinline__ float minus2log_fast(uint32_t w) { return -1.3862943611198906f * __log2f(u01_fast(w)); }

// The radius from the special-function unit's square root (relative error
// below 2^-22; exact 0 at U = 1), and the shifted angle 2 pi U - pi =
// 2 pi (w + 1/2) 2^-32 - pi formed from the word in one fused multiply-add.
__device__ __forceinline__ float sqrt_fast(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void box_muller_fast(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float r = sqrt_fast(minus2log_fast(wa));  // -2 ln U >= 0
  float s, c;
  constexpr float kTwoPi = 6.28318530717958647692f;
  __sincosf(fmaf(__uint2float_rn(wb), kTwoPi * 0x1p-32f, kTwoPi * 0x1p-33f - 3.14159265358979323846f), &s, &c);
  z0 = -(r * c);
  z1 = -(r * s);
}

// The same pairs scaled by 1/sqrt(2), the real and imaginary parts of a unit
// complex normal: the radius is sqrt(-ln U) instead of sqrt(-2 ln U), the
// angle unchanged (no separate multiplication of each normal).
__device__ __forceinline__ void box_muller_half(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  const double r = sqrt(-ln_u33(wa));
  double s, c;
  sincos_2pi_u33(wb, s, c);
  z0 = r * c;
  z1 = r * s;
}
__device__ __forceinline__ void box_muller_fast_half(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float r = sqrt_fast(-0.69314718055994531f * __log2f(u01_fast(wa)));  // -ln U >= 0
  float s, c;
  constexpr float kTwoPi = 6.28318530717958647692f;
  __sincosf(fmaf(__uint2float_rn(wb), kTwoPi * 0x1p-32f, kTwoPi * 0x1p-33f - 3.14159265358979323846f), &s, &c);
  z0 = -(r * c);
  z1 = -(r * s);
}

// Precision dispatch: FP64 uses the table-driven construction above, the
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
template <typename T>
__device__ __forceinline__ void half_normal_pair(uint32_t wa, uint32_t wb, T& z0, T& z1);
template <>
__device__ __forceinline__ void half_normal_pair<double>(uint32_t wa, uint32_t wb, double& z0, double& z1) {
  box_muller_half(wa, wb, z0, z1);
}
template <>
__device__ __forceinline__ void half_normal_pair<float>(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  box_muller_fast_half(wa, wb, z0, z1);
}

// -2 ln U of one word: the squared radius of a Box-Muller pair, i.e. the sum
// of the squares of the two normals the pair yields.
template <typename T>
__device__ __forceinline__ T radius2(uint32_t w);
template <>
__device__ __forceinline__ double radius2<double>(uint32_t w) {
  return -2.0 * ln_u33(w);
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
constexpr uint32_t kStreamChi2 = 5;    // the chi-square variate of each shell

// X ~ chi^2_n for the covariance draw of shell b (Alg. 2 on k-shells, drawn
// once per shell), in FP64 in both precision forms.
//   n = 1:  X = z^2, z the first Box-Muller normal of call (b, sweep, chain, 5):
//           Alg. 2's u = G^2 literally.
//   n >= 2: X = 2 Gamma(n/2) by Marsaglia & Tsang (2000, ACM TOMS 26(3)):
//           d = n/2 - 1/3, c = 1/sqrt(9 d); attempt k uses call
//           (b + 256 k, sweep, chain, 5): x = the first normal of words (w0, w1),
//           U = U(w2), v = (1 + c x)^3, accepted when v > 0 and
//           ln U < x^2/2 + d - d v + d ln v, giving X = 2 d v.
// Every product and sum is rounded on its own (no contraction), in the
// order written.  Returns -1 if none of 64 attempts is accepted (probability
// far below 1e-60); the caller then keeps the shell's P.
__device__ inline double chi2_shell(long long n, uint32_t b, uint32_t sweep, uint32_t cid, uint32_t k0,
                                    uint32_t k1) {
  if (n == 1) {
    const u32x4 w = philox4x32_10(b, sweep, cid, kStreamChi2, k0, k1);
    double z0, z1;
    box_muller(w.x, w.y, z0, z1);
    return __dmul_rn(z0, z0);
  }
  const double alpha = 0.5 * double(n);  // exact
  const double d = __dsub_rn(alpha, 1.0 / 3.0);
  const double c = __ddiv_rn(1.0, __dsqrt_rn(__dmul_rn(9.0, d)));
  for (uint32_t k = 0; k < 64; ++k) {
    const u32x4 w = philox4x32_10(b + 256u * k, sweep, cid, kStreamChi2, k0, k1);
    double x, x1;
    box_muller(w.x, w.y, x, x1);
    double v = __dadd_rn(1.0, __dmul_rn(c, x));
    if (!(v > 0.0)) continue;
    v = __dmul_rn(__dmul_rn(v, v), v);
    const double lhs = ln_u33(w.z);
    const double rhs = __dadd_rn(__dsub_rn(__dadd_rn(__dmul_rn(__dmul_rn(0.5, x), x), d), __dmul_rn(d, v)),
                                 __dmul_rn(d, log(v)));
    if (lhs < rhs) return __dmul_rn(__dmul_rn(2.0, d), v);
  }
  return -1.0;
}

}  // namespace mg
