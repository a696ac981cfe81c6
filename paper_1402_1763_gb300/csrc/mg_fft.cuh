// In-register DFT codelets for the hand-written 3D FFT of the messenger sweep.
//
// The orthonormal transform of Sec. 3.1 (Alg. 1, "ONT") is realised as a 3D
// real FFT.  Each 1D line of length N = P*Q is split into two stages of small
// DFTs that live entirely in registers (these codelets), with one shared-memory
// exchange between the stages and an inter-stage twiddle read from a table.
// Codelet sizes: 1, 2, 3, 4 directly, 6/8/12/16 as two-factor compositions.
// All internal twiddles are roots of unity of order dividing 48 and are folded
// in at compile time.
#pragma once
#include <cstdint>

namespace mg {

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename T>
__device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
// multiply by +i (S = +1) or -i (S = -1)
template <int S, typename T>
__device__ __forceinline__ cx<T> cmul_i(cx<T> a) {
  if constexpr (S > 0) return {-a.im, a.re};
  else return {a.im, -a.re};
}

// FP32 complex adds and subtracts as one packed two-lane instruction (the
// FADD2 / FFMA2 forms of sm_100 and later): a value's real and imaginary parts
// are one register pair, so a butterfly's add costs one instruction instead
// of two.  Each lane rounds exactly as the scalar operation does.
__device__ __forceinline__ float2 pk(cx<float> a) { return make_float2(a.re, a.im); }
__device__ __forceinline__ cx<float> unpk(float2 v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 psub2(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rr;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rr, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rr;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ cx<float> cadd(cx<float> a, cx<float> b) { return unpk(__fadd2_rn(pk(a), pk(b))); }
__device__ __forceinline__ cx<float> csub(cx<float> a, cx<float> b) { return unpk(psub2(pk(a), pk(b))); }
// d + s * (t.im, t.re): the +-i t terms of the radix-2^k butterflies, one FFMA2
__device__ __forceinline__ cx<float> cfma_swap(cx<float> t, float2 s, cx<float> d) {
  return unpk(__ffma2_rn(make_float2(t.im, t.re), s, pk(d)));
}

// cos and sin of 2*pi*i/48 for i = 0..12 (first quadrant, 25 digits).
__host__ __device__ constexpr double kCos48q(int i) {
  return i == 0 ? 1.0 : i == 1 ? 0.9914448613738104111445575 : i == 2 ? 0.9659258262890682867497432
       : i == 3 ? 0.9238795325112867561281832 : i == 4 ? 0.8660254037844386467637232
       : i == 5 ? 0.7933533402912351645797770 : i == 6 ? 0.7071067811865475244008444
       : i == 7 ? 0.6087614290087206394160975 : i == 8 ? 0.5
       : i == 9 ? 0.3826834323650897717284600 : i == 10 ? 0.2588190451025207623488988
       : i == 11 ? 0.1305261922200515915484062 : 0.0;
}
// cos(2 pi i / 48) and sin(2 pi i / 48) for any integer i (reduced mod 48).
__host__ __device__ constexpr double kCos48(int i) {
  i = ((i % 48) + 48) % 48;
  return i <= 12 ? kCos48q(i) : i <= 24 ? -kCos48q(24 - i) : i <= 36 ? -kCos48q(i - 24) : kCos48q(48 - i);
}
__host__ __device__ constexpr double kSin48(int i) { return kCos48(i - 12); }

// v * exp(DIR * 2 pi i * E / R): the compile-time twiddle of a composite codelet.
// DIR = -1 for the forward transform, +1 for the inverse.
template <int R, int DIR, int E, typename T>
__device__ __forceinline__ cx<T> twiddle_c(cx<T> v) {
  static_assert(48 % R == 0, "codelet order must divide 48");
  constexpr int i = (((DIR * E * (48 / R)) % 48) + 48) % 48;
  if constexpr (i == 0) return v;
  else if constexpr (i == 12) return cmul_i<+1>(v);
  else if constexpr (i == 24) return {-v.re, -v.im};
  else if constexpr (i == 36) return cmul_i<-1>(v);
  else {
    constexpr double c = kCos48(i), s = kSin48(i);
    return cmul(v, cx<T>{T(c), T(s)});
  }
}

template <int R, int DIR, typename T>
struct Dft;

template <int DIR, typename T>
struct Dft<1, DIR, T> {
  static __device__ __forceinline__ void run(cx<T>*) {}
};

template <int DIR, typename T>
struct Dft<2, DIR, T> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR, typename T>
struct Dft<3, DIR, T> {
  // X1 = a0 - (a1+a2)/2 + DIR*i*(sqrt3/2)*(a1-a2), X2 = the conjugate-sign partner.
  static __device__ __forceinline__ void run(cx<T>* v) {
    constexpr T h = T(0.8660254037844386467637232);
    cx<T> s = cadd(v[1], v[2]);
    cx<T> d = csub(v[1], v[2]);
    cx<T> m = {v[0].re - T(0.5) * s.re, v[0].im - T(0.5) * s.im};
    cx<T> r = cmul_i<DIR>(cscale(d, h));
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <int DIR, typename T>
struct Dft<4, DIR, T> {
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    cx<T> s13 = cadd(v[1], v[3]), d13 = cmul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

// FP32 radix 3 and 4 on packed pairs: the same arithmetic lane by lane, with
// the +-i factors folded into one FFMA2 of the swapped difference.
template <int DIR>
struct Dft<3, DIR, float> {
  static __device__ __forceinline__ void run(cx<float>* v) {
    constexpr float h = 0.8660254037844386467637232f;
    const cx<float> s = cadd(v[1], v[2]);
    const cx<float> d = csub(v[1], v[2]);
    const cx<float> m = unpk(__ffma2_rn(pk(s), make_float2(-0.5f, -0.5f), pk(v[0])));
    v[0] = cadd(v[0], s);
    // r = DIR i h d = DIR h (-d.im, d.re); v1 = m + r, v2 = m - r
    v[1] = cfma_swap(d, make_float2(-DIR * h, DIR * h), m);
    v[2] = cfma_swap(d, make_float2(DIR * h, -DIR * h), m);
  }
};

template <int DIR>
struct Dft<4, DIR, float> {
  static __device__ __forceinline__ void run(cx<float>* v) {
    const cx<float> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const cx<float> s13 = cadd(v[1], v[3]), t = csub(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    // d13 = DIR i t = DIR (-t.im, t.re); v1 = d02 + d13, v3 = d02 - d13
    v[1] = cfma_swap(t, make_float2(-float(DIR), float(DIR)), d02);
    v[3] = cfma_swap(t, make_float2(float(DIR), -float(DIR)), d02);
  }
};

// Two-factor composition R = R1 * R2, natural order in and out:
//   X[c + R1 d] = sum_b W_R2^{bd} W_R^{bc} sum_a W_R1^{ac} x[R2 a + b].
template <int R1, int R2, int DIR, typename T>
struct DftComp {
  static constexpr int R = R1 * R2;
  template <int B, int C>
  static __device__ __forceinline__ void tw(cx<T>* y) {
    y[B * R1 + C] = twiddle_c<R, DIR, B * C>(y[B * R1 + C]);
    if constexpr (C + 1 < R1) tw<B, C + 1>(y);
    else if constexpr (B + 1 < R2) tw<B + 1, 0>(y);
  }
  static __device__ __forceinline__ void run(cx<T>* v) {
    cx<T> y[R];
#pragma unroll
    for (int b = 0; b < R2; ++b) {
      cx<T> a[R1];
#pragma unroll
      for (int i = 0; i < R1; ++i) a[i] = v[R2 * i + b];
      Dft<R1, DIR, T>::run(a);
#pragma unroll
      for (int c = 0; c < R1; ++c) y[b * R1 + c] = a[c];
    }
    tw<0, 0>(y);
#pragma unroll
    for (int c = 0; c < R1; ++c) {
      cx<T> a[R2];
#pragma unroll
      for (int b = 0; b < R2; ++b) a[b] = y[b * R1 + c];
      Dft<R2, DIR, T>::run(a);
#pragma unroll
      for (int d = 0; d < R2; ++d) v[c + R1 * d] = a[d];
    }
  }
};

template <int DIR, typename T>
struct Dft<6, DIR, T> : DftComp<2, 3, DIR, T> {};
template <int DIR, typename T>
struct Dft<8, DIR, T> : DftComp<2, 4, DIR, T> {};
template <int DIR, typename T>
struct Dft<12, DIR, T> : DftComp<4, 3, DIR, T> {};
template <int DIR, typename T>
struct Dft<16, DIR, T> : DftComp<4, 4, DIR, T> {};

// Two-stage split N = P * Q of every supported line length (P, Q <= 16).
// Lines along x and y have length n, rows along z are half-length complex
// transforms of length n/2 (real-to-complex packing).
template <int N>
struct Split;
#define MG_SPLIT(N_, P_, Q_)              \
  template <>                             \
  struct Split<N_> {                      \
    static constexpr int P = P_, Q = Q_; \
  };
MG_SPLIT(4, 2, 2)
MG_SPLIT(6, 2, 3)
MG_SPLIT(8, 4, 2)
MG_SPLIT(12, 4, 3)
MG_SPLIT(16, 4, 4)
MG_SPLIT(24, 8, 3)
MG_SPLIT(32, 8, 4)
MG_SPLIT(48, 12, 4)
MG_SPLIT(64, 8, 8)
MG_SPLIT(96, 12, 8)
MG_SPLIT(128, 16, 8)
MG_SPLIT(192, 16, 12)
MG_SPLIT(256, 16, 16)
#undef MG_SPLIT

}  // namespace mg
