// Pass X of the two-pass sweep: forward x-FFT, the signal draw per mode,
// the k-shell sums, and the inverse x-FFT, on tiles of 32 x-pencils.
//
//   * signal draw (Sec. 3.1, Alg. 1 second loop): s_hat = mu + sigma xi with
//     mu = S/(S + T) t_hat and sigma^2 = S T/(S + T), T = tau for the unitary
//     transform; S_hat = (M/V) P(shell) and 0 at k = 0.
//   * shell sums for the covariance draw (Sec. 3.2, Alg. 2 on shells):
//     sigma_b = sum w |s_hat|^2 (the chi-square variate X_b is drawn once per
//     shell by the shell draw).
//
// A CTA owns 32 consecutive pencils (lanes) and all n values of x.  The FFT of
// length n = P*Q runs as: stage F1 (DFT_Q per p, from global), exchange through
// shared memory, stage F2 (DFT_P per v) -> modes kx = Q u + v in registers ->
// draw -> inverse stage I1 (IDFT_P) back into the same shared slots -> stage
// I2 (IDFT_Q per p) -> global.  Warp lanes are pencils at the same kx, so the
// shell ids along a warp come in runs, reduced with a segmented warp scan.
#pragma once
#include "mg_device.cuh"
#include "mg_launch.h"

namespace mg {

// Shell accumulators per warp: FP32 keeps an error-free (hi, lo) FP32 pair per
// value (TwoSum), FP64 a plain double; both are combined in FP64 per tile.
// kWords: the words of the two-value form (adjoint and mixing sweeps); the
// plain sweep sums one value and uses the first half of each shell's words.
template <typename T>
struct Acc;
template <>
struct Acc<float> {
  static constexpr int kWordsPerValue = 2;
  static constexpr int kWords = 4;  // hi1, lo1, hi2, lo2
  static __device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    const float e = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += e;
  }
  static __device__ __forceinline__ void add(float* a, float x1, float x2) {
    float h1 = a[0], l1 = a[1], h2 = a[2], l2 = a[3];
    two_sum(h1, l1, x1);
    two_sum(h2, l2, x2);
    a[0] = h1;
    a[1] = l1;
    a[2] = h2;
    a[3] = l2;
  }
  static __device__ __forceinline__ void add1(float* a, float x1) {
    float h1 = a[0], l1 = a[1];
    two_sum(h1, l1, x1);
    a[0] = h1;
    a[1] = l1;
  }
};
template <>
struct Acc<double> {
  static constexpr int kWordsPerValue = 1;
  static constexpr int kWords = 2;
  static __device__ __forceinline__ void add(double* a, double x1, double x2) {
    a[0] += x1;
    a[1] += x2;
  }
  static __device__ __forceinline__ void add1(double* a, double x1) { a[0] += x1; }
};

// Segmented warp reduction of NV values (v1, and v2 if NV == 2) over runs of
// equal shell id, then the head of each run adds the run's sums to this warp's
// accumulators (kWordsPerValue * NV words per shell).  bin < 0 marks lanes
// that contribute nothing.  When the shell ids do not decrease along the warp
// (always the case for pencils of consecutive kz at one (kx, ky)) the run
// heads hold distinct shells and update in parallel; otherwise they update
// one after another in lane order.  Both orders are fixed, so the sums are
// deterministic.
template <typename T, int NV = 2>
__device__ __forceinline__ void shell_accumulate(T v1, T v2, int bin, T* accw, int lane) {
  constexpr int kW = Acc<T>::kWordsPerValue * NV;
  const unsigned full = 0xffffffffu;
  const int prevb = __shfl_up_sync(full, bin, 1);
  const bool head = (lane == 0) || (prevb != bin);
  const unsigned heads = __ballot_sync(full, head);
  const bool monotone = __all_sync(full, lane == 0 || prevb <= bin);
  const unsigned later = (lane == 31) ? 0u : (heads & (full << (lane + 1)));
  const int run_end = later ? (__ffs(later) - 2) : 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const T o1 = __shfl_down_sync(full, v1, off);
    T o2 = T(0);
    if constexpr (NV == 2) o2 = __shfl_down_sync(full, v2, off);
    if (lane + off <= run_end) {
      v1 += o1;
      if constexpr (NV == 2) v2 += o2;
    }
  }
  auto add = [&]() {
    if constexpr (NV == 2) Acc<T>::add(accw + bin * kW, v1, v2);
    else Acc<T>::add1(accw + bin * kW, v1);
  };
  const bool writer = head && bin >= 0;
  if (monotone) {
    if (writer) add();
  } else {
    unsigned hm = __ballot_sync(full, writer);
    while (hm) {
      const int src = __ffs(hm) - 1;
      if (lane == src) add();
      __syncwarp();
      hm &= hm - 1;
    }
  }
}

// Shell id of stored mode (kx, ky, kz) and its coefficients (a/M, sd/sqrt(M));
// the DC mode gets id -1 and the zero coefficients of entry B+1.  The id
// depends on |m|^2 only, so the modes kx and n - kx share it.
template <typename T, int N>
__device__ __forceinline__ int mode_bin(int kx, int ky, int kz, const ChainDev<T>& cd) {
  constexpr int H = N / 2;
  const int mx = kx <= H ? kx : kx - N;
  const int my = ky <= H ? ky : ky - N;
  const int m2 = mx * mx + my * my + kz * kz;
  int b = m2 == 0 ? -1 : int(__ldg(cd.bin_of_m2 + m2));
#ifdef MG_CHECKED
  // shell ids come from a host table; the per-warp sums and the coefficients
  // hold B + 1 shells
  if (b > cd.B) {
    flag_bounds(cd.status);
    b = -1;  // contributes nothing, coefficients of the DC entry
  }
#endif
  return b;
}
template <typename T, int N>
__device__ __forceinline__ int mode_shell(int kx, int ky, int kz, const ChainDev<T>& cd, cx<T>& cf) {
  const int bin = mode_bin<T, N>(kx, ky, kz, cd);
  cf = ldc<T>(cd.coef + (bin < 0 ? cd.B + 1 : bin));
  return bin;
}

// Philox call (stream 1) shared by the stored modes kx' and n - kx' at
// (ky, kz), kx' <= n/2: the stored index of (kx', ky, kz).  Mode kx' takes the
// normals of words (w0, w1), mode n - kx' those of words (w2, w3).
template <int N>
__device__ __forceinline__ uint32_t pair_call(int kxp, int ky, int kz) {
  return uint32_t((kxp * N + ky) * (N / 2 + 1) + kz);
}

// The complex unit noise xi of one stored mode (kx, ky, kz) (Sec. 3.1, the
// signal draw's G for a complex mode): (z0 + i z1)/sqrt(2) from its own word
// pair of the call it shares with n - kx.  On the kz = 0 and n/2 planes both
// k and -k are stored: of each pair the member with the smaller ky n + kx is
// canonical and draws its own noise, the other takes the conjugate of it,
// and a self-conjugate mode is real, xi = z0.  Canonical modes lie in rows
// ky <= n - ky, so a row ky > n/2 takes every draw from the call of row
// n - ky: mode kx there is the conjugate of mode n - kx of that row, i.e. of
// the other word pair (the same one when kx is 0 or n/2).
template <typename T, int N>
__device__ __forceinline__ cx<T> mode_xi(int kx, int ky, int kz, uint32_t sweep, uint32_t k0, uint32_t k1,
                                         uint32_t cid) {
  constexpr int H = N / 2;
  const bool a_lo = kx <= H;
  const int lo = a_lo ? kx : N - kx;
  const bool selfx = lo == 0 || lo == H;  // kx = n - kx (mod n)
  const bool edge = kz == 0 || kz == H;
  const int py = (N - ky) % N;
  const bool flip = edge && py < ky;         // conjugate of row py's draw
  const bool ypair = edge && py == ky;       // kx and n - kx are each other's partners
  const bool use_hi = flip ? (a_lo && !selfx) : (!ypair && !a_lo);
  const bool conj = flip || (ypair && !a_lo);
  const u32x4 w = philox4x32_10(pair_call<N>(lo, flip ? py : ky, kz), sweep, cid, kStreamModes, k0, k1);
  T z0, z1;  // the normals / sqrt(2)
  half_normal_pair<T>(use_hi ? w.z : w.x, use_hi ? w.w : w.y, z0, z1);
  if (ypair && selfx) return {z0 * T(1.41421356237309504880), T(0)};
  return {z0, conj ? -z1 : z1};
}

// The noise of the two stored modes kx and n - kx at (ky, kz) (the same mode
// twice if kx is 0 or n/2), as mode_xi gives it, from one Philox call: words
// (w0, w1) for the member with kx <= n/2 and (w2, w3) for the other, of the
// row's own call, or on the kz = 0 and n/2 planes for rows ky > n/2 the
// conjugates of the crossed pairs of row n - ky's call.
template <typename T, int N>
__device__ __forceinline__ void xi_pair(int kx, int ky, int kz, uint32_t sweep, uint32_t k0, uint32_t k1,
                                        uint32_t cid, cx<T>& xa, cx<T>& xb) {
  constexpr int H = N / 2;
  const bool a_lo = kx <= H;
  const int lo = a_lo ? kx : N - kx;
  const bool selfx = lo == 0 || lo == H;
  const bool edge = kz == 0 || kz == H;
  const int py = (N - ky) % N;
  const bool flip = edge && py < ky;
  const u32x4 w = philox4x32_10(pair_call<N>(lo, flip ? py : ky, kz), sweep, cid, kStreamModes, k0, k1);
  T z0, z1, z2, z3;  // the normals / sqrt(2)
  half_normal_pair<T>(w.x, w.y, z0, z1);
  half_normal_pair<T>(w.z, w.w, z2, z3);
  cx<T> xl = {z0, z1}, xh = {z2, z3};
  if (edge) {
    if (flip) {
      const cx<T> l = xl;
      xl = selfx ? cconj(l) : cconj(xh);
      xh = selfx ? xl : cconj(l);
    } else if (py == ky) {
      xl = selfx ? cx<T>{z0 * T(1.41421356237309504880), T(0)} : xl;
      xh = selfx ? xl : cconj(xl);
    }
  }
  xa = a_lo ? xl : xh;
  xb = a_lo ? xh : xl;
}

// The signal draw of one stored mode with its noise xi and its shell's
// coefficients cf = (a/M, sd/sqrt(M)): F is the unnormalised forward DFT of
// t, i.e. sqrt(M) t_hat, and the result is s_hat / sqrt(M), the value the
// unnormalised inverse transforms turn into s.  Reports w |s_hat|^2 / M (the
// shell draw multiplies the sums by M), w the mode's dof weight.
template <typename T>
__device__ __forceinline__ cx<T> signal_draw(cx<T> F, cx<T> cf, cx<T> xi, T wgt, T& sig) {
  const cx<T> s = {cf.re * F.re + cf.im * xi.re, cf.re * F.im + cf.im * xi.im};
  sig = wgt * (s.re * s.re + s.im * s.im);
  return s;
}

// The signal draw of one stored mode, with its shell id (or -1: DC or a
// padding lane, which then contribute nothing to the shell sums).
template <typename T, int N>
__device__ __forceinline__ cx<T> draw_mode(cx<T> F, int kx, int ky, int kz, bool valid,
                                           const ChainDev<T>& cd, uint32_t sweep, uint32_t k0, uint32_t k1,
                                           uint32_t cid, int& bin, T& sig) {
  constexpr int H = N / 2;
  cx<T> cf;
  bin = mode_shell<T, N>(kx, ky, kz, cd, cf);
  const cx<T> xi = mode_xi<T, N>(kx, ky, kz, sweep, k0, k1, cid);
  const cx<T> s = signal_draw<T>(F, cf, xi, (kz == 0 || kz == H) ? T(1) : T(2), sig);
  if (!valid || bin < 0) {
    bin = -1;
    sig = T(0);
  }
  return s;
}

template <typename T, int N, int MODE>
__device__ __forceinline__ cx<T> adjoint_mode(cx<T> G, cx<T> Ft, int kx, int ky, int kz, bool valid,
                                              const ChainDev<T>& cd, uint32_t sweep, uint32_t k0, uint32_t k1,
                                              uint32_t cid, int& bin, T& grad, T& loss);

// Adjoint of the signal draw of one mode (fixed P).  In mode kXAdjTop, G is
// the unnormalised x transform of the final state, i.e. n s_hat / sqrt(M); the
// loss term is w_l |s_hat|^2 and the adjoint seed G = sqrt(M) mu with
// mu = 2 w_l s_hat / w.  In kXAdjMid, G = sqrt(M) mu comes from the adjoint y/z
// pass.  Ft is the unnormalised transform of the forward messenger field t.
// With the shell's (a/M, sd/sqrt(M)) the gradient of log P_b gets
// w (1 - a) Re(conj G (a/M Ft + sd/(2 sqrt M) xi)), and the value returned,
// (a/M) G = a mu / sqrt(M), feeds the inverse transforms.
template <typename T, int N, int MODE>
__device__ __forceinline__ cx<T> adjoint_mode(cx<T> G, cx<T> Ft, int kx, int ky, int kz, bool valid,
                                              const ChainDev<T>& cd, uint32_t sweep, uint32_t k0, uint32_t k1,
                                              uint32_t cid, int& bin, T& grad, T& loss) {
  constexpr int H = N / 2;
  const int mx = kx <= H ? kx : kx - N;
  const int my = ky <= H ? ky : ky - N;
  const int m2 = mx * mx + my * my + kz * kz;
  const bool edge = (kz == 0) || (kz == H);
  const T wd = edge ? T(1) : T(2);
  bool dc = (m2 == 0);
  bin = dc ? -1 : int(__ldg(cd.bin_of_m2 + m2));
#ifdef MG_CHECKED
  if (bin > cd.B) {  // shell ids come from a host table (see mode_bin)
    flag_bounds(cd.status);
    bin = -1;
    dc = true;
  }
#endif
  const cx<T> cf = ldc<T>(cd.coef + (dc ? cd.B + 1 : bin));
  loss = T(0);
  if constexpr (MODE == kXAdjTop) {
    const size_t j = size_t(kx * N + ky) * (H + 1) + kz;
    const T wl = valid ? cd.wloss[j] : T(0);
    const T M = T(double(N) * double(N) * double(N));
    loss = wl * (M / (T(N) * T(N))) * (G.re * G.re + G.im * G.im);
    const T sc = T(2) * wl * (M / T(N)) / wd;
    G = {G.re * sc, G.im * sc};
  }
  const cx<T> xi = mode_xi<T, N>(kx, ky, kz, sweep, k0, k1, cid);
  const T am = cf.re;  // a / M
  const T a_ = am * T(double(N) * double(N) * double(N));
  const cx<T> u = {am * Ft.re + T(0.5) * cf.im * xi.re, am * Ft.im + T(0.5) * cf.im * xi.im};
  grad = wd * (T(1) - a_) * (G.re * u.re + G.im * u.im);
  if (!valid || dc) {
    bin = -1;
    grad = T(0);
    loss = T(0);
  }
  return {am * G.re, am * G.im};
}

template <typename T, int N>
struct PassXShape {
  static constexpr int H = N / 2;
  static constexpr int P = Split<N>::P, Q = Split<N>::Q;
  static constexpr int LW = 32;
  static constexpr int kMainTiles = (N * H + LW - 1) / LW;
  static constexpr int kNyqTiles = (N + LW - 1) / LW;
  static constexpr int kTiles = kMainTiles + kNyqTiles;
  static constexpr size_t kXchgBytes = size_t(N) * LW * sizeof(typename VT<T>::c2);
  static size_t smem_bytes(int nwarps, int B, bool dual = false) {
    return (dual ? 2 : 1) * kXchgBytes + size_t(nwarps) * (B + 1) * Acc<T>::kWords * sizeof(T);
  }
};

// One tile of 32 pencils of one chain (`block` = chain * tiles + tile).
// Called by pass_x_kernel and by the persistent sweep kernel.
template <typename T, int N, int NT, int MODE = kXSweep>
__device__ __forceinline__ void pass_x_tile(const LaunchArgs<T>& a, int block, unsigned char* smem_raw) {
  using S = PassXShape<T, N>;
  using V2 = typename VT<T>::c2;
  using TL = TwLayout<N>;
  constexpr int H = S::H, P = S::P, Q = S::Q, LW = S::LW;
  constexpr int NW = NT / 32;
  constexpr bool kAdj = MODE == kXAdjTop || MODE == kXAdjMid;
  constexpr bool kMixDraw = MODE == kXMixDraw, kMixScale = MODE == kXMixScale;
  constexpr int kNV = (kAdj || kMixDraw) ? 2 : 1;  // values the shell sums carry
  static_assert(NT % 32 == 0, "whole warps");
  V2* xs = reinterpret_cast<V2*>(smem_raw);  // [N][LW], slot p*Q + v
  V2* xs2 = reinterpret_cast<V2*>(smem_raw + S::kXchgBytes);  // adjoint: second input
  T* acc = reinterpret_cast<T*>(smem_raw + (kAdj ? 2 : 1) * S::kXchgBytes);

  const int tile = block % S::kTiles;
  const int chain = block / S::kTiles;
  const ChainDev<T> cd = a.chains[chain];
  const uint32_t k0 = a.k0[chain], k1 = a.k1[chain], cid = a.cid[chain];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B1 = cd.B + 1;
  const uint32_t sweep = *a.sweep_ctr;

  for (int i = threadIdx.x; i < NW * B1 * Acc<T>::kWords; i += NT) acc[i] = T(0);

  const bool nyq_tile = tile >= S::kMainTiles;
  int ky, kz;
  bool valid;
  size_t off;  // element offset of this lane's pencil at x = 0
  size_t stride;
  if (!nyq_tile) {
    const int f = tile * LW + lane;
    valid = f < N * H;
    ky = valid ? f / H : 0;
    kz = valid ? f % H : 0;
    off = valid ? f : 0;
    stride = size_t(N) * H;
  } else {
    ky = (tile - S::kMainTiles) * LW + lane;
    valid = ky < N;
    if (!valid) ky = 0;
    kz = H;
    off = ky;
    stride = N;
  }
  V2* base = (nyq_tile ? cd.nyq : cd.main) + off;
  const V2* base_in = base;
  const V2* base2 = nullptr;
  if constexpr (kAdj) {
    base_in = (nyq_tile ? cd.nyq_in : cd.main_in) + off;
    base2 = (nyq_tile ? cd.nyq2 : cd.main2) + off;
  }

  // Prefetch into L2 the pencils of the tile pf_units ahead in launch order
  // (CTAs start in launch order as earlier ones finish, so it starts soon),
  // so its first loads hit L2 rather than HBM.  Main tiles only; lines that
  // start past the last pencil are skipped.
  if constexpr (!kAdj) {
    const int nb = block + a.pf_units;
    if (a.pf_units > 0 && nb < S::kTiles * a.n_chains && nb % S::kTiles < S::kMainTiles) {
      const int f0 = (nb % S::kTiles) * LW;
      const V2* nbase = a.chains[nb / S::kTiles].main + f0;
      constexpr int kPerLine = 128 / int(sizeof(V2));
      constexpr int kLines = (LW + kPerLine - 1) / kPerLine;
      for (int i = threadIdx.x; i < N * kLines; i += NT) {
        const int kx = i / kLines, ln = i % kLines;
        if (f0 + ln * kPerLine < N * H) {
          const V2* pa = nbase + size_t(kx) * N * H + ln * kPerLine;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pa));
        }
      }
    }
  }

  // Mixing sweep, second half: the modes (kx = slot index) come back from k
  // space; the column loop below scales them and runs the inverse stage I1.
  if constexpr (kMixScale) {
    for (int kx = warp; kx < N; kx += NW)
      stc<T>(xs + kx * LW + lane, valid ? ldcg<T>(base + size_t(kx) * stride) : cx<T>{T(0), T(0)});
  }

  // Stage F1: DFT_Q over q of x[p + P q], twiddle W_N^{p v}, to slot p*Q + v.
  for (int it = threadIdx.x; it < (kMixScale ? 0 : LW * P); it += NT) {
    const int p = it / LW;
    cx<T> w[Q];
    ld_tw_row<T, Q>(a.tw + TL::kCpv + p * Q, w);
#pragma unroll
    for (int inp = 0; inp < (kAdj ? 2 : 1); ++inp) {
      const V2* src = inp == 0 ? base_in : base2;
      V2* dst = inp == 0 ? xs : xs2;
      cx<T> v[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) v[q] = valid ? ldcg<T>(src + size_t(p + P * q) * stride) : cx<T>{T(0), T(0)};
      Dft<Q, -1, T>::run(v);
#pragma unroll
      for (int vq = 0; vq < Q; ++vq) stc<T>(dst + (p * Q + vq) * LW + lane, vq == 0 ? v[vq] : cmul(v[vq], w[vq]));
    }
  }
  __syncthreads();

  // Stage F2 + draw + inverse stage I1, in place in the slots of column v.
  // The modes kx = Q u + v pass through their shared-memory slots u*Q + v so
  // that the draw runs as one compact (not unrolled) loop over u.
  T* accw = acc + warp * B1 * Acc<T>::kWords;
  // Sweep tiles with an even Q and enough column pairs for every thread take
  // the columns {v, Q-v} (item 0: {0, Q/2}) together: mode kx = Q u + v and
  // mode n - kx = Q (P-1-u) + (Q-v) (or, in columns 0 and Q/2, the partner in
  // the same column) are both in the thread, share one shell, and enter the
  // shell sums as one term.
  // Plain sweeps sum the signal power w |s_hat|^2 alone (the chi-square
  // variate is drawn per shell by the shell draw); mixing draws accumulate
  // (w |y|^2, w Re(conj(y) F)) and leave the modes in k space.
  constexpr bool kPair = !kAdj && !kMixScale && Q % 2 == 0 && (LW * (Q / 2)) % NT == 0;
  if constexpr (kMixScale) {
    // s_hat_new / sqrt(M) = y sqrt(S_new / S_old) per shell, then I1.
    for (int it = threadIdx.x; it < LW * Q; it += NT) {
      const int vq = it / LW;
      cx<T> X[P];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int bin = mode_bin<T, N>(Q * p + vq, ky, kz, cd);
        const T r = cd.mscale[bin < 0 ? cd.B + 1 : bin];
        X[p] = cscale(ldc<T>(xs + (p * Q + vq) * LW + lane), r);
      }
      Dft<P, +1, T>::run(X);
      cx<T> w[P];
      ld_tw_row<T, P>(a.tw + TL::kCvp + vq * P, w);
#pragma unroll
      for (int p = 0; p < P; ++p) stc<T>(xs + (p * Q + vq) * LW + lane, p == 0 ? X[p] : cmulc(X[p], w[p]));
    }
  } else if constexpr (kPair) {
    auto f2_col = [&](int vq) {
      cx<T> X[P];
#pragma unroll
      for (int p = 0; p < P; ++p) X[p] = ldc<T>(xs + (p * Q + vq) * LW + lane);
      Dft<P, -1, T>::run(X);
#pragma unroll
      for (int u = 0; u < P; ++u) stc<T>(xs + (u * Q + vq) * LW + lane, X[u]);
    };
    auto i1_col = [&](int vq) {
      cx<T> X[P];
#pragma unroll
      for (int p = 0; p < P; ++p) X[p] = ldc<T>(xs + (p * Q + vq) * LW + lane);
      Dft<P, +1, T>::run(X);
      cx<T> w[P];
      ld_tw_row<T, P>(a.tw + TL::kCvp + vq * P, w);
#pragma unroll
      for (int p = 0; p < P; ++p) stc<T>(xs + (p * Q + vq) * LW + lane, p == 0 ? X[p] : cmulc(X[p], w[p]));
    };
    for (int it = threadIdx.x; it < LW * (Q / 2); it += NT) {
      const int g = it / LW;  // the same for the whole warp
      const int va = g, vb = g == 0 ? Q / 2 : Q - g;
      f2_col(va);
      f2_col(vb);
      // g > 0: P pairs (u, P-1-u) across the two columns.  g == 0: the
      // self-paired modes kx = 0 and n/2 alone, then the pairs (u, P-u) of
      // column 0 and (u, P-1-u) of column Q/2.
      const int steps = g == 0 ? P + 1 : P;
#pragma unroll 1
      for (int t = 0; t < steps; ++t) {
        int ua, ca, ub, cb;
        bool two = true;
        if (g != 0) {
          ua = t;
          ca = va;
          ub = P - 1 - t;
          cb = vb;
        } else if (t < 2) {
          ua = t * (P / 2);
          ca = 0;
          ub = ua;
          cb = 0;
          two = false;
        } else if (t < P / 2 + 1) {
          ua = t - 1;
          ca = 0;
          ub = P - ua;
          cb = 0;
        } else {
          ua = t - (P / 2 + 1);
          ca = Q / 2;
          ub = P - 1 - ua;
          cb = Q / 2;
        }
        V2* sa = xs + (ua * Q + ca) * LW + lane;
        V2* sb = xs + (ub * Q + cb) * LW + lane;
        cx<T> cf;
        int bin = mode_shell<T, N>(Q * ua + ca, ky, kz, cd, cf);
        // The two modes kx and n - kx draw from one Philox call; both draws
        // are made unconditionally (a lone mode draws itself twice and keeps
        // one).
        const cx<T> Fa = ldc<T>(sa), Fb = ldc<T>(sb);
        cx<T> xa, xb;
        xi_pair<T, N>(Q * ua + ca, ky, kz, sweep, k0, k1, cid, xa, xb);
        const T wgt = (kz == 0 || kz == H) ? T(1) : T(2);
        T sg, sg2, ch = T(0), ch2 = T(0);
        const cx<T> ya = signal_draw<T>(Fa, cf, xa, wgt, sg);
        const cx<T> yb = signal_draw<T>(Fb, cf, xb, wgt, sg2);
        if constexpr (kMixDraw) {
          ch = wgt * (ya.re * Fa.re + ya.im * Fa.im);
          ch2 = wgt * (yb.re * Fb.re + yb.im * Fb.im);
        }
        stc<T>(sa, ya);
        if (two) {
          stc<T>(sb, yb);
          sg += sg2;
          ch += ch2;
        }
        if (!valid || bin < 0) {
          bin = -1;
          sg = T(0);
          ch = T(0);
        }
        if constexpr (kMixDraw) shell_accumulate<T, 2>(sg, ch, bin, accw, lane);
        else shell_accumulate<T, 1>(sg, T(0), bin, accw, lane);
      }
      if constexpr (!kMixDraw) {
        i1_col(va);
        i1_col(vb);
      }
    }
  } else {
    for (int it = threadIdx.x; it < LW * Q; it += NT) {
      const int vq = it / LW;
      cx<T> X[P];
#pragma unroll
      for (int p = 0; p < P; ++p) X[p] = ldc<T>(xs + (p * Q + vq) * LW + lane);
      Dft<P, -1, T>::run(X);
#pragma unroll
      for (int u = 0; u < P; ++u) stc<T>(xs + (u * Q + vq) * LW + lane, X[u]);
      if constexpr (kAdj) {
#pragma unroll
        for (int p = 0; p < P; ++p) X[p] = ldc<T>(xs2 + (p * Q + vq) * LW + lane);
        Dft<P, -1, T>::run(X);
#pragma unroll
        for (int u = 0; u < P; ++u) stc<T>(xs2 + (u * Q + vq) * LW + lane, X[u]);
      }
#pragma unroll 1
      for (int u = 0; u < P; ++u) {
        V2* slot = xs + (u * Q + vq) * LW + lane;
        int bin;
        T sg, ch = T(0);
        cx<T> y;
        if constexpr (kMixDraw) {
          const cx<T> F = ldc<T>(slot);
          cx<T> cf;
          bin = mode_shell<T, N>(Q * u + vq, ky, kz, cd, cf);
          const T wgt = (kz == 0 || kz == H) ? T(1) : T(2);
          y = signal_draw<T>(F, cf, mode_xi<T, N>(Q * u + vq, ky, kz, sweep, k0, k1, cid), wgt, sg);
          ch = wgt * (y.re * F.re + y.im * F.im);
          if (!valid || bin < 0) {
            bin = -1;
            sg = T(0);
            ch = T(0);
          }
        } else if constexpr (!kAdj) {
          y = draw_mode<T, N>(ldc<T>(slot), Q * u + vq, ky, kz, valid, cd, sweep, k0, k1, cid, bin, sg);
        } else {
          y = adjoint_mode<T, N, MODE>(ldc<T>(slot), ldc<T>(xs2 + (u * Q + vq) * LW + lane), Q * u + vq, ky, kz,
                                       valid, cd, sweep, k0, k1, cid, bin, sg, ch);
        }
        stc<T>(slot, y);
        shell_accumulate<T, kNV>(sg, ch, bin, accw, lane);
      }
      if constexpr (!kMixDraw) {
#pragma unroll
        for (int p = 0; p < P; ++p) X[p] = ldc<T>(xs + (p * Q + vq) * LW + lane);
        Dft<P, +1, T>::run(X);
        cx<T> w[P];
        ld_tw_row<T, P>(a.tw + TL::kCvp + vq * P, w);
#pragma unroll
        for (int p = 0; p < P; ++p) stc<T>(xs + (p * Q + vq) * LW + lane, p == 0 ? X[p] : cmulc(X[p], w[p]));
      }
    }
  }
  __syncthreads();

  // Mixing sweep, first half: the drawn modes go to k space (kx = slot index).
  if constexpr (kMixDraw) {
    if (valid)
      for (int kx = warp; kx < N; kx += NW) stc<T>(base + size_t(kx) * stride, ldc<T>(xs + kx * LW + lane));
  }

  // Stage I2: IDFT_Q over v of slot p*Q + v, out to x = p + P q (adjoint
  // passes write the adjoint state, held in main/nyq).
  for (int it = threadIdx.x; it < (kMixDraw ? 0 : LW * P); it += NT) {
    const int p = it / LW;
    cx<T> v[Q];
#pragma unroll
    for (int vq = 0; vq < Q; ++vq) v[vq] = ldc<T>(xs + (p * Q + vq) * LW + lane);
    Dft<Q, +1, T>::run(v);
    if (valid) {
#pragma unroll
      for (int q = 0; q < Q; ++q) stc<T>(base + size_t(p + P * q) * stride, v[q]);
    }
  }

  // Per-tile shell sums: combine the warps in a fixed order, then FP64 (the
  // second value is 0 in plain sweeps).
  double* part = cd.partial + size_t(tile) * B1 * 2;
  constexpr int kW = Acc<T>::kWordsPerValue * kNV;  // words per shell in a warp's sums
  for (int b = threadIdx.x; b < (kMixScale ? 0 : B1); b += NT) {
    if constexpr (sizeof(T) == 4) {
      float h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
      for (int w2 = 0; w2 < NW; ++w2) {
        const float* ac = acc + w2 * B1 * Acc<T>::kWords + b * kW;
        Acc<float>::two_sum(h1, l1, ac[0]);
        l1 += ac[1];
        if constexpr (kNV == 2) {
          Acc<float>::two_sum(h2, l2, ac[2]);
          l2 += ac[3];
        }
      }
      part[2 * b + 0] = double(h1) + double(l1);
      part[2 * b + 1] = double(h2) + double(l2);
    } else {
      double s1 = 0.0, s2 = 0.0;
      for (int w2 = 0; w2 < NW; ++w2) {
        const double* ac = acc + w2 * B1 * Acc<T>::kWords + b * kW;
        s1 += ac[0];
        if constexpr (kNV == 2) s2 += ac[1];
      }
      part[2 * b + 0] = s1;
      part[2 * b + 1] = s2;
    }
  }
}

template <typename T, int N, int NT, int MINB, int MODE = kXSweep>
__global__ void __launch_bounds__(NT, MINB) pass_x_kernel(const __grid_constant__ LaunchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_x_tile<T, N, NT, MODE>(a, int(blockIdx.x), smem_raw);
}

}  // namespace mg
