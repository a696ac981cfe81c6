// Device-side data structures shared by the sweep kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "mg_fft.cuh"
#include "mg_rng.cuh"

namespace mg {

template <typename T>
struct VT;
template <>
struct VT<float> {
  using c2 = float2;
};
template <>
struct VT<double> {
  using c2 = double2;
};

template <typename T>
__device__ __forceinline__ cx<T> ldc(const typename VT<T>::c2* p) {
  const typename VT<T>::c2 v = *p;
  return {v.x, v.y};
}
// Load through L2 only: chain state is streamed once per pass, and inside the
// persistent sweep another SM may have rewritten it since this SM last saw
// the line, so it must not come from a (non-coherent) L1 copy.
template <typename T>
__device__ __forceinline__ cx<T> ldcg(const typename VT<T>::c2* p) {
  const typename VT<T>::c2 v = __ldcg(p);
  return {v.x, v.y};
}
template <typename T>
__device__ __forceinline__ void stc(typename VT<T>::c2* p, cx<T> a) {
  typename VT<T>::c2 v;
  v.x = a.re;
  v.y = a.im;
  *p = v;
}

// sqrt(x) for x >= 0 as the messenger draw needs it: correctly rounded in
// FP64; in FP32 the special-function unit's root (relative error below 2^-22,
// well inside the FP32 path's error budget, one instruction).
__device__ __forceinline__ double msg_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float msg_sqrt(float x) { return sqrt_fast(x); }

// Double-float sums (hi, lo) of FP32 values for the recorded samples: the
// exact sum of (hi, lo) and q is hi + lo + q; TwoSum (Knuth) gives s + e =
// hi + q exactly, the error joins lo, and Fast2Sum renormalises so |lo| <=
// ulp(hi)/2.  Relative accuracy about 2^-44 over any number of additions.
__device__ __forceinline__ void df_add(float& hi, float& lo, float q, float qe) {
  const float s = hi + q;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (q - bp);
  const float t = lo + (e + qe);
  hi = s + t;
  lo = t - (hi - s);
}
// (h0, l0) += x0 and (h1, l1) += x1
__device__ __forceinline__ void df_add_sample(float& h0, float& l0, float& h1, float& l1, float x0, float x1) {
  df_add(h0, l0, x0, 0.f);
  df_add(h1, l1, x1, 0.f);
}
// (h0, l0) += x0^2 and (h1, l1) += x1^2, each square split exactly into
// x * x and its rounding error fma(x, x, -x * x) (the product rounded on its
// own: __fmul_rn is never contracted into the following addition)
__device__ __forceinline__ void df_add_square(float& h0, float& l0, float& h1, float& l1, float x0, float x1) {
  const float p0 = __fmul_rn(x0, x0), p1 = __fmul_rn(x1, x1);
  df_add(h0, l0, p0, fmaf(x0, x0, -p0));
  df_add(h1, l1, p1, fmaf(x1, x1, -p1));
}

// Position of voxel (x, y, z) of an n^3 grid (n = P Q) in the sums of the
// recorded samples: [x][z/4][slot][z%4] with slot = (y mod P) Q + y div P,
// the order in which pass YZ's messenger stage visits the rows (consecutive
// lanes take consecutive slots), so a warp's accesses of four voxels each are
// one contiguous block.
__host__ __device__ inline size_t sums_index(int n, int P, int Q, int x, int y, int z) {
  const int slot = (y % P) * Q + y / P;
  return ((size_t(x) * size_t(n / 4) + size_t(z / 4)) * size_t(n) + size_t(slot)) * 4 + size_t(z % 4);
}

// Modes of pass YZ (mg_pass_yz.cuh).
enum PassYZMode : int {
  kModeSweep = 0,        // inverse -> messenger draw -> forward (the hot path)
  kModeMaterialize = 1,  // inverse only, write s to ChainDev::s_out
  kModeLoad = 2,         // read s from ChainDev::s_in, forward only
  kModeAdjoint = 3,      // adjoint of the messenger step: inverse -> lam_t;
                         // dd += lam_t (observed rows only); b lam_t -> forward
  kModeSweepRecord = 4,  // kModeSweep that also adds the incoming s to the
                         // chain's sums (s1, s2) when *rec_now is set
};

// Device status bits (sticky on the context once read by the host).
enum : int { kStNumeric = 1, kStTimeout = 2, kStBadInput = 4, kStNoObserved = 8, kStBounds = 16 };

// Largest grid size the kernels are instantiated for (the bounds-checked build
// compiles the small sizes only).
#ifndef MG_MAX_N
#define MG_MAX_N 256
#endif

// Bounds-checked build (-DMG_CHECKED): every device index that comes from a
// table built on the host, not from compile-time loop limits over the grid and
// the tile, is compared with its buffer before use.  A violation sets
// kStBounds in the context's status word (reported as MG_EBOUNDS, sticky) and
// the access is skipped; nothing traps.  Without MG_CHECKED the checks are not
// compiled.
__device__ __forceinline__ void flag_bounds(int* status) {
  if (status) atomicOr(status, kStBounds);
}

// One chain as the sweep kernels see it.  State layout (per chain):
//   main[x][ky][kz]  kz in [0, n/2)  complex: the spectrum with x still in
//                    real space (the x-transform is undone at the end of pass X)
//   nyq[x][ky]                      complex: the kz = n/2 plane, same form
// Group data (shared by all chains of one data set), for the messenger draw
// t = c + b s + sqrt(tau b) g:
//   row_info[x][y]  (offset, lo | hi << 16): the z-range [lo, hi) of the row
//                   that holds observed voxels (lo, hi multiples of 4), and
//                   where it starts in bc_rows; unobserved voxels have b = 1,
//                   c = 0 and are not stored there
//   bc_rows[]       (b, c) of those ranges, row after row
//   bin_of_m2[m^2]  shell id of a mode with |m|^2 = m^2 (B = overflow shell)
template <typename T>
struct ChainDev {
  typename VT<T>::c2* main;
  typename VT<T>::c2* nyq;
  const uint2* row_info;
  const typename VT<T>::c2* bc_rows;
  const typename VT<T>::c2* coef;  // [B+2]: (a / M, sd / sqrt(M)) per shell; [B+1] = DC
  const T* mscale;                 // [B+2] mixing sweeps: sqrt(S_new / S_old) per shell; [B+1] = DC
  double* partial;                 // [tiles][B+1][2]: per-tile (sigma_b, X_b)
  const uint8_t* bin_of_m2;
  T* s_out;                        // real-space output of the materialise pass
  const T* s_in;                   // real-space input of the load pass
  // adjoint passes only (see mg_adjoint):
  const typename VT<T>::c2* main_in;  // pass X: first input state (else main)
  const typename VT<T>::c2* nyq_in;
  const typename VT<T>::c2* main2;    // pass X: the recomputed y/z transform of t
  const typename VT<T>::c2* nyq2;
  const T* wloss;                     // [n][n][n/2+1] loss weight per stored mode
  T* dd;                              // [M] sum of lam_t over the adjoint sweeps (observed rows)
  double* s1;                         // [M] sum of the recorded samples of s (record_every > 0):
                                      // FP64, or for FP32 chains a (hi, lo) float pair
  double* s2;                         // [M] sum of their squares, the same way
  int* status;                        // the context's device status word
  uint32_t bc_rows_len;               // complex entries in bc_rows
  T tau;
  int B;
};

// Kernel parameters of one pass launch.  The Philox keys and chain ids sit in
// the parameter space so every CTA reads them with a uniform index; a launch
// covers at most kMaxLaunchChains chains (the host splits larger batches).
constexpr int kMaxLaunchChains = 64;
template <typename T>
struct LaunchArgs {
  const ChainDev<T>* chains;
  const uint32_t* sweep_ctr;
  const typename VT<T>::c2* tw;  // twiddle tables of this grid size (TwLayout)
  int n_chains;
  int pf_units;  // pass X: prefetch into L2 the input of tile + pf_units (0: none)
  const int* rec_now;  // pass YZ record mode: nonzero if the incoming state is a sample to add
  uint32_t k0[kMaxLaunchChains];
  uint32_t k1[kMaxLaunchChains];
  uint32_t cid[kMaxLaunchChains];
};

// Twiddle tables of one grid size n = P Q (rows of length n/2 = P2 Q2), all
// W_n^e = exp(-2 pi i e / n), laid out so that a stage reads the twiddles it
// needs as one contiguous row:
//   lin[k]      W_n^k,        k < n
//   cvp[v][p]   W_n^{p v},    v < Q, p < P    (column/x stages looping over v)
//   cpv[p][v]   W_n^{p v},    p < P, v < Q    (column/x stages looping over p)
//   rvp[v][p]   W_n^{2 p v},  v < Q2, p < P2  (row stages looping over v)
//   rpv[p][v]   W_n^{2 p v},  p < P2, v < Q2  (row stages looping over p)
template <int N>
struct TwLayout {
  static constexpr int kLin = 0, kCvp = N, kCpv = 2 * N, kRvp = 3 * N, kRpv = 3 * N + N / 2;
  // kLin in column order of the row stages: entry v*P2 + u = W_N^(Q2 u + v)
  static constexpr int kLinT = 4 * N;
  static constexpr int kSize = 4 * N + N / 2;
};

// Load K consecutive complex twiddles (16-byte vector loads where aligned).
template <typename T, int K>
__device__ __forceinline__ void ld_tw_row(const typename VT<T>::c2* __restrict__ row, cx<T>* w) {
  if constexpr (sizeof(T) == 4 && K % 2 == 0) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
    for (int i = 0; i < K / 2; ++i) {
      const float4 q = __ldg(r4 + i);
      w[2 * i] = {q.x, q.y};
      w[2 * i + 1] = {q.z, q.w};
    }
  } else {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const typename VT<T>::c2 q = __ldg(row + i);
      w[i] = {q.x, q.y};
    }
  }
}

// Load two consecutive complex twiddles row[0], row[1] (one 16-byte load in
// FP32; row must then be 16-byte aligned).
template <typename T>
__device__ __forceinline__ void ld_tw2(const typename VT<T>::c2* __restrict__ row, cx<T>& w0, cx<T>& w1) {
  if constexpr (sizeof(T) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(row));
    w0 = {q.x, q.y};
    w1 = {q.z, q.w};
  } else {
    const typename VT<T>::c2 a = __ldg(row), b = __ldg(row + 1);
    w0 = {a.x, a.y};
    w1 = {b.x, b.y};
  }
}

// What the P-draw kernel needs per chain.
struct DrawDev {
  const double* partial;
  int n_tiles;
  int B;
  const long long* n_b;
  double* P;
  double* sig_last;
  double* chi_last;
  void* coef;    // float2 or double2 [B+2]
  void* mscale;  // float or double [B+2] (mixing sweeps)
  double tau;
  double M;
  double V;
  uint32_t k0, k1, cid;  // Philox key and chain id (mixing sweeps' proposals)
};

}  // namespace mg
