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
template <typename T>
__device__ __forceinline__ void stc(typename VT<T>::c2* p, cx<T> a) {
  typename VT<T>::c2 v;
  v.x = a.re;
  v.y = a.im;
  *p = v;
}

// Device status bits (sticky on the context once read by the host).
enum : int { kStNumeric = 1, kStTimeout = 2, kStBadInput = 4, kStNoObserved = 8 };

// One chain as the sweep kernels see it.  State layout (per chain):
//   main[x][ky][kz]  kz in [0, n/2)  complex: the spectrum with x still in
//                    real space (the x-transform is undone at the end of pass X)
//   nyq[x][ky]                      complex: the kz = n/2 plane, same form
// Group data (shared by all chains of one data set):
//   bc[x][y][z]     (b, c) of the messenger draw t = c + b s + sqrt(tau b) g
//   bin_of_m2[m^2]  shell id of a mode with |m|^2 = m^2 (B = overflow shell)
template <typename T>
struct ChainDev {
  typename VT<T>::c2* main;
  typename VT<T>::c2* nyq;
  const typename VT<T>::c2* bc;
  const typename VT<T>::c2* coef;  // [B+2]: (a / M, sd / sqrt(M)) per shell; [B+1] = DC
  double* partial;                 // [tiles][B+1][2]: per-tile (sigma_b, X_b)
  const uint8_t* bin_of_m2;
  T* s_out;                        // real-space output of the materialise pass
  const T* s_in;                   // real-space input of the load pass
  T tau;
  uint32_t k0, k1, chain_id;
  int B;
};

// What the P-draw kernel needs per chain.
struct DrawDev {
  const double* partial;
  int n_tiles;
  int B;
  const long long* n_b;
  double* P;
  double* sig_last;
  double* chi_last;
  void* coef;  // float2 or double2 [B+2]
  double tau;
  double M;
  double V;
};

}  // namespace mg
