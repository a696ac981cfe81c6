// Small kernels around the two sweep passes: set-up of the messenger
// constants (Sec. 2 and the t-conditional of Sec. 3.1), the per-shell
// inverse-gamma draw (Sec. 3.2, Alg. 2 on shells), chain statistics and the
// raw Philox fill used to check the generator bit for bit.
#pragma once
#include "mg_device.cuh"

namespace mg {

// tau bound: min over observed voxels of N_i / R_i^2 (Sec. 2, diagonal R).
// Positive doubles order like their bit patterns, so the minimum is an
// integer atomicMin and independent of the order of the updates.  Also flags
// invalid inputs (R < 0, N <= 0 where R > 0, non-finite) and counts observed
// voxels.
__global__ void tau_bound_kernel(const double* __restrict__ N, const double* __restrict__ R,
                                 const double* __restrict__ d, size_t M, unsigned long long* min_bits,
                                 unsigned long long* n_obs, int* status) {
  unsigned long long local_min = 0x7FF0000000000000ull;  // +inf
  unsigned long long local_obs = 0;
  int bad = 0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x) {
    const double r = R[i], n = N[i], dd = d[i];
    if (!(r >= 0.0) || !isfinite(r)) bad = 1;
    if (r > 0.0) {
      if (!(n > 0.0) || !isfinite(n) || !isfinite(dd)) bad = 1;
      const double q = __ddiv_rn(n, __dmul_rn(r, r));
      if (q > 0.0 && isfinite(q)) {
        const unsigned long long b = __double_as_longlong(q);
        local_min = b < local_min ? b : local_min;
      } else {
        bad = 1;
      }
      ++local_obs;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_down_sync(0xffffffffu, local_min, off);
    local_min = o < local_min ? o : local_min;
    local_obs += __shfl_down_sync(0xffffffffu, local_obs, off);
    bad |= __shfl_down_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(min_bits, local_min);
    atomicAdd(n_obs, local_obs);
    if (bad) atomicOr(status, kStBadInput);
  }
}

// Per-voxel constants of the messenger draw t = c + b s + sqrt(tau b) g:
//   observed:   N~ = max(N - R tau R, 0), b = N~ / (tau R^2 + N~),
//               c = tau / (tau R^2 + N~) * R * d
//   unobserved: b = 1, c = 0   (mu = s, sigma^2 = T).
// Products and sums are rounded one by one (no FMA contraction).
// Also writes gamma = dc/dd = tau R / (tau R^2 + N~) (0 unobserved), the
// factor through which the data enter the messenger draw.
template <typename T>
__global__ void messenger_constants_kernel(const double* __restrict__ N, const double* __restrict__ R,
                                           const double* __restrict__ d, size_t M, double tau,
                                           typename VT<T>::c2* __restrict__ bc, T* __restrict__ gamma) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x) {
    const double r = R[i];
    double b = 1.0, c = 0.0, gm = 0.0;
    if (__dmul_rn(r, r) > 0.0) {
      double nt = __dsub_rn(N[i], __dmul_rn(__dmul_rn(r, tau), r));
      nt = nt > 0.0 ? nt : 0.0;
      const double den = __dadd_rn(__dmul_rn(tau, __dmul_rn(r, r)), nt);
      b = __ddiv_rn(nt, den);
      gm = __dmul_rn(__ddiv_rn(tau, den), r);
      c = __dmul_rn(gm, d[i]);
    }
    typename VT<T>::c2 v;
    v.x = T(b);
    v.y = T(c);
    bc[i] = v;
    gamma[i] = T(gm);
  }
}

// The observed z-range of each z-row (x, y): [lo, hi) spans the voxels with
// R > 0, widened to multiples of 4 (lo down, hi up); a row with none gets
// [0, 0).  One warp per row; lohi[row] = lo | hi << 16.
__global__ void row_range_kernel(const double* __restrict__ R, int n, size_t rows, uint32_t* __restrict__ lohi) {
  const int lane = threadIdx.x & 31;
  const size_t warps = size_t(gridDim.x) * blockDim.x / 32;
  for (size_t row = (blockIdx.x * size_t(blockDim.x) + threadIdx.x) / 32; row < rows; row += warps) {
    int lo = n, hi = 0;
    for (int z = lane; z < n; z += 32)
      if (R[row * n + z] > 0.0) {
        lo = min(lo, z);
        hi = max(hi, z + 1);
      }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
      if (hi <= lo) lo = hi = 0;
      lo &= ~3;
      hi = (hi + 3) & ~3;
      lohi[row] = uint32_t(lo) | (uint32_t(hi) << 16);
    }
  }
}

// Copy each row's observed z-range of (b, c) into the compact row store.
template <typename T>
__global__ void pack_rows_kernel(const typename VT<T>::c2* __restrict__ bc, const uint2* __restrict__ row_info,
                                 int n, typename VT<T>::c2* __restrict__ bc_rows) {
  const size_t M = size_t(n) * n * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x) {
    const uint2 ri = row_info[i / n];
    const uint32_t z = uint32_t(i % n), lo = ri.y & 0xffffu, hi = ri.y >> 16;
    if (z >= lo && z < hi) bc_rows[ri.x + (z - lo)] = bc[i];
  }
}

// New data d: c = gamma d (b does not depend on d).
template <typename T>
__global__ void set_data_kernel(const T* __restrict__ gamma, const double* __restrict__ d, size_t M,
                                typename VT<T>::c2* __restrict__ bc) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x)
    bc[i].y = T(double(gamma[i]) * d[i]);
}

// Adjoint: add one sweep's per-tile (gradient, loss) partials of every shell
// to the running totals, summing the tiles in a fixed order.  Grid: B+1.
__global__ void adjoint_reduce_kernel(const double* __restrict__ partial, int n_tiles, int B1,
                                      double* __restrict__ grad, double* __restrict__ loss) {
  const int b = blockIdx.x;
  __shared__ double r1[256], r2[256];
  double s1 = 0.0, s2 = 0.0;
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    s1 += partial[(size_t(t) * B1 + b) * 2 + 0];
    s2 += partial[(size_t(t) * B1 + b) * 2 + 1];
  }
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    grad[b] += r1[0];
    loss[b] += r2[0];
  }
}

// The kernels' unit normals from given Philox words (mg_normals).
template <typename T>
__global__ void normals_kernel(const uint32_t* __restrict__ words, long long n_pairs, T* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pairs;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t wa = words[2 * i], wb = words[2 * i + 1];
    T z0, z1;
    normal_pair<T>(wa, wb, z0, z1);
    out[3 * i] = z0;
    out[3 * i + 1] = z1;
    out[3 * i + 2] = radius2<T>(wa);
  }
}

// The sweep counter set on the device: *ctr = *base + add (no host round trip).
__global__ void sweep_ctr_kernel(uint32_t* __restrict__ ctr, const uint32_t* __restrict__ base, uint32_t add) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *ctr = *base + add;
}

// The adjoint's loss weights in device precision.  On the kz = 0 and n/2
// planes both k and -k are stored; the loss counts each with its own weight,
// but the transforms act on the Hermitian part of a plane only, so the
// adjoint seed uses the pair's mean weight (the loss is the same since
// |s_hat(k)| = |s_hat(-k)|).
template <typename T>
__global__ void adjoint_weights_kernel(const double* __restrict__ w, int n, T* __restrict__ out) {
  const int H = n / 2;
  const size_t total = size_t(n) * n * (H + 1);
  for (size_t j = blockIdx.x * size_t(blockDim.x) + threadIdx.x; j < total; j += size_t(gridDim.x) * blockDim.x) {
    const int kz = int(j % (H + 1));
    const size_t r = j / (H + 1);
    const int ky = int(r % n), kx = int(r / n);
    double v = w[j];
    if (kz == 0 || kz == H) {
      const size_t jp = (size_t((n - kx) % n) * n + (n - ky) % n) * (H + 1) + kz;
      v = 0.5 * (w[j] + w[jp]);
    }
    out[j] = T(v);
  }
}

// dL/dd = gamma * (lam_t summed over the adjoint sweeps), widened to FP64
// for the caller (gamma = dc/dd = tau R / (tau R^2 + N~), 0 unobserved).
template <typename T>
__global__ void widen_kernel(const T* __restrict__ x, const T* __restrict__ g, size_t M, double* __restrict__ y) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x)
    y[i] = double(g[i]) * double(x[i]);
}

// Shell draw and the next sweep's per-shell coefficients.  One CTA per
// (chain, shell): sum the per-tile partials sigma_b in a fixed order in FP64
// (deterministic), then S_b = sigma_b / X_b with X_b ~ chi^2_{n_b} drawn once
// per shell (chi2_shell), i.e. S_b | s ~ InvGamma(n_b/2, sigma_b/2) from
// Jeffreys' prior (Sec. 3.2, Alg. 2 on shells); P_b = (V/M) S_b.  Empty shells,
// and shells whose sigma_b or X_b is not positive and finite (flagged), keep
// their P.  Then a_b = S/(S + tau), sd_b = sqrt(S tau / (S + tau)) (Sec. 3.1),
// stored as (a_b / M, sd_b / sqrt(M)) for pass X; the DC entry is 0.
// draw = 0: only recompute the coefficients from P (set-up, mg_set_pk).
// fix_P != 0: sum the shells but keep P (the signal sampler alone).
// sweep_ctr (a sweep, not set-up): word 0 is the sweep counter, which the
// chi-square draws read; the last CTA to finish advances it (word 1 counts
// the finished CTAs), so no CTA can read an advanced counter.
template <typename T>
__global__ void shell_draw_kernel(const DrawDev* __restrict__ chains, int draw, int fix_P, int* status,
                                  uint32_t* sweep_ctr) {
  const DrawDev cd = chains[blockIdx.x];
  const int b = blockIdx.y;
  const bool active = b <= cd.B;  // the same for the whole CTA
  const int B1 = cd.B + 1;
  __shared__ double r1[256];
  double s1 = 0.0;
  if (draw && active) {
    for (int t = threadIdx.x; t < cd.n_tiles; t += blockDim.x) s1 += cd.partial[(size_t(t) * B1 + b) * 2 + 0];
  }
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) r1[threadIdx.x] += r1[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  if (active) {
    double P = cd.P[b];
    if (draw) {
      const double sig = r1[0] * cd.M;  // pass X sums w |s_hat|^2 / M
      double chi = 0.0;
      if (!fix_P && cd.n_b[b] > 0) {
        chi = chi2_shell(cd.n_b[b], uint32_t(b), *sweep_ctr, cd.cid, cd.k0, cd.k1);
        if (sig > 0.0 && chi > 0.0 && isfinite(sig) && isfinite(chi)) {
          P = (cd.V / cd.M) * sig / chi;
        } else {
          atomicOr(status, kStNumeric);
        }
      }
      cd.sig_last[b] = sig;
      cd.chi_last[b] = chi;
      cd.P[b] = P;
    }
    const double Sh = (cd.M / cd.V) * P;
    const double a = Sh / (Sh + cd.tau);
    const double sd = sqrt(Sh * cd.tau / (Sh + cd.tau));
    typename VT<T>::c2* coef = static_cast<typename VT<T>::c2*>(cd.coef);
    typename VT<T>::c2 v;
    v.x = T(a / cd.M);
    v.y = T(sd / sqrt(cd.M));
    coef[b] = v;
    if (b == 0) {
      v.x = T(0);
      v.y = T(0);
      coef[cd.B + 1] = v;
    }
  }
  if (sweep_ctr) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    if (atomicAdd(sweep_ctr + 1, 1u) == total - 1u) {
      sweep_ctr[1] = 0u;
      atomicAdd(sweep_ctr, 1u);
    }
  }
}

// A draw from N(mu, sigma^2) restricted to (0, inf) from shell b's Philox
// calls (b + 256 k, sweep, chain, 4), k < 64: plain rejection of the first
// Box-Muller normal of words (w0, w1) when a = -mu/sigma <= 1/2, else Robert's
// (1995) exponential rejection with rate (a + sqrt(a^2 + 4))/2, U(w0) for the
// exponential and U(w1) for the test.  Returns false if no attempt succeeds.
__device__ inline bool truncated_normal_positive(double mu, double sigma, uint32_t b, uint32_t sweep,
                                                 uint32_t cid, uint32_t k0, uint32_t k1, double* out) {
  const double a = -mu / sigma;
  const double lam = 0.5 * (a + sqrt(a * a + 4.0));
  for (uint32_t k = 0; k < 64; ++k) {
    const u32x4 w = philox4x32_10(b + 256u * k, sweep, cid, kStreamMixing, k0, k1);
    double z;
    if (a <= 0.5) {
      double z1;
      box_muller(w.x, w.y, z, z1);
      if (!(z > a)) continue;
    } else {
      const double u0 = (2.0 * double(w.x) + 1.0) * 0x1p-33;
      const double u1 = (2.0 * double(w.y) + 1.0) * 0x1p-33;
      z = a - log(u0) / lam;
      const double dz = z - lam;
      if (!(u1 <= exp(-0.5 * dz * dz))) continue;
    }
    *out = mu + sigma * z;
    return true;
  }
  return false;
}

// Mixing sweep, shell step (Sec. 3.3, Alg. 3 on k-shells).  One CTA per
// (chain, shell).  Pass X left per tile, per shell, the sums of w |y|^2 and
// w Re(conj(y) F) with y = a t_hat/sqrt(M) + sd xi/sqrt(M) (the plain draw
// scaled by 1/sqrt(M)) and F = sqrt(M) t_hat; with x = y sqrt(M/S) they give
//   B = sum w |x|^2 = (M/S) sum w |y|^2,   A = sum w Re(conj(x) t_hat) = sum w Re(conj(y) F) / sqrt(S).
// u = sqrt(S_b) then takes one Metropolis-Hastings step: proposal
// u' ~ N(A/B, tau/B) truncated to u' > 0, accepted with probability
// min(1, u/u') (the conditional of u is proportional to
// u^-1 exp(-B (u - A/B)^2 / (2 tau))), the acceptance uniform being U(w3) of
// attempt 0.  Writes P, sigma_b = S_new B, the acceptance flag, the scale
// sqrt(S_new/S_old) that turns y into s_hat_new / sqrt(M) in pass X, and the
// next sweep's coefficients.  The sweep counter is read, not advanced (the
// sweep's last kernel advances it).
template <typename T>
__global__ void mixing_draw_kernel(const DrawDev* __restrict__ chains, int* status, const uint32_t* sweep_ctr) {
  const DrawDev cd = chains[blockIdx.x];
  const int b = blockIdx.y;
  if (b > cd.B) return;
  const int B1 = cd.B + 1;
  __shared__ double r1[256], r2[256];
  double s1 = 0.0, s2 = 0.0;
  for (int t = threadIdx.x; t < cd.n_tiles; t += blockDim.x) {
    s1 += cd.partial[(size_t(t) * B1 + b) * 2 + 0];
    s2 += cd.partial[(size_t(t) * B1 + b) * 2 + 1];
  }
  r1[threadIdx.x] = s1;
  r2[threadIdx.x] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      r1[threadIdx.x] += r1[threadIdx.x + w];
      r2[threadIdx.x] += r2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const uint32_t sweep = *sweep_ctr;
  const double S_old = (cd.M / cd.V) * cd.P[b];
  double S_new = S_old;
  double Bx = 0.0;
  int acc = 0;
  if (cd.n_b[b] > 0) {
    Bx = r1[0] * cd.M / S_old;
    const double Ax = r2[0] / sqrt(S_old);
    if (Bx > 0.0 && isfinite(Ax) && isfinite(Bx)) {
      double up;
      if (truncated_normal_positive(Ax / Bx, sqrt(cd.tau / Bx), uint32_t(b), sweep, cd.cid, cd.k0, cd.k1, &up)) {
        const u32x4 w0 = philox4x32_10(uint32_t(b), sweep, cd.cid, kStreamMixing, cd.k0, cd.k1);
        const double alpha = (2.0 * double(w0.w) + 1.0) * 0x1p-33;
        if (alpha * up < sqrt(S_old)) {
          S_new = up * up;
          acc = 1;
        }
      }
    } else {
      atomicOr(status, kStNumeric);
    }
  }
  const double P = (cd.V / cd.M) * S_new;
  cd.P[b] = P;
  cd.sig_last[b] = S_new * Bx;
  cd.chi_last[b] = double(acc);
  T* ms = static_cast<T*>(cd.mscale);
  ms[b] = T(sqrt(S_new / S_old));
  const double a = S_new / (S_new + cd.tau);
  const double sd = sqrt(S_new * cd.tau / (S_new + cd.tau));
  typename VT<T>::c2* coef = static_cast<typename VT<T>::c2*>(cd.coef);
  typename VT<T>::c2 v;
  v.x = T(a / cd.M);
  v.y = T(sd / sqrt(cd.M));
  coef[b] = v;
  if (b == 0) {
    ms[cd.B + 1] = T(0);
    v.x = T(0);
    v.y = T(0);
    coef[cd.B + 1] = v;
  }
}

// Over-dispersed start of one chain: P_b *= exp(sigma z_b), z_b the first
// Box-Muller normal of Philox call (b, 0, chain, 2).
__global__ void disperse_start_kernel(double* __restrict__ P, int B1, double sigma, uint32_t k0, uint32_t k1,
                                      uint32_t cid) {
  for (int b = threadIdx.x; b < B1; b += blockDim.x) {
    const u32x4 w = philox4x32_10(uint32_t(b), 0u, cid, kStreamStart, k0, k1);
    double z0, z1;
    box_muller(w.x, w.y, z0, z1);
    P[b] *= exp(sigma * z0);
  }
}

// Every chain's P into one row-major staging array of B_max+1 columns (zero
// padded).  Grid: chains.
__global__ void gather_pk_kernel(const DrawDev* __restrict__ chains, int B1max, double* __restrict__ out) {
  const DrawDev cd = chains[blockIdx.x];
  for (int b = threadIdx.x; b < B1max; b += blockDim.x)
    out[size_t(blockIdx.x) * B1max + b] = b <= cd.B ? cd.P[b] : 0.0;
}

// Advance the device sweep counter (end of a mixing sweep).
__global__ void sweep_bump_kernel(uint32_t* sweep_ctr) { atomicAdd(sweep_ctr, 1u); }

// One recorded sample s added to the per-voxel sums of s and s^2 (FP64, or
// double-float pairs for FP32 samples), with the arithmetic of the record
// mode of pass YZ, which does the same inside the sweep.
__device__ __forceinline__ void add_moment(double x, double* s1, double* s2, size_t i) {
  s1[i] += x;
  s2[i] = fma(x, x, s2[i]);
}
__device__ __forceinline__ void add_moment(float x, double* s1, double* s2, size_t i) {
  float2* p1 = reinterpret_cast<float2*>(s1) + i;
  float2* p2 = reinterpret_cast<float2*>(s2) + i;
  float2 u = *p1, w = *p2;
  df_add(u.x, u.y, x, 0.f);
  const float p = __fmul_rn(x, x);
  df_add(w.x, w.y, p, fmaf(x, x, -p));
  *p1 = u;
  *p2 = w;
}
// s: the materialised field in natural [x][y][z] order; the sums in the
// order of sums_index.
template <typename T>
__global__ void moments_kernel(const T* __restrict__ s, double* __restrict__ s1, double* __restrict__ s2, int n,
                               int P, int Q) {
  const size_t M = size_t(n) * n * n;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < M; i += size_t(gridDim.x) * blockDim.x) {
    const int z = int(i % n), y = int((i / n) % n), x = int(i / (size_t(n) * n));
    add_moment(s[i], s1, s2, sums_index(n, P, Q, x, y, z));
  }
}

// Efficiency analysis of a recorded P(k) trace (Sec. 4, statistical
// efficiency; trace[r][b], r < R records, B1 shells).  One CTA of 256 threads
// per shell; sums are formed per thread in a fixed stride order and combined
// by a fixed tree, so results are deterministic.
__device__ inline double block_sum_256(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Autocorrelation of shell b's amplitudes,
//   C_n = [1/(R-n) sum_{i<R-n} (P_i - m)(P_{i+n} - m)] / var,
// m and var the trace mean and (1/R) variance, for n = 0 .. max_lag
// (max_lag < R), and the correlation length n_c = the first n >= 1 with
// C_n < 0.1 (-1 if none up to max_lag).  A constant trace (held shell) has
// C_n = 1 and n_c = -1.
__global__ void pk_acf_kernel(const double* __restrict__ trace, long long R, int B1, int max_lag,
                              double* __restrict__ acf, int* __restrict__ nc) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  // mean about the first sample, so that a constant trace has exactly zero variance
  const double x0 = trace[b];
  double s = 0.0;
  for (long long r = threadIdx.x; r < R; r += 256) s += trace[r * B1 + b] - x0;
  const double m = x0 + block_sum_256(s, red) / double(R);
  s = 0.0;
  for (long long r = threadIdx.x; r < R; r += 256) {
    const double d = trace[r * B1 + b] - m;
    s += d * d;
  }
  const double var = block_sum_256(s, red) / double(R);
  int first = -1;
  for (int n = 0; n <= max_lag; ++n) {
    double c = 1.0;
    if (var > 0.0) {
      s = 0.0;
      for (long long r = threadIdx.x; r + n < R; r += 256) s += (trace[r * B1 + b] - m) * (trace[(r + n) * B1 + b] - m);
      c = block_sum_256(s, red) / (double(R - n) * var);
    }
    if (threadIdx.x == 0) {
      acf[size_t(b) * (max_lag + 1) + n] = c;
      if (first < 0 && n >= 1 && c < 0.1) first = n;
    }
  }
  if (threadIdx.x == 0) nc[b] = first;
}

// Quantile q of shell b's amplitudes with linear interpolation between order
// statistics: h = (R-1) q, k = floor(h), value x_(k) + (h - k)(x_(k+1) - x_(k)).
// The order statistic of rank k is found by ranking every element
// (rank = #{x_j < x_i} + #{j < i : x_j = x_i}, a permutation).  Grid: (B1, n_q).
__global__ void pk_quantile_kernel(const double* __restrict__ trace, long long R, int B1,
                                   const double* __restrict__ q, double* __restrict__ out) {
  __shared__ double xk[2];
  const int b = blockIdx.x, iq = blockIdx.y;
  const double h = double(R - 1) * q[iq];
  const long long k = (long long)floor(h);
  const long long k1 = k + 1 < R ? k + 1 : k;
  for (long long i = threadIdx.x; i < R; i += blockDim.x) {
    const double xi = trace[i * B1 + b];
    long long rank = 0;
    for (long long j = 0; j < R; ++j) {
      const double xj = trace[j * B1 + b];
      rank += (xj < xi) || (xj == xi && j < i);
    }
    if (rank == k) xk[0] = xi;
    if (rank == k1) xk[1] = xi;
  }
  __syncthreads();
  if (threadIdx.x == 0) out[size_t(b) * gridDim.y + iq] = xk[0] + (h - double(k)) * (xk[1] - xk[0]);
}

// Gelman-Rubin potential scale reduction of shell b's amplitudes over m
// chains' traces (records burn .. R-1, n = R - burn >= 2 per chain): chain
// means and unbiased variances, W = mean of the variances,
// B = n/(m-1) sum_j (mean_j - mean)^2, var+ = (n-1)/n W + B/n,
// R-hat = sqrt(var+ / W); 1 for a shell whose chains are all constant and
// equal, +inf if they are constant but differ.  One CTA per shell.
__global__ void pk_rhat_kernel(const double* const* __restrict__ traces, int m, long long R, long long burn,
                               int B1, double* __restrict__ out) {
  __shared__ double red[256], mj[256], vj[256];  // m <= 256
  const int b = blockIdx.x;
  const long long n = R - burn;
  for (int j = 0; j < m; ++j) {
    const double* tr = traces[j];
    const double x0 = tr[burn * B1 + b];  // mean about the first sample (exact for a constant chain)
    double s = 0.0;
    for (long long r = burn + threadIdx.x; r < R; r += 256) s += tr[r * B1 + b] - x0;
    const double mean_j = x0 + block_sum_256(s, red) / double(n);
    s = 0.0;
    for (long long r = burn + threadIdx.x; r < R; r += 256) {
      const double d = tr[r * B1 + b] - mean_j;
      s += d * d;
    }
    const double var_j = block_sum_256(s, red) / double(n - 1);
    if (threadIdx.x == 0) {
      mj[j] = mean_j;
      vj[j] = var_j;
    }
  }
  if (threadIdx.x != 0) return;
  double mean = 0.0, W = 0.0;
  for (int j = 0; j < m; ++j) {
    mean += mj[j];
    W += vj[j];
  }
  mean /= m;
  W /= m;
  double ss = 0.0;
  for (int j = 0; j < m; ++j) ss += (mj[j] - mean) * (mj[j] - mean);
  const double Bv = double(n) / double(m - 1) * ss;
  const double vplus = double(n - 1) / double(n) * W + Bv / double(n);
  double r;
  if (W > 0.0) r = sqrt(vplus / W);
  else r = Bv > 0.0 ? INFINITY : 1.0;
  out[b] = r;
}

__global__ void philox_fill_kernel(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                   long long n, uint4* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const u32x4 w = philox4x32_10(c0 + uint32_t(i), c1, c2, c3, k0, k1);
    out[i] = make_uint4(w.x, w.y, w.z, w.w);
  }
}

}  // namespace mg
