// Pass YZ of the two-pass sweep, one x-plane per CTA cluster:
//   inverse y-FFT and C2R z-FFT of the previous signal s_hat -> s (real plane)
//   -> messenger draw t | s, d per voxel (Sec. 3.1, Alg. 1 first loop)
//   -> R2C z-FFT and forward y-FFT of t.
//
// The plane (n rows of n/2 packed complex values: column 0 carries the kz = 0
// and kz = n/2 planes as its real and imaginary parts) lives in shared memory,
// split by rows over the C CTAs of a thread-block cluster when it does not fit
// one CTA; column stages reach the other CTAs' rows through distributed shared
// memory.  Every stage reads a set of slots into registers, transforms them and
// writes the results back into the same set of slots, so stages need a barrier
// between them but no second buffer.
//
// Layouts (n = P Q along y, n/2 = P2 Q2 along z):
//   row slot s = p*Q + q holds y = p + P q (the order the y-stages produce);
//   within a row, column l is kz (packed at l = 0).
#pragma once
#include <cooperative_groups.h>

#include "mg_device.cuh"

namespace mg {

namespace cg = cooperative_groups;


template <typename T, int N, int C>
struct PassYZShape {
  static constexpr int H = N / 2;
  static constexpr int P = Split<N>::P, Q = Split<N>::Q;
  static constexpr int P2 = Split<H>::P, Q2 = Split<H>::Q;
  static constexpr int ROWS = N / C;
  static constexpr int RS = H + 1;  // padded row stride (complex elements)
  static constexpr int PC = P / C, QC = Q / C;
  static_assert(P % C == 0 && Q % C == 0, "cluster size must divide both y factors");
  static_assert(P2 % 2 == 0, "row stage pairs adjacent p");
  static constexpr size_t kSmemBytes = (size_t(ROWS) * RS + N) * sizeof(typename VT<T>::c2);
};

// Distributed shared memory through 32-bit shared::cluster addresses: mapa
// turns this CTA's shared address into the same offset in CTA `rank`.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_dsmem(uint32_t addr, cx<float> v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.re), "f"(v.im) : "memory");
}
__device__ __forceinline__ void st_dsmem(uint32_t addr, cx<double> v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.re), "d"(v.im) : "memory");
}
__device__ __forceinline__ cx<float> ld_dsmem(uint32_t addr, float) {
  cx<float> v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.re), "=f"(v.im) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ cx<double> ld_dsmem(uint32_t addr, double) {
  cx<double> v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.re), "=d"(v.im) : "r"(addr) : "memory");
  return v;
}

// p[0..3] += (a.re, a.im, b.re, b.im) with vector accesses (p 16-byte
// aligned for float, 32-byte for double).
__device__ __forceinline__ void add4(float* p, cx<float> a, cx<float> b) {
  float4* q = reinterpret_cast<float4*>(p);
  float4 v = *q;
  v.x += a.re;
  v.y += a.im;
  v.z += b.re;
  v.w += b.im;
  *q = v;
}
__device__ __forceinline__ void add4(double* p, cx<double> a, cx<double> b) {
  double2* q = reinterpret_cast<double2*>(p);
  double2 u = q[0], v = q[1];
  u.x += a.re;
  u.y += a.im;
  v.x += b.re;
  v.y += b.im;
  q[0] = u;
  q[1] = v;
}

// The sums of recorded samples: s1[0..3] += x, s2[0..3] += x^2 for the four
// voxels x = (a.re, a.im, b.re, b.im), with the arithmetic of
// moments_kernel, so fused and separate accumulation agree bit for bit.
// FP64 samples: FP64 sums (s1, s2 32-byte aligned).
__device__ __forceinline__ void add_moments(double* s1, double* s2, cx<double> a, cx<double> b) {
  double2* p1 = reinterpret_cast<double2*>(s1);
  double2* p2 = reinterpret_cast<double2*>(s2);
  double2 u = p1[0], v = p1[1], w = p2[0], z = p2[1];
  u.x += a.re;
  u.y += a.im;
  v.x += b.re;
  v.y += b.im;
  w.x = fma(a.re, a.re, w.x);
  w.y = fma(a.im, a.im, w.y);
  z.x = fma(b.re, b.re, z.x);
  z.y = fma(b.im, b.im, z.y);
  p1[0] = u;
  p1[1] = v;
  p2[0] = w;
  p2[1] = z;
}
// FP32 samples: each sum a double-float (hi, lo) pair of floats in the same
// 8 bytes (FP32 arithmetic only; GB300's FP64 rate is a small fraction of its
// FP32 rate).
__device__ __forceinline__ void add_moments(double* s1, double* s2, cx<float> a, cx<float> b) {
  float4* p1 = reinterpret_cast<float4*>(s1);
  float4* p2 = reinterpret_cast<float4*>(s2);
  float4 u = p1[0], v = p1[1], w = p2[0], z = p2[1];  // (hi, lo) of two voxels each
  df_add_sample(u.x, u.y, u.z, u.w, a.re, a.im);
  df_add_sample(v.x, v.y, v.z, v.w, b.re, b.im);
  df_add_square(w.x, w.y, w.z, w.w, a.re, a.im);
  df_add_square(z.x, z.y, z.z, z.w, b.re, b.im);
  p1[0] = u;
  p1[1] = v;
  p2[0] = w;
  p2[1] = z;
}

template <int C>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (C == 1) {
    __syncthreads();
  } else {
    cg::this_cluster().sync();
  }
}

// A cluster barrier split into its two halves.  The arrive releases this
// thread's earlier writes (and marks its reads of other CTAs' shared memory
// as done); the wait acquires the other CTAs' released writes.  Work placed
// between the two (here: global stores) neither delays the other CTAs nor
// has to be drained before the arrive.  With C == 1 the pair is one
// __syncthreads.
template <int C>
__device__ __forceinline__ void cluster_arrive() {
  if constexpr (C > 1) asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
template <int C>
__device__ __forceinline__ void cluster_wait() {
  if constexpr (C > 1) asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
  else __syncthreads();
}

// One x-plane of one chain (`unit` = plane * n_chains + chain), the CTA's part
// when C > 1.  Called by pass_yz_kernel (one unit per CTA or cluster) and by
// the persistent sweep kernel (C = 1, units taken from a work queue).
template <typename T, int N, int C, int MODE, int NT>
__device__ __forceinline__ void pass_yz_unit(const LaunchArgs<T>& a, int unit, unsigned char* smem_raw) {
  using S = PassYZShape<T, N, C>;
  using V2 = typename VT<T>::c2;
  using TL = TwLayout<N>;
  const typename VT<T>::c2* __restrict__ tw = a.tw;
  constexpr int H = S::H, P = S::P, Q = S::Q, P2 = S::P2, Q2 = S::Q2;
  constexpr int ROWS = S::ROWS, RS = S::RS, PC = S::PC, QC = S::QC;
  // FP32 folds the real-transform pre/post-processing into the row stages
  // (two columns of P2 values per thread); in FP64 those registers would
  // spill, so the pre/post-processing stays a stage of its own there.
  constexpr bool kFuseRows = sizeof(T) == 4;
  V2* rows = reinterpret_cast<V2*>(smem_raw);
  V2* col0 = rows + ROWS * RS;

  unsigned rank = 0;
  uint32_t rbase[C];  // shared::cluster address of each CTA's rows (C > 1)
  uint32_t col0_r0 = 0;
  if constexpr (C > 1) {
    rank = cg::this_cluster().block_rank();
#pragma unroll
    for (int r = 0; r < C; ++r) rbase[r] = map_to_rank(smem_addr(rows), uint32_t(r));
    col0_r0 = map_to_rank(smem_addr(col0), 0u);
  }
  constexpr uint32_t kEl = sizeof(V2);
  const int x = unit / a.n_chains;
  const int chain = unit % a.n_chains;
  const ChainDev<T> cd = a.chains[chain];
  const uint32_t k0 = a.k0[chain], k1 = a.k1[chain], cid = a.cid[chain];
  V2* mainp = cd.main + size_t(x) * N * H;
  V2* nyqp = cd.nyq + size_t(x) * N;
  const uint32_t sweep = *a.sweep_ctr;
  const T tau = cd.tau;
  bool rec = false;
  if constexpr (MODE == kModeSweepRecord) rec = *a.rec_now != 0;

  // Every CTA of the cluster must be running before another writes into its
  // shared memory.  The arrive needs no ordering; the wait comes after this
  // thread's first global loads of stage I1 are in flight.
  if constexpr (C > 1) {
    if constexpr (MODE == kModeLoad) cluster_barrier<C>();
    else asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
  }

  if constexpr (MODE != kModeLoad) {
    // Column stage I1 (per v of this CTA): IDFT_P over u of X[Q u + v] from
    // global, twiddle W_N^{-p v}, to slot p*Q + v (whichever CTA owns it).
    // A thread issues the loads of BI items before transforming any of them.
    constexpr int TI1 = H * QC;
    constexpr int BI = TI1 >= 2 * NT ? 2 : 1;
    bool start_wait = C > 1;  // the start barrier's wait is still due
    for (int it0 = threadIdx.x; it0 < TI1; it0 += BI * NT) {
      cx<T> X[BI][P];
#pragma unroll
      for (int b = 0; b < BI; ++b) {
        const int it = it0 + b * NT;
        if (it < TI1) {
          const int l = it % H;
          const int v = int(rank) * QC + it / H;
#pragma unroll
          for (int u = 0; u < P; ++u) X[b][u] = ldcg<T>(mainp + size_t(Q * u + v) * H + l);
          if (l == 0) {
#pragma unroll
            for (int u = 0; u < P; ++u) {
              const cx<T> y = ldcg<T>(nyqp + Q * u + v);
              X[b][u] = {X[b][u].re - y.im, X[b][u].im + y.re};
            }
          }
        }
      }
      if constexpr (C > 1) {
        if (start_wait) {
          cluster_wait<C>();
          start_wait = false;
        }
      }
#pragma unroll
      for (int b = 0; b < BI; ++b) {
        const int it = it0 + b * NT;
        if (it >= TI1) continue;
        const int l = it % H;
        const int v = int(rank) * QC + it / H;
        Dft<P, +1, T>::run(X[b]);
        cx<T> w[P];
        ld_tw_row<T, P>(tw + TL::kCvp + v * P, w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const cx<T> y = p == 0 ? X[b][p] : cmulc(X[b][p], w[p]);
          // slot p*Q + v lives in CTA p / PC at local row (p % PC)*Q + v
          const int off = ((p % PC) * Q + v) * RS + l;
          if constexpr (C == 1) stc<T>(rows + off, y);
          else st_dsmem(rbase[p / PC] + uint32_t(off) * kEl, y);
        }
      }
    }
    if constexpr (C > 1) {
      if (start_wait) cluster_wait<C>();
    }
    cluster_barrier<C>();

    // Column stage I2 (per p of this CTA, local): IDFT_Q over v; y = p + P q
    // goes to slot p*Q + q.
    for (int it = threadIdx.x; it < H * PC; it += NT) {
      const int l = it % H;
      const int pl = it / H;  // local p index; slots pl*Q + v are local rows
      cx<T> Z[Q];
#pragma unroll
      for (int v = 0; v < Q; ++v) Z[v] = ldc<T>(rows + (pl * Q + v) * RS + l);
      Dft<Q, +1, T>::run(Z);
#pragma unroll
      for (int q = 0; q < Q; ++q) stc<T>(rows + (pl * Q + q) * RS + l, Z[q]);
    }
    __syncthreads();

    if constexpr (kFuseRows) {
      // Row stage I1 with the C2R pre-processing of the z-transform folded in.
      // The C2R runs as a half-length complex IDFT of
      //   Z'[k] = (X[k] + conj X[H-k]) + i W_n^{-k} (X[k] - conj X[H-k]),
      // Z'[0] = (X0 + X_{n/2}) + i (X0 - X_{n/2}) from the packed column 0.
      // Element k = Q2 u + v pairs with H - k, which sits in column Q2 - v
      // (row u' = P2-1-u), or in column 0 itself (u' = P2-u) for v = 0, or in
      // column Q2/2 itself (u' = P2-1-u).  One item therefore takes the two
      // columns {v, Q2-v} (item 0: {0, Q2/2}), forms Z' in registers, runs the
      // IDFT_P2 of each column and twiddles by W_{n/2}^{-p v} into column slots
      // p*Q2 + v.
      constexpr int NG = (Q2 + 1) / 2;
      for (int it = threadIdx.x; it < ROWS * NG; it += NT) {
        const int r = it % ROWS;
        const int g = it / ROWS;
        V2* row = rows + r * RS;
        const int va = g;
        const int vb = g == 0 ? (Q2 % 2 == 0 ? Q2 / 2 : -1) : Q2 - g;
        cx<T> A[P2], Bc[P2];
  #pragma unroll
        for (int u = 0; u < P2; ++u) A[u] = ldc<T>(row + Q2 * u + va);
        if (vb >= 0) {
  #pragma unroll
          for (int u = 0; u < P2; ++u) Bc[u] = ldc<T>(row + Q2 * u + vb);
        }
        const V2* twa = tw + TL::kLinT + va * P2;
        const V2* twb = tw + TL::kLinT + (vb >= 0 ? vb : 0) * P2;
        // x at element k, y at its partner H - k: the pre-processed value at k
        auto pre = [](cx<T> x, cx<T> y, cx<T> w) {
          const cx<T> e = cadd(x, cconj(y)), d = csub(x, cconj(y));
          return cadd(e, cmul_i<+1>(cmulc(d, w)));
        };
        if (g == 0) {
          {
            const cx<T> z = A[0];
            A[0] = {z.re + z.im, z.re - z.im};
          }
  #pragma unroll
          for (int u = 1; u <= P2 / 2; ++u) {
            const cx<T> x = A[u], y = A[P2 - u];
            A[u] = pre(x, y, ldc<T>(twa + u));
            if (P2 - u != u) A[P2 - u] = pre(y, x, ldc<T>(twa + P2 - u));
          }
          if (vb >= 0) {
  #pragma unroll
            for (int u = 0; u < P2 / 2; u += 2) {
              cx<T> w0, w1, w2, w3;
              ld_tw2<T>(twb + u, w0, w1);
              ld_tw2<T>(twb + P2 - 2 - u, w2, w3);
              const cx<T> x0 = Bc[u], y0 = Bc[P2 - 1 - u], x1 = Bc[u + 1], y1 = Bc[P2 - 2 - u];
              Bc[u] = pre(x0, y0, w0);
              Bc[P2 - 1 - u] = pre(y0, x0, w3);
              Bc[u + 1] = pre(x1, y1, w1);
              Bc[P2 - 2 - u] = pre(y1, x1, w2);
            }
          }
        } else {
  #pragma unroll
          for (int u = 0; u < P2; u += 2) {
            cx<T> w0, w1, w2, w3;
            ld_tw2<T>(twa + u, w0, w1);
            ld_tw2<T>(twb + P2 - 2 - u, w2, w3);
            const cx<T> x0 = A[u], y0 = Bc[P2 - 1 - u], x1 = A[u + 1], y1 = Bc[P2 - 2 - u];
            A[u] = pre(x0, y0, w0);
            Bc[P2 - 1 - u] = pre(y0, x0, w3);
            A[u + 1] = pre(x1, y1, w1);
            Bc[P2 - 2 - u] = pre(y1, x1, w2);
          }
        }
        Dft<P2, +1, T>::run(A);
  #pragma unroll
        for (int p = 0; p < P2; p += 2) {
          cx<T> w0, w1;
          ld_tw2<T>(tw + TL::kRvp + va * P2 + p, w0, w1);
          stc<T>(row + p * Q2 + va, p == 0 ? A[p] : cmulc(A[p], w0));
          stc<T>(row + (p + 1) * Q2 + va, cmulc(A[p + 1], w1));
        }
        if (vb >= 0) {
          Dft<P2, +1, T>::run(Bc);
  #pragma unroll
          for (int p = 0; p < P2; p += 2) {
            cx<T> w0, w1;
            ld_tw2<T>(tw + TL::kRvp + vb * P2 + p, w0, w1);
            stc<T>(row + p * Q2 + vb, p == 0 ? Bc[p] : cmulc(Bc[p], w0));
            stc<T>(row + (p + 1) * Q2 + vb, cmulc(Bc[p + 1], w1));
          }
        }
      }
      __syncthreads();
    } else {
      // Row pre-processing for the C2R z-transform through a half-length
      // complex IDFT: Z'[k] = (X[k] + conj X[H-k]) + i W_n^{-k} (X[k] - conj X[H-k]).
      for (int it = threadIdx.x; it < ROWS * (H / 2 + 1); it += NT) {
        const int r = it % ROWS;
        const int k = it / ROWS;
        V2* row = rows + r * RS;
        if (k == 0) {
          const cx<T> z = ldc<T>(row);
          stc<T>(row, cx<T>{z.re + z.im, z.re - z.im});
        } else {
          const int kk = H - k;
          const cx<T> a = ldc<T>(row + k), b = ldc<T>(row + kk);
          {
            const cx<T> e = cadd(a, cconj(b)), d = csub(a, cconj(b));
            stc<T>(row + k, cadd(e, cmul_i<+1>(cmulc(d, ldc<T>(tw + k)))));
          }
          if (kk != k) {
            const cx<T> e = cadd(b, cconj(a)), d = csub(b, cconj(a));
            stc<T>(row + kk, cadd(e, cmul_i<+1>(cmulc(d, ldc<T>(tw + kk)))));
          }
        }
      }
      __syncthreads();

      // Row stage I1 (per v2): IDFT_P2 over u of Z'[Q2 u + v2], twiddle
      // W_{n/2}^{-p v2} = W_n^{-2 p v2}, back to column p*Q2 + v2.
      for (int it = threadIdx.x; it < ROWS * Q2; it += NT) {
        const int r = it % ROWS;
        const int v = it / ROWS;
        V2* row = rows + r * RS;
        cx<T> X[P2];
  #pragma unroll
        for (int u = 0; u < P2; ++u) X[u] = ldc<T>(row + Q2 * u + v);
        Dft<P2, +1, T>::run(X);
        cx<T> w[P2];
        ld_tw_row<T, P2>(tw + TL::kRvp + v * P2, w);
  #pragma unroll
        for (int p = 0; p < P2; ++p) stc<T>(row + p * Q2 + v, p == 0 ? X[p] : cmulc(X[p], w[p]));
      }
      __syncthreads();
    }
  }

  // Row stage I2 + messenger draw + forward stage F1, per pair (p, p+1):
  // IDFT_Q2 gives z[m] = s[2m] + i s[2m+1] for m = p + P2 q, so a pair holds
  // the four consecutive voxels 2m..2m+3 (m even) = one Philox call.
  for (int it = threadIdx.x; it < ROWS * (P2 / 2); it += NT) {
    const int r = it % ROWS;
    const int pp = 2 * (it / ROWS);
    V2* row = rows + r * RS;
    const int sg = int(rank) * ROWS + r;
    const int y = sg / Q + P * (sg % Q);
    const size_t vox_row = (size_t(x) * N + y) * N;
    cx<T> Z0[Q2], Z1[Q2];
    if constexpr (MODE != kModeLoad) {
#pragma unroll
      for (int v = 0; v < Q2; ++v) {
        Z0[v] = ldc<T>(row + pp * Q2 + v);
        Z1[v] = ldc<T>(row + (pp + 1) * Q2 + v);
      }
      Dft<Q2, +1, T>::run(Z0);
      Dft<Q2, +1, T>::run(Z1);
    }
    // Messenger constants: only the row's observed z-range is stored; a
    // group of four voxels outside it has b = 1, c = 0 and needs no load.
    // Each group's constants are loaded ahead of their use (L2 latency).
    constexpr bool kBC = MODE == kModeSweep || MODE == kModeSweepRecord || MODE == kModeAdjoint;  // uses (b, c)
    uint32_t lo = 0, hi = 0;
    const typename VT<T>::c2* brow = nullptr;
    if constexpr (kBC) {
      const uint2 ri = __ldg(cd.row_info + size_t(x) * N + y);
      lo = ri.y & 0xffffu;
      hi = ri.y >> 16;
      brow = cd.bc_rows + ri.x;
#ifdef MG_CHECKED
      // the row's observed range and its offset come from a host table: the
      // range must lie in the row, 4-voxel aligned, and inside bc_rows
      if (!(lo <= hi && hi <= uint32_t(N) && lo % 4 == 0 && hi % 4 == 0 &&
            size_t(ri.x) + (hi - lo) <= size_t(cd.bc_rows_len))) {
        flag_bounds(cd.status);
        lo = hi = 0;  // treated as unobserved: no load
      }
#endif
    }
    auto load_group = [&](int z, cx<T>* out) {
      if (uint32_t(z) >= lo && uint32_t(z) < hi) {
        ld_tw_row<T, 4>(brow + (z - int(lo)), out);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = {T(1), T(0)};
      }
    };
    // (FP32 only: in FP64 the second group in flight costs spills)
    constexpr int kAhead = sizeof(T) == 4 ? 2 : 1;
    cx<T> bc_next[4], bc_next2[4];
    if constexpr (kBC) {
      load_group(2 * pp, bc_next);
      if (kAhead == 2 && Q2 > 1) load_group(2 * (pp + P2), bc_next2);
    }
#pragma unroll
    for (int q = 0; q < Q2; ++q) {
      const int z0 = 2 * (pp + P2 * q);  // voxels z0 .. z0+3
      const size_t i0 = vox_row + z0;
      cx<T> bcv[4];
      if constexpr (kBC) {
#pragma unroll
        for (int k = 0; k < 4; ++k) bcv[k] = bc_next[k];
        if constexpr (kAhead == 2) {
#pragma unroll
          for (int k = 0; k < 4; ++k) bc_next[k] = bc_next2[k];
          if (q + 2 < Q2) load_group(2 * (pp + P2 * (q + 2)), bc_next2);
        } else {
          if (q + 1 < Q2) load_group(2 * (pp + P2 * (q + 1)), bc_next);
        }
      }
      if constexpr (MODE == kModeMaterialize) {
        T* o = cd.s_out + i0;
        o[0] = Z0[q].re;
        o[1] = Z0[q].im;
        o[2] = Z1[q].re;
        o[3] = Z1[q].im;
      } else if constexpr (MODE == kModeLoad) {
        // The state holds the y/z transform of s divided by n^2, the form the
        // x pass leaves behind (its inverse x transform is unnormalised and
        // the unitary 1/sqrt(M) factors sit in the draw coefficients).
        const T* si = cd.s_in + i0;
        const T sc = T(1.0 / (double(N) * double(N)));
        Z0[q] = {si[0] * sc, si[1] * sc};
        Z1[q] = {si[2] * sc, si[3] * sc};
      } else if constexpr (MODE == kModeAdjoint) {
        // t = c + b s + sd g with c = gamma d: d receives gamma lam_t, s
        // receives b lam_t (the transposes of the per-voxel affine map).
        // gamma is the same in every sweep and vanishes outside the row's
        // observed range, so dd sums lam_t there only, over the K adjoint
        // sweeps, and is multiplied by gamma once at the end.
        if (uint32_t(z0) >= lo && uint32_t(z0) < hi) add4(cd.dd + i0, Z0[q], Z1[q]);
        Z0[q] = {bcv[0].re * Z0[q].re, bcv[1].re * Z0[q].im};
        Z1[q] = {bcv[2].re * Z1[q].re, bcv[3].re * Z1[q].im};
      } else {
        if constexpr (MODE == kModeSweepRecord) {
          // the incoming state is a recorded sample: its s (exactly what the
          // materialise pass writes) goes into the sums of s and s^2, stored
          // in row-slot order so the warp's accesses are contiguous
          if (rec) {
            const size_t j = ((size_t(x) * (N / 4) + size_t(z0 / 4)) * N + size_t(sg)) * 4;  // sums_index
            add_moments(cd.s1 + j, cd.s2 + j, Z0[q], Z1[q]);
          }
        }
        const u32x4 w = philox4x32_10(uint32_t(i0 >> 2), sweep, cid, kStreamMessenger, k0, k1);
        T g0, g1, g2, g3;
        normal_pair<T>(w.x, w.y, g0, g1);
        normal_pair<T>(w.z, w.w, g2, g3);
        const cx<T> bc0 = bcv[0], bc1 = bcv[1], bc2 = bcv[2], bc3 = bcv[3];
        Z0[q].re = bc0.im + bc0.re * Z0[q].re + msg_sqrt(tau * bc0.re) * g0;
        Z0[q].im = bc1.im + bc1.re * Z0[q].im + msg_sqrt(tau * bc1.re) * g1;
        Z1[q].re = bc2.im + bc2.re * Z1[q].re + msg_sqrt(tau * bc2.re) * g2;
        Z1[q].im = bc3.im + bc3.re * Z1[q].im + msg_sqrt(tau * bc3.re) * g3;
      }
    }
    if constexpr (MODE != kModeMaterialize) {
      Dft<Q2, -1, T>::run(Z0);
      Dft<Q2, -1, T>::run(Z1);
      cx<T> w0[Q2], w1[Q2];
      ld_tw_row<T, Q2>(tw + TL::kRpv + pp * Q2, w0);
      ld_tw_row<T, Q2>(tw + TL::kRpv + (pp + 1) * Q2, w1);
#pragma unroll
      for (int v = 0; v < Q2; ++v) {
        stc<T>(row + pp * Q2 + v, v == 0 ? Z0[v] : cmul(Z0[v], w0[v]));
        stc<T>(row + (pp + 1) * Q2 + v, v == 0 ? Z1[v] : cmul(Z1[v], w1[v]));
      }
    }
  }
  if constexpr (MODE == kModeMaterialize) return;
  __syncthreads();

  if constexpr (kFuseRows) {
    // Row stage F2 with the R2C post-processing folded in: DFT_P2 over p of
    // column slots p*Q2 + v gives Z[k], k = Q2 u + v, and
    //   X[k] = (Z[k] + conj Z[H-k])/2 - i W_n^{k} (Z[k] - conj Z[H-k])/2,
    // with the real X[0], X[n/2] packed as X[0] + i X[n/2].  Items take the
    // column pairs of row stage I1.
    {
      constexpr int NG = (Q2 + 1) / 2;
      for (int it = threadIdx.x; it < ROWS * NG; it += NT) {
        const int r = it % ROWS;
        const int g = it / ROWS;
        V2* row = rows + r * RS;
        const int va = g;
        const int vb = g == 0 ? (Q2 % 2 == 0 ? Q2 / 2 : -1) : Q2 - g;
        cx<T> A[P2], Bc[P2];
  #pragma unroll
        for (int p = 0; p < P2; ++p) A[p] = ldc<T>(row + p * Q2 + va);
        Dft<P2, -1, T>::run(A);
        if (vb >= 0) {
  #pragma unroll
          for (int p = 0; p < P2; ++p) Bc[p] = ldc<T>(row + p * Q2 + vb);
          Dft<P2, -1, T>::run(Bc);
        }
        const V2* twa = tw + TL::kLinT + va * P2;
        const V2* twb = tw + TL::kLinT + (vb >= 0 ? vb : 0) * P2;
        // x at element k, y at its partner H - k: the post-processed value at k
        auto post = [](cx<T> x, cx<T> y, cx<T> w) {
          const T h = T(0.5);
          const cx<T> e = cscale(cadd(x, cconj(y)), h), o = cscale(csub(x, cconj(y)), h);
          return cadd(e, cmul(cmul_i<-1>(o), w));
        };
        if (g == 0) {
          {
            const cx<T> z = A[0];
            A[0] = {z.re + z.im, z.re - z.im};
          }
  #pragma unroll
          for (int u = 1; u <= P2 / 2; ++u) {
            const cx<T> x = A[u], y = A[P2 - u];
            A[u] = post(x, y, ldc<T>(twa + u));
            if (P2 - u != u) A[P2 - u] = post(y, x, ldc<T>(twa + P2 - u));
          }
          if (vb >= 0) {
  #pragma unroll
            for (int u = 0; u < P2 / 2; u += 2) {
              cx<T> w0, w1, w2, w3;
              ld_tw2<T>(twb + u, w0, w1);
              ld_tw2<T>(twb + P2 - 2 - u, w2, w3);
              const cx<T> x0 = Bc[u], y0 = Bc[P2 - 1 - u], x1 = Bc[u + 1], y1 = Bc[P2 - 2 - u];
              Bc[u] = post(x0, y0, w0);
              Bc[P2 - 1 - u] = post(y0, x0, w3);
              Bc[u + 1] = post(x1, y1, w1);
              Bc[P2 - 2 - u] = post(y1, x1, w2);
            }
          }
        } else {
  #pragma unroll
          for (int u = 0; u < P2; u += 2) {
            cx<T> w0, w1, w2, w3;
            ld_tw2<T>(twa + u, w0, w1);
            ld_tw2<T>(twb + P2 - 2 - u, w2, w3);
            const cx<T> x0 = A[u], y0 = Bc[P2 - 1 - u], x1 = A[u + 1], y1 = Bc[P2 - 2 - u];
            A[u] = post(x0, y0, w0);
            Bc[P2 - 1 - u] = post(y0, x0, w3);
            A[u + 1] = post(x1, y1, w1);
            Bc[P2 - 2 - u] = post(y1, x1, w2);
          }
        }
  #pragma unroll
        for (int u = 0; u < P2; ++u) stc<T>(row + Q2 * u + va, A[u]);
        if (vb >= 0) {
  #pragma unroll
          for (int u = 0; u < P2; ++u) stc<T>(row + Q2 * u + vb, Bc[u]);
        }
      }
    }
    __syncthreads();
  } else {
    // Row stage F2 (per v2): DFT_P2 over p of column p*Q2 + v2 -> Z''[Q2 u + v2].
    for (int it = threadIdx.x; it < ROWS * Q2; it += NT) {
      const int r = it % ROWS;
      const int v = it / ROWS;
      V2* row = rows + r * RS;
      cx<T> X[P2];
  #pragma unroll
      for (int p = 0; p < P2; ++p) X[p] = ldc<T>(row + p * Q2 + v);
      Dft<P2, -1, T>::run(X);
  #pragma unroll
      for (int u = 0; u < P2; ++u) stc<T>(row + Q2 * u + v, X[u]);
    }
    __syncthreads();

    // Row post-processing of the R2C z-transform:
    // X[k] = (Z[k] + conj Z[H-k])/2 - i W_n^{k} (Z[k] - conj Z[H-k])/2, and the
    // real X[0], X[n/2] packed as X[0] + i X[n/2].
    for (int it = threadIdx.x; it < ROWS * (H / 2 + 1); it += NT) {
      const int r = it % ROWS;
      const int k = it / ROWS;
      V2* row = rows + r * RS;
      if (k == 0) {
        const cx<T> z = ldc<T>(row);
        stc<T>(row, cx<T>{z.re + z.im, z.re - z.im});
      } else {
        const int kk = H - k;
        const cx<T> a = ldc<T>(row + k), b = ldc<T>(row + kk);
        const T h = T(0.5);
        {
          const cx<T> e = cscale(cadd(a, cconj(b)), h), o = cscale(csub(a, cconj(b)), h);
          stc<T>(row + k, cadd(e, cmul(cmul_i<-1>(o), ldc<T>(tw + k))));
        }
        if (kk != k) {
          const cx<T> e = cscale(cadd(b, cconj(a)), h), o = cscale(csub(b, cconj(a)), h);
          stc<T>(row + kk, cadd(e, cmul(cmul_i<-1>(o), ldc<T>(tw + kk))));
        }
      }
    }
    __syncthreads();
  }

  // Column stage F1 (per p of this CTA, local): DFT_Q over q of slot p*Q + q,
  // twiddle W_N^{p v}, back to slot p*Q + v.
  for (int it = threadIdx.x; it < H * PC; it += NT) {
    const int l = it % H;
    const int pl = it / H;
    const int p = int(rank) * PC + pl;
    cx<T> Z[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) Z[q] = ldc<T>(rows + (pl * Q + q) * RS + l);
    Dft<Q, -1, T>::run(Z);
    cx<T> w[Q];
    ld_tw_row<T, Q>(tw + TL::kCpv + p * Q, w);
#pragma unroll
    for (int v = 0; v < Q; ++v) stc<T>(rows + (pl * Q + v) * RS + l, v == 0 ? Z[v] : cmul(Z[v], w[v]));
  }
  cluster_barrier<C>();

  // Column stage F2 (per v of this CTA): DFT_P over p of slot p*Q + v (any
  // CTA) -> X[Q u + v] -> global; the packed column 0 goes to CTA 0's scratch.
  // A thread's last batch of items is stored to global memory after it has
  // arrived at the final cluster barrier, so the arrive does not wait for
  // those stores to drain (with one batch per thread, the common case, no
  // global store precedes the arrive).
  constexpr int TF2 = H * QC;
  constexpr int BF = TF2 >= 2 * NT ? 2 : 1;
  auto f2_transform = [&](int it0, cx<T> (&X)[BF][P]) {
#pragma unroll
    for (int b = 0; b < BF; ++b) {
      const int it = it0 + b * NT;
      if (it < TF2) {
        const int l = it % H;
        const int v = int(rank) * QC + it / H;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          const int off = ((p % PC) * Q + v) * RS + l;
          if constexpr (C == 1) X[b][p] = ldc<T>(rows + off);
          else X[b][p] = ld_dsmem(rbase[p / PC] + uint32_t(off) * kEl, T(0));
        }
      }
    }
#pragma unroll
    for (int b = 0; b < BF; ++b) {
      const int it = it0 + b * NT;
      if (it >= TF2) continue;
      const int v = int(rank) * QC + it / H;
      Dft<P, -1, T>::run(X[b]);
      if (it % H == 0) {
#pragma unroll
        for (int u = 0; u < P; ++u) {
          if constexpr (C == 1) stc<T>(col0 + Q * u + v, X[b][u]);
          else st_dsmem(col0_r0 + uint32_t(Q * u + v) * kEl, X[b][u]);
        }
      }
    }
  };
  auto f2_store = [&](int it0, const cx<T> (&X)[BF][P]) {
#pragma unroll
    for (int b = 0; b < BF; ++b) {
      const int it = it0 + b * NT;
      if (it >= TF2 || it % H == 0) continue;
      const int l = it % H;
      const int v = int(rank) * QC + it / H;
#pragma unroll
      for (int u = 0; u < P; ++u) stc<T>(mainp + size_t(Q * u + v) * H + l, X[b][u]);
    }
  };
  int it0 = threadIdx.x;
  for (; it0 + BF * NT < TF2; it0 += BF * NT) {
    cx<T> X[BF][P];
    f2_transform(it0, X);
    f2_store(it0, X);
  }
  {
    cx<T> X[BF][P];
    const bool last = it0 < TF2;
    if (last) f2_transform(it0, X);
    cluster_arrive<C>();
    if (last) f2_store(it0, X);
  }
  cluster_wait<C>();

  // Unpack column 0: F = A + i B with A (kz = 0) and B (kz = n/2) Hermitian in ky.
  if (rank == 0) {
    for (int ky = threadIdx.x; ky < N; ky += NT) {
      const cx<T> f = ldc<T>(col0 + ky);
      const cx<T> g = cconj(ldc<T>(col0 + (N - ky) % N));
      const T h = T(0.5);
      stc<T>(mainp + size_t(ky) * H, cscale(cadd(f, g), h));
      stc<T>(nyqp + ky, cmul_i<-1>(cscale(csub(f, g), h)));
    }
  }
}

template <typename T, int N, int C, int MODE, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) pass_yz_kernel(const __grid_constant__ LaunchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_yz_unit<T, N, C, MODE, NT>(a, int(blockIdx.x) / C, smem_raw);
}

}  // namespace mg
