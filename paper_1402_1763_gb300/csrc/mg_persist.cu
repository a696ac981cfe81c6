// One persistent launch per sweep for batches of chains of uneven grid sizes.
//
// Sec. 3.4 of the paper runs independent chains side by side.  Here every
// chain of every grid size advances by one sweep inside a single kernel: CTAs
// take work units from an in-order queue —
//   [pass YZ units of every chain] [pass X tiles of every chain] [shell draws]
// — and a unit waits (bounded spin) until the units it depends on for the same
// chain are done: an x tile waits for all y/z planes of its chain, a shell draw
// for all x tiles of its chain.  Because units are dequeued in order and
// dependencies point to earlier units, every awaited unit is already held by a
// running CTA, so the queue cannot deadlock.  A wait that exceeds its cycle
// budget sets the timeout status bit, skips its unit's work and still marks
// the unit done, so no other wait depends on it forever.
#include "mg_launch.h"
#include "mg_pass_x.cuh"
#include "mg_pass_yz.cuh"
#include "mg_persist.h"

#include <algorithm>

namespace mg {

namespace {

constexpr int kPersistThreads = 256;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 spins until *p >= target or the budget runs out; the whole CTA
// learns the outcome.  Returns false on timeout (status bit set).
__device__ bool wait_for(const unsigned* p, unsigned target, long long budget, int* status, int* flag) {
  if (threadIdx.x == 0) {
    const long long t0 = clock64();
    int ok = 1;
    while (ld_acquire(p) < target) {
      if (clock64() - t0 > budget) {
        atomicOr(status, kStTimeout);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    *flag = ok;
  }
  __syncthreads();
  const bool ok = *flag != 0;
  __syncthreads();
  return ok;
}

// Publish a finished unit: every thread's writes are fenced at GPU scope
// before thread 0 bumps the counter other CTAs wait on.
__device__ __forceinline__ void mark_done(unsigned* p) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(p, 1u);
}

// Shell draw of one chain by one CTA: per shell, the tiles' partials are split
// over thread groups in a fixed way and combined in a fixed order.
template <typename T>
__device__ void draw_chain(const DrawDev& cd, int fix_P, int* status, double* red, uint32_t sweep) {
  const int B1 = cd.B + 1;
  const int groups = kPersistThreads / B1;  // >= 1 since B1 <= 255 < 256
  const int b = threadIdx.x % B1, g = threadIdx.x / B1;
  double s1 = 0.0;
  if (g < groups) {
    for (int t = g; t < cd.n_tiles; t += groups)
      s1 += __ldcg(cd.partial + (size_t(t) * B1 + b) * 2 + 0);  // written by other SMs this launch
    red[g * B1 + b] = s1;
  }
  __syncthreads();
  if (threadIdx.x < B1) {
    double sig = 0.0;
    for (int k = 0; k < groups; ++k) sig += red[k * B1 + threadIdx.x];
    sig *= cd.M;  // pass X sums w |s_hat|^2 / M
    const int bb = threadIdx.x;
    double P = cd.P[bb];
    double chi = 0.0;
    if (!fix_P && cd.n_b[bb] > 0) {
      chi = chi2_shell(cd.n_b[bb], uint32_t(bb), sweep, cd.cid, cd.k0, cd.k1);  // Alg. 2 on shells
      if (sig > 0.0 && chi > 0.0 && isfinite(sig) && isfinite(chi)) P = (cd.V / cd.M) * sig / chi;
      else atomicOr(status, kStNumeric);
    }
    cd.sig_last[bb] = sig;
    cd.chi_last[bb] = chi;
    cd.P[bb] = P;
    const double Sh = (cd.M / cd.V) * P;
    const double a = Sh / (Sh + cd.tau);
    const double sd = sqrt(Sh * cd.tau / (Sh + cd.tau));
    typename VT<T>::c2* coef = static_cast<typename VT<T>::c2*>(cd.coef);
    typename VT<T>::c2 v;
    v.x = T(a / cd.M);
    v.y = T(sd / sqrt(cd.M));
    coef[bb] = v;
    if (bb == 0) {
      v.x = T(0);
      v.y = T(0);
      coef[cd.B + 1] = v;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void run_yz(const PersistArgs<T>& a, int k, int local, unsigned char* smem) {
  switch (a.n[k]) {
#define MG_P(N_) \
  case N_:       \
    pass_yz_unit<T, N_, 1, kModeSweep, kPersistThreads>(a.cls[k], local, smem); \
    break;
    MG_P(16)
    MG_P(24)
    MG_P(32)
#if MG_MAX_N >= 48
    MG_P(48)
#endif
#if MG_MAX_N >= 64
    MG_P(64)
#endif
#if MG_MAX_N >= 96
    MG_P(96)
#endif
#if MG_MAX_N >= 128
    MG_P(128)
#endif
#undef MG_P
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void run_x(const PersistArgs<T>& a, int k, int local, unsigned char* smem) {
  switch (a.n[k]) {
#define MG_P(N_) \
  case N_:       \
    pass_x_tile<T, N_, kPersistThreads, kXSweep>(a.cls[k], local, smem); \
    break;
    MG_P(16)
    MG_P(24)
    MG_P(32)
#if MG_MAX_N >= 48
    MG_P(48)
#endif
#if MG_MAX_N >= 64
    MG_P(64)
#endif
#if MG_MAX_N >= 96
    MG_P(96)
#endif
#if MG_MAX_N >= 128
    MG_P(128)
#endif
#undef MG_P
    default:
      break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kPersistThreads, 2) persistent_sweep_kernel(const __grid_constant__ PersistArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_unit, s_flag;
  __shared__ double s_red[kPersistThreads * 2];
  unsigned* next = a.ctr;
  unsigned* draws_done = a.ctr + 1;
  unsigned* yz_done = a.ctr + 2;
  unsigned* x_done = a.ctr + 2 + a.n_chains_total;
  for (;;) {
    __syncthreads();  // the previous unit is finished with shared memory
    if (threadIdx.x == 0) s_unit = int(atomicAdd(next, 1u));
    __syncthreads();
    const int u = s_unit;
    if (u >= a.total) break;
    if (u < a.x_begin[0]) {  // pass YZ unit
      int k = 0;
      while (u >= a.yz_begin[k + 1]) ++k;
      const int local = u - a.yz_begin[k];
      run_yz<T>(a, k, local, smem_raw);
      mark_done(yz_done + a.ctx_chain[k][local % a.cls[k].n_chains]);
    } else if (u < a.draw_begin) {  // pass X tile
      int k = 0;
      while (u >= a.x_begin[k + 1]) ++k;
      const int local = u - a.x_begin[k];
      const int gc = a.ctx_chain[k][local / a.tiles[k]];
      if (wait_for(yz_done + gc, unsigned(a.n[k]), a.timeout, a.status, &s_flag)) run_x<T>(a, k, local, smem_raw);
      mark_done(x_done + gc);
    } else {  // shell draw of one chain
      const int gc = u - a.draw_begin;
      const DrawDev cd = a.draw[gc];
      if (wait_for(x_done + gc, unsigned(cd.n_tiles), a.timeout, a.status, &s_flag))
        draw_chain<T>(cd, a.fix_P, a.status, s_red, __ldcg(a.sweep_ctr));  // advanced only after every draw
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        if (atomicAdd(draws_done, 1u) + 1u == unsigned(a.n_chains_total)) atomicAdd(a.sweep_ctr, 1u);
      }
    }
  }
}

template <typename T>
size_t smem_needed(int n, int B_max) {
  constexpr int NW = kPersistThreads / 32;
  switch (n) {
#define MG_P(N_) \
  case N_:       \
    return std::max(PassYZShape<T, N_, 1>::kSmemBytes, PassXShape<T, N_>::smem_bytes(NW, B_max));
    MG_P(16)
    MG_P(24)
    MG_P(32)
#if MG_MAX_N >= 48
    MG_P(48)
#endif
#if MG_MAX_N >= 64
    MG_P(64)
#endif
#if MG_MAX_N >= 96
    MG_P(96)
#endif
#if MG_MAX_N >= 128
    MG_P(128)
#endif
#undef MG_P
    default:
      return 0;
  }
}

}  // namespace

bool persist_supports(int n) {
  return n <= MG_MAX_N && (n == 16 || n == 24 || n == 32 || n == 48 || n == 64 || n == 96 || n == 128);
}

template <typename T>
size_t persist_smem(const PersistArgs<T>& a, int B_max) {
  size_t s = 0;
  for (int k = 0; k < a.ncls; ++k) s = std::max(s, smem_needed<T>(a.n[k], B_max));
  return s;
}

template <typename T>
cudaError_t launch_persistent(const PersistArgs<T>& a, int B_max, int grid, cudaStream_t st) {
  const size_t smem = persist_smem(a, B_max);
  cudaError_t e = cudaFuncSetAttribute(persistent_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess || grid == 0) return e;
  persistent_sweep_kernel<T><<<grid, kPersistThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
int persist_grid(const PersistArgs<T>& a, int B_max) {
  const size_t smem = persist_smem(a, B_max);
  if (cudaFuncSetAttribute(persistent_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
      cudaSuccess)
    return 0;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_sweep_kernel<T>, kPersistThreads, smem) !=
      cudaSuccess)
    return 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return per_sm * sms;
}

template cudaError_t launch_persistent<float>(const PersistArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_persistent<double>(const PersistArgs<double>&, int, int, cudaStream_t);
template int persist_grid<float>(const PersistArgs<float>&, int);
template int persist_grid<double>(const PersistArgs<double>&, int);

}  // namespace mg
