// mg_shell_sums_noalloc: the k-shell sums of a given spectrum without any
// device allocation (declared in include/mg.h).
//
// Some callers cannot allocate device memory at the point where they need the
// shell power of a sample: code running under a memory-pool budget that is
// already spent, real-time pipelines that forbid allocation (and its implicit
// synchronisation) after start-up, or host code sitting between kernels it does
// not own.  This entry point computes sigma_b = sum_{k in b} w_k |s_hat_k|^2 and
// n_b = sum_{k in b} w_k over the stored modes of a half-complex spectrum, like
// the shell sums inside the sweep, but keeps its per-block partial sums in the
// file-scope array below instead of a buffer the library allocates.
//
// Every sum is formed in a fixed order (segmented warp sums, per-warp running
// sums in lane order, warps and then blocks combined in index order), so two
// calls on the same input give the same bits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/mg.h"

namespace mg {
void set_thread_error(const char* msg);  // mg_api.cu: text for mg_last_error(NULL)
}

namespace {

// Fixed scratch: kNoallocBlocks blocks x (n_bins + 1) shells x 2 values.
constexpr int kNoallocBlocks = 256;
constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxShells = 255;  // n_bins + 1 <= 255
constexpr size_t kNoallocScratchDoubles = size_t(kNoallocBlocks) * kNoallocMaxShells * 2;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];  // 1,044,480 bytes

// Shell of a mode with integer |m|^2 = m2 for n_bins linear shells on
// [0, k_Nyq): the largest b with b^2 h^2 <= B^2 m2 (ties to the upper shell),
// B (overflow) past the last edge.
__device__ __forceinline__ int linear_shell(unsigned long long m2, int B, int h) {
  const unsigned long long t = (unsigned long long)B * B * m2;
  unsigned long long q = (unsigned long long)sqrt(double(t));
  while (q * q > t) --q;
  while ((q + 1) * (q + 1) <= t) ++q;
  const int b = int(q / (unsigned long long)h);
  return b >= B ? B : b;
}

// One warp's 32 consecutive modes: sums of (sg, wt) over runs of equal shell
// id (fixed shuffle tree), then each run head adds its run to this warp's
// running sums acc[b][2].  With non-decreasing ids along the warp the heads hold
// distinct shells and add in parallel; otherwise (a row boundary inside the
// warp) they add one after another in lane order.
__device__ __forceinline__ void warp_shell_add(double sg, double wt, int b, double* acc, int lane) {
  const unsigned full = 0xffffffffu;
  const int prevb = __shfl_up_sync(full, b, 1);
  const bool head = (lane == 0) || (prevb != b);
  const unsigned heads = __ballot_sync(full, head);
  const bool monotone = __all_sync(full, lane == 0 || prevb <= b);
  const unsigned later = (lane == 31) ? 0u : (heads & (full << (lane + 1)));
  const int run_end = later ? (__ffs(later) - 2) : 31;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double o1 = __shfl_down_sync(full, sg, off);
    const double o2 = __shfl_down_sync(full, wt, off);
    if (lane + off <= run_end) {
      sg += o1;
      wt += o2;
    }
  }
  const bool writer = head && b >= 0;
  if (monotone) {
    if (writer) {
      acc[2 * b + 0] += sg;
      acc[2 * b + 1] += wt;
    }
  } else {
    unsigned hm = __ballot_sync(full, writer);
    while (hm) {
      const int src = __ffs(hm) - 1;
      if (lane == src) {
        acc[2 * b + 0] += sg;
        acc[2 * b + 1] += wt;
      }
      __syncwarp();
      hm &= hm - 1;
    }
  }
}

template <typename C2>
__global__ void __launch_bounds__(kNoallocThreads) shell_partials_kernel(const C2* __restrict__ s_hat, int n, int B,
                                                                         double* __restrict__ scratch) {
  constexpr int NW = kNoallocThreads / 32;
  const int h = n / 2;
  const int B1 = B + 1;
  const size_t Mh = size_t(n) * n * (h + 1);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  extern __shared__ double acc[];  // [NW][B1][2] per-warp running sums
  for (int i = threadIdx.x; i < NW * 2 * B1; i += kNoallocThreads) acc[i] = 0.0;
  __syncthreads();
  double* accw = acc + size_t(warp) * 2 * B1;
  const size_t stride = size_t(gridDim.x) * kNoallocThreads;
  // j0 is the same for the whole warp, so every lane takes part in the shuffles
  for (size_t j0 = size_t(blockIdx.x) * kNoallocThreads + size_t(warp) * 32; j0 < Mh; j0 += stride) {
    const size_t j = j0 + lane;
    int b = -1;
    double sg = 0.0, wt = 0.0;
    if (j < Mh) {
      const int kz = int(j % (h + 1));
      const int ky = int((j / (h + 1)) % n);
      const int kx = int(j / (size_t(h + 1) * n));
      const int mx = kx <= h ? kx : kx - n, my = ky <= h ? ky : ky - n;
      const unsigned long long m2 = (unsigned long long)(mx * mx + my * my + kz * kz);
      if (m2 != 0) {  // the DC mode belongs to no shell
        b = linear_shell(m2, B, h);
        const double w = (kz == 0 || kz == h) ? 1.0 : 2.0;
        const double re = double(s_hat[j].x), im = double(s_hat[j].y);
        sg = w * (re * re + im * im);
        wt = w;
      }
    }
    warp_shell_add(sg, wt, b, accw, lane);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < B1; b += kNoallocThreads) {
    double s = 0.0, c = 0.0;
    for (int w = 0; w < NW; ++w) {
      s += acc[(size_t(w) * B1 + b) * 2 + 0];
      c += acc[(size_t(w) * B1 + b) * 2 + 1];
    }
    scratch[(size_t(blockIdx.x) * B1 + b) * 2 + 0] = s;
    scratch[(size_t(blockIdx.x) * B1 + b) * 2 + 1] = c;
  }
}

__global__ void shell_combine_kernel(const double* __restrict__ scratch, int B, double* __restrict__ sigma,
                                     double* __restrict__ nmodes) {
  const int B1 = B + 1;
  for (int b = threadIdx.x; b < B1; b += blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < kNoallocBlocks; ++k) {
      s += scratch[(size_t(k) * B1 + b) * 2 + 0];
      c += scratch[(size_t(k) * B1 + b) * 2 + 1];
    }
    sigma[b] = s;
    if (nmodes) nmodes[b] = c;
  }
}

// The scratch array's device address is looked up (cudaGetSymbolAddress, with
// the device current) once per CUDA context and kept: a new context on the
// same device (after cudaDeviceReset) gets a fresh lookup, and a failed lookup
// is not kept, so a later call tries again.  The context is identified by the
// driver's unique context id, reached through the runtime's driver entry
// points (no link against the driver library).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long g_ctx_id[kMaxDevices];  // 0: nothing cached
double* g_scratch_ptr[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the current context, or 0 if it cannot be had.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  unsigned long long id = 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  // makes the device's primary context current if no context is yet
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) return e;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (id != 0 && g_ctx_id[dev] == id) {
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_ctx_id[dev] = id;  // id 0 (no context id available): looked up again next call
  g_scratch_ptr[dev] = static_cast<double*>(p);
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

void cuda_error_text(const char* what, cudaError_t e) {
  const std::string msg = std::string("mg_shell_sums_noalloc: ") + what + ": " + cudaGetErrorString(e);
  mg::set_thread_error(msg.c_str());  // copied
}

}  // namespace

extern "C" mg_status mg_shell_sums_noalloc(const void* s_hat, int32_t precision, int32_t n, int32_t n_bins,
                                           double* sigma_out, double* nmodes_out, void* stream) {
  if (!s_hat || !sigma_out) {
    mg::set_thread_error("mg_shell_sums_noalloc: null s_hat or sigma_out");
    return MG_EINVAL;
  }
  if (precision != 32 && precision != 64) {
    mg::set_thread_error("mg_shell_sums_noalloc: precision must be 32 or 64");
    return MG_EINVAL;
  }
  if (n < 4 || n % 2 != 0 || n > 4096) {
    mg::set_thread_error("mg_shell_sums_noalloc: n must be even, 4 <= n <= 4096");
    return MG_EINVAL;
  }
  if (n_bins < 1 || n_bins + 1 > kNoallocMaxShells) {
    mg::set_thread_error("mg_shell_sums_noalloc: n_bins must be 1..254 (the fixed scratch holds 255 shells)");
    return MG_EINVAL;
  }
  // an error left by earlier work on this thread is reported as such, not as
  // a failure of these launches
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    cuda_error_text("a CUDA error from earlier work is pending (nothing launched)", e);
    return MG_ECUDA;
  }
  double* scratch = nullptr;
  e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    cuda_error_text("cudaGetSymbolAddress of the scratch array failed", e);
    return MG_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = size_t(kNoallocThreads / 32) * 2 * (n_bins + 1) * sizeof(double);
  if (precision == 64)
    shell_partials_kernel<double2><<<kNoallocBlocks, kNoallocThreads, smem, st>>>(
        static_cast<const double2*>(s_hat), n, n_bins, scratch);
  else
    shell_partials_kernel<float2><<<kNoallocBlocks, kNoallocThreads, smem, st>>>(static_cast<const float2*>(s_hat),
                                                                                 n, n_bins, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_error_text("launch of the partial-sum kernel failed", e);
    return MG_ECUDA;
  }
  shell_combine_kernel<<<1, 256, 0, st>>>(scratch, n_bins, sigma_out, nmodes_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cuda_error_text("launch of the combining kernel failed", e);
    return MG_ECUDA;
  }
  return MG_OK;
}
