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
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/mg.h"

namespace mg {
void set_thread_error(const char* msg);  // mg_api.cu: text for mg_last_error(NULL)
}

namespace {

// Fixed scratch: kNoallocBlocks blocks x (n_bins + 1) shells x 2 values.
constexpr int kNoallocBlocks = 256;
constexpr int kNoallocMaxShells = 255;  // n_bins + 1 <= 255
constexpr size_t kNoallocScratchDoubles = size_t(kNoallocBlocks) * kNoallocMaxShells * 2;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];  // 1,044,480 bytes

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
double* g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_err[kMaxDevices];

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

template <typename C2>
__global__ void shell_partials_kernel(const C2* __restrict__ s_hat, int n, int B, double* __restrict__ scratch) {
  const int h = n / 2;
  const int B1 = B + 1;
  const size_t Mh = size_t(n) * n * (h + 1);
  extern __shared__ double sm[];  // [B1][2] block partials
  for (int i = threadIdx.x; i < 2 * B1; i += blockDim.x) sm[i] = 0.0;
  __syncthreads();
  for (size_t j = blockIdx.x * size_t(blockDim.x) + threadIdx.x; j < Mh; j += size_t(gridDim.x) * blockDim.x) {
    const int kz = int(j % (h + 1));
    const int ky = int((j / (h + 1)) % n);
    const int kx = int(j / (size_t(h + 1) * n));
    const int mx = kx <= h ? kx : kx - n, my = ky <= h ? ky : ky - n;
    const unsigned long long m2 = (unsigned long long)(mx * mx + my * my + kz * kz);
    if (m2 == 0) continue;  // the DC mode belongs to no shell
    const int b = linear_shell(m2, B, h);
    const double w = (kz == 0 || kz == h) ? 1.0 : 2.0;
    const double re = double(s_hat[j].x), im = double(s_hat[j].y);
    // shared-memory atomics: order-dependent rounding only within one block's
    // running sums; the block totals are combined in a fixed order below
    atomicAdd(&sm[2 * b + 0], w * (re * re + im * im));
    atomicAdd(&sm[2 * b + 1], w);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * B1; i += blockDim.x) scratch[size_t(blockIdx.x) * 2 * B1 + i] = sm[i];
}

__global__ void shell_combine_kernel(const double* __restrict__ scratch, int B, double* __restrict__ sigma,
                                     double* __restrict__ nmodes) {
  const int B1 = B + 1;
  for (int b = threadIdx.x; b < B1; b += blockDim.x) {
    double s = 0.0, c = 0.0;
    for (int k = 0; k < kNoallocBlocks; ++k) {
      s += scratch[size_t(k) * 2 * B1 + 2 * b + 0];
      c += scratch[size_t(k) * 2 * B1 + 2 * b + 1];
    }
    sigma[b] = s;
    if (nmodes) nmodes[b] = c;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(g_once[dev], [dev] {
    void* p = nullptr;
    g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    g_scratch_ptr[dev] = static_cast<double*>(p);
  });
  if (g_scratch_err[dev] != cudaSuccess) return g_scratch_err[dev];
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
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
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) {
    mg::set_thread_error("mg_shell_sums_noalloc: cudaGetSymbolAddress of the scratch array failed");
    return MG_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t smem = size_t(2) * (n_bins + 1) * sizeof(double);
  if (precision == 64)
    shell_partials_kernel<double2><<<kNoallocBlocks, 256, smem, st>>>(static_cast<const double2*>(s_hat), n, n_bins,
                                                                       scratch);
  else
    shell_partials_kernel<float2><<<kNoallocBlocks, 256, smem, st>>>(static_cast<const float2*>(s_hat), n, n_bins,
                                                                      scratch);
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  shell_combine_kernel<<<1, 256, 0, st>>>(scratch, n_bins, sigma_out, nmodes_out);
  if (cudaGetLastError() != cudaSuccess) return MG_ECUDA;
  return MG_OK;
}
