// mg_fp64_fma_peak: the FP64 fused multiply-add throughput of the current
// device, measured with CUDA events (declared in include/mg.h).  The FP64
// sweep is bound by the FP64 pipe rather than by HBM (GB300's FP64 rate is a
// small fraction of its FP32 rate), so its roofline denominator is this rate.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/mg.h"

namespace mg {
void set_thread_error(const char* msg);
}

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hide the pipe latency)

__global__ void __launch_bounds__(256) dfma_kernel(double* out, double a, double b, int iters) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  out[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

mg_status cuda_fail(const char* what, cudaError_t e) {
  const std::string msg = std::string("mg_fp64_fma_peak: ") + what + ": " + cudaGetErrorString(e);
  mg::set_thread_error(msg.c_str());
  return MG_ECUDA;
}

}  // namespace

extern "C" mg_status mg_fp64_fma_peak(double* gflops, void* stream) {
  if (!gflops) {
    mg::set_thread_error("mg_fp64_fma_peak: null output");
    return MG_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail("device query", e);
  const int threads = 256, blocks = sms * 8, iters = 4000;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status status = MG_OK;
  float best = 0.f;
  e = cudaMalloc(&out, size_t(blocks) * threads * sizeof(double));
  if (e != cudaSuccess) return cuda_fail("cudaMalloc", e);
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    status = cuda_fail("cudaEventCreate", e);
  } else {
    dfma_kernel<<<blocks, threads, 0, st>>>(out, 1.0000001, 1e-9, iters / 10);  // warm-up
    for (int rep = 0; rep < 3 && status == MG_OK; ++rep) {
      cudaEventRecord(e0, st);
      dfma_kernel<<<blocks, threads, 0, st>>>(out, 1.0000001, 1e-9, iters);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
          (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        status = cuda_fail("timed launch", e);
        break;
      }
      if (rep == 0 || ms < best) best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (status != MG_OK) return status;
  const double flops = 2.0 * kChains * double(blocks) * threads * iters;
  *gflops = flops / (double(best) * 1e-3) / 1e9;
  return MG_OK;
}
