// Launcher of pass YZ for one precision (included by mg_pass_yz_f32.cu and
// mg_pass_yz_f64.cu so the two precisions compile in parallel).
#pragma once
#include "mg_launch.h"
#include "mg_pass_yz.cuh"

namespace mg {
namespace yzimpl {

// Threads per CTA and the resident CTAs per SM the register budget targets:
// two CTAs per SM wherever two planes (or plane slices) fit in shared memory.
template <typename T, int N, int C>
constexpr int yz_minblocks() {
  return 2 * PassYZShape<T, N, C>::kSmemBytes <= 220 * 1024 ? 2 : 1;
}
template <typename T, int N, int C>
constexpr int yz_threads() {
  return N < 48 ? 128 : (yz_minblocks<T, N, C>() == 2 ? 256 : 512);
}

template <typename T, int N, int C, int MODE>
cudaError_t run(const LaunchArgs<T>& args, cudaStream_t st) {
  const int n_chains = args.n_chains;
  constexpr int NT = yz_threads<T, N, C>();
  using S = PassYZShape<T, N, C>;
  auto kern = pass_yz_kernel<T, N, C, MODE, NT, yz_minblocks<T, N, C>()>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::kSmemBytes));
  if (e != cudaSuccess || n_chains == 0) return e;  // n_chains == 0: set attributes only
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(C) * unsigned(N) * unsigned(n_chains), 1, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = S::kSmemBytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args);
}

template <typename T, int N, int C>
cudaError_t run_mode(int mode, const LaunchArgs<T>& args, cudaStream_t st) {
  switch (mode) {
    case kModeSweep:
      return run<T, N, C, kModeSweep>(args, st);
    case kModeMaterialize:
      return run<T, N, C, kModeMaterialize>(args, st);
    case kModeLoad:
      return run<T, N, C, kModeLoad>(args, st);
    case kModeAdjoint:
      return run<T, N, C, kModeAdjoint>(args, st);
    case kModeSweepRecord:
      return run<T, N, C, kModeSweepRecord>(args, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace yzimpl
}  // namespace mg
