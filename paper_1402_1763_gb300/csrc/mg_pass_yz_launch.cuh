// Launcher of pass YZ for one precision (included by mg_pass_yz_f32.cu and
// mg_pass_yz_f64.cu so the two precisions compile in parallel).
#pragma once
#include "mg_launch.h"
#include "mg_pass_yz.cuh"

namespace mg {
namespace yzimpl {

template <int N>
constexpr int yz_threads() {
  return N >= 128 ? 512 : (N >= 48 ? 256 : 128);
}

template <typename T, int N, int C, int MODE>
cudaError_t run(const ChainDev<T>* d_chains, int n_chains, const uint32_t* d_sweep, const void* tw,
                cudaStream_t st) {
  constexpr int NT = yz_threads<N>();
  using S = PassYZShape<T, N, C>;
  auto kern = pass_yz_kernel<T, N, C, MODE, NT>;
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
  return cudaLaunchKernelEx(&cfg, kern, d_chains, n_chains, d_sweep,
                            static_cast<const typename VT<T>::c2*>(tw));
}

template <typename T, int N, int C>
cudaError_t run_mode(int mode, const ChainDev<T>* d_chains, int n_chains, const uint32_t* d_sweep,
                     const void* tw, cudaStream_t st) {
  switch (mode) {
    case kModeSweep:
      return run<T, N, C, kModeSweep>(d_chains, n_chains, d_sweep, tw, st);
    case kModeMaterialize:
      return run<T, N, C, kModeMaterialize>(d_chains, n_chains, d_sweep, tw, st);
    case kModeLoad:
      return run<T, N, C, kModeLoad>(d_chains, n_chains, d_sweep, tw, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace yzimpl
}  // namespace mg
