// Pass YZ instantiations, FP64.
#include "mg_pass_yz_launch.cuh"

namespace mg {

template <>
cudaError_t launch_pass_yz<double>(int n, int C, int mode, const LaunchArgs<double>& args, cudaStream_t st) {
  using namespace yzimpl;
#define MG_CASE(N_, C_) \
  if (n == N_ && C == C_) return run_mode<double, N_, C_>(mode, args, st);
  MG_CASE(8, 1)
  MG_CASE(12, 1)
  MG_CASE(16, 1)
  MG_CASE(24, 1)
  MG_CASE(32, 1)
#if MG_MAX_N >= 48
  MG_CASE(48, 1)
#endif
#if MG_MAX_N >= 64
  MG_CASE(64, 1)
#endif
#if MG_MAX_N >= 96
  MG_CASE(96, 1)
#endif
#if MG_MAX_N >= 128
  MG_CASE(128, 1)
#endif
#if MG_MAX_N >= 192
  MG_CASE(192, 2)
#endif
#if MG_MAX_N >= 256
  MG_CASE(256, 4)
#endif
#undef MG_CASE
  return cudaErrorInvalidValue;
}

}  // namespace mg
