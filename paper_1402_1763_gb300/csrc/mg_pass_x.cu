// Instantiations and launcher of pass X (see mg_pass_x.cuh).
#include "mg_launch.h"
#include "mg_pass_x.cuh"

namespace mg {

namespace {
template <int N>
constexpr int pass_x_threads() {
  // threads per CTA: 32 pencils x (threads per pencil)
  return N >= 128 ? 256 : (N >= 32 ? 128 : 64);
}
// resident CTAs per SM the register budget is sized for (FP32 tiles are small
// enough in shared memory for three)
template <typename T, int N>
constexpr int pass_x_minblocks() {
  return (sizeof(T) == 4 && N >= 128) ? 3 : 1;
}

template <typename T, int N, int MODE>
cudaError_t run_x(const LaunchArgs<T>& args_in, int B_max, cudaStream_t st) {
  const int n_chains = args_in.n_chains;
  constexpr int NT = pass_x_threads<N>();
  using S = PassXShape<T, N>;
  constexpr bool adj = MODE == kXAdjTop || MODE == kXAdjMid;
  const size_t smem = S::smem_bytes(NT / 32, B_max, adj);
  auto kern = pass_x_kernel<T, N, NT, adj ? 1 : pass_x_minblocks<T, N>(), MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess || n_chains == 0) return e;  // n_chains == 0: set attributes only
  // Prefetch distance: one CTA per SM ahead in launch order.  A whole
  // resident wave ahead (3 CTAs per SM) let L2 evict about a quarter of the
  // prefetched lines before use (23 % more DRAM reads); a third of a wave
  // keeps DRAM reads at the algorithmic bytes.
  LaunchArgs<T> args = args_in;
  args.pf_units = sm_count();
  const unsigned grid = unsigned(S::kTiles) * unsigned(n_chains);
  kern<<<grid, NT, smem, st>>>(args);
  return cudaGetLastError();
}
}  // namespace

int pass_x_tiles(int n) {
  const int lw = 32;
  return (n * (n / 2) + lw - 1) / lw + (n + lw - 1) / lw;
}

template <typename T, int N>
cudaError_t run_x_mode(int mode, const LaunchArgs<T>& args, int B_max, cudaStream_t st) {
  switch (mode) {
    case kXSweep:
      return run_x<T, N, kXSweep>(args, B_max, st);
    case kXAdjTop:
      return run_x<T, N, kXAdjTop>(args, B_max, st);
    case kXAdjMid:
      return run_x<T, N, kXAdjMid>(args, B_max, st);
    case kXMixDraw:
      return run_x<T, N, kXMixDraw>(args, B_max, st);
    case kXMixScale:
      return run_x<T, N, kXMixScale>(args, B_max, st);
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_pass_x(int n, int mode, const LaunchArgs<T>& args, int B_max, cudaStream_t st) {
  switch (n) {
#define MG_CASE(N_) \
  case N_:          \
    return run_x_mode<T, N_>(mode, args, B_max, st);
    MG_CASE(8)
    MG_CASE(12)
    MG_CASE(16)
    MG_CASE(24)
    MG_CASE(32)
#if MG_MAX_N >= 48
    MG_CASE(48)
#endif
#if MG_MAX_N >= 64
    MG_CASE(64)
#endif
#if MG_MAX_N >= 96
    MG_CASE(96)
#endif
#if MG_MAX_N >= 128
    MG_CASE(128)
#endif
#if MG_MAX_N >= 192
    MG_CASE(192)
#endif
#if MG_MAX_N >= 256
    MG_CASE(256)
#endif
#undef MG_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_pass_x<float>(int, int, const LaunchArgs<float>&, int, cudaStream_t);
template cudaError_t launch_pass_x<double>(int, int, const LaunchArgs<double>&, int, cudaStream_t);

}  // namespace mg
