// Host-side launchers of the sweep kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mg_device.cuh"

namespace mg {

// Grid sizes the kernels are compiled for: n = 2^a 3^b, 8 <= n <= 256, n % 4 == 0.
bool supported_n(int n);

// Pass YZ cluster sizes compiled for (n, precision); the first is the default.
int yz_cluster_choices(int n, int precision, int* out, int max_out);
size_t yz_smem_bytes(int n, int C, int precision);

// Multiprocessors of the current device (0 if the query fails): how far
// ahead in launch order pass X prefetches a tile's input into L2.
inline int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// n_chains == 0 only sets the kernels' attributes (done once, outside any
// stream capture).
template <typename T>
cudaError_t launch_pass_yz(int n, int C, int mode, const LaunchArgs<T>& args, cudaStream_t st);

int pass_x_tiles(int n);

enum PassXMode : int {
  kXSweep = 0,     // forward x FFT, signal draw, shell sums, inverse x FFT
  kXAdjTop = 1,    // adjoint of the last sweep: loss from the final state, gradient terms
  kXAdjMid = 2,    // adjoint of an earlier sweep
  kXMixDraw = 3,   // mixing sweep: forward x FFT, draw y = x sqrt(S/M), the sums of
                   // w |y|^2 and w Re(conj(y) F); the modes stay in k space
  kXMixScale = 4,  // mixing sweep: scale each mode by sqrt(S_new/S_old) of its shell,
                   // inverse x FFT
};
template <typename T>
cudaError_t launch_pass_x(int n, int mode, const LaunchArgs<T>& args, int B_max, cudaStream_t st);

}  // namespace mg
