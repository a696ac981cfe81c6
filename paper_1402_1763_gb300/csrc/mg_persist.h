// Parameters of the persistent one-launch sweep (mg_persist.cu).
#pragma once
#include <cuda_runtime.h>

#include "mg_device.cuh"

namespace mg {

constexpr int kMaxPersistClasses = 6;

// Grid sizes the persistent kernel covers (pass YZ without clusters).
bool persist_supports(int n);

template <typename T>
struct PersistArgs {
  LaunchArgs<T> cls[kMaxPersistClasses];  // one per grid size, <= kMaxLaunchChains chains each
  int n[kMaxPersistClasses];
  int tiles[kMaxPersistClasses];
  int ctx_chain[kMaxPersistClasses][kMaxLaunchChains];  // context chain index of each class chain
  int yz_begin[kMaxPersistClasses + 1];                 // queue ranges of the y/z planes per class
  int x_begin[kMaxPersistClasses + 1];                  // queue ranges of the x tiles per class
  int draw_begin;                                       // then one shell draw per chain
  int total;
  int ncls;
  int n_chains_total;
  int fix_P;
  long long timeout;       // cycle budget of each wait
  unsigned* ctr;           // [2 + 2 n_chains_total]: queue head, draws done, y/z done, x done
  const DrawDev* draw;     // indexed by context chain
  int* status;
  uint32_t* sweep_ctr;
};

template <typename T>
cudaError_t launch_persistent(const PersistArgs<T>& a, int B_max, int grid, cudaStream_t st);
template <typename T>
int persist_grid(const PersistArgs<T>& a, int B_max);

}  // namespace mg
