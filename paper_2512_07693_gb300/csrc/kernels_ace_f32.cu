// float32 instantiation of the ACE kernels (pair arithmetic in float32 with
// compensated channel sums; forces accumulated in float64).
#include "apip_internal.h"

namespace apip {
__constant__ float c_norm_f[(kLmaxCap + 1) * (kLmaxCap + 1)];
}  // namespace apip

#include "ace_device.cuh"

namespace apip {

template <> __device__ __forceinline__ float ynorm<float>(int k) { return c_norm_f[k]; }

template <> void ace_set_norms<float>(const double* norms, int count) {
  float f[(kLmaxCap + 1) * (kLmaxCap + 1)];
  for (int k = 0; k < count; ++k) f[k] = (float)norms[k];
  cudaMemcpyToSymbol(c_norm_f, f, sizeof(float) * count);
}

template <> void launch_ace<float>(const Args<float>& a, const AceDev<float>& t, int blocks, cudaStream_t s) {
  launch_ace_impl<float>(a, t, blocks, s);
}

template <> int ace_occupancy<float>(int l_max, int group, int npool, size_t* smem_bytes) {
  return ace_occupancy_impl<float>(l_max, group, npool, smem_bytes);
}

}  // namespace apip
