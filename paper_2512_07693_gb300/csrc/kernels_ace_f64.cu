// float64 instantiation of the ACE kernels (the parity path).
#include "apip_internal.h"

namespace apip {
__constant__ double c_norm_d[(kLmaxCap + 1) * (kLmaxCap + 1)];
}  // namespace apip

#include "ace_device.cuh"

namespace apip {

template <> __device__ __forceinline__ double ynorm<double>(int k) { return c_norm_d[k]; }

template <> void ace_set_norms<double>(const double* norms, int count) {
  cudaMemcpyToSymbol(c_norm_d, norms, sizeof(double) * count);
}

template <> void launch_ace<double>(const Args<double>& a, const AceDev<double>& t, int blocks, cudaStream_t s) {
  launch_ace_impl<double>(a, t, blocks, s);
}

template <> int ace_occupancy<double>(int l_max, int group, int npool, size_t* smem_bytes) {
  return ace_occupancy_impl<double>(l_max, group, npool, smem_bytes);
}

}  // namespace apip
