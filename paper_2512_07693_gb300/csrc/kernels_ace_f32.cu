// float instantiation of the body-order-4 ACE kernel (ace_pool.cuh).
#include "apip_internal.h"

namespace apip {
namespace {
__constant__ float c_norm[(kLmaxCap + 1) * (kLmaxCap + 1)];
struct Consts {
  static __device__ __forceinline__ float ynorm(int k) { return c_norm[k]; }
};
}  // namespace
}  // namespace apip

#include "ace_pool.cuh"

namespace apip {

template <> cudaError_t ace_pool_set_norms<float>(const double* norms, int count) {
  float f[(kLmaxCap + 1) * (kLmaxCap + 1)];
  for (int k = 0; k < count; ++k) f[k] = (float)norms[k];
  return cudaMemcpyToSymbol(c_norm, f, sizeof(float) * count);
}

template <> void launch_ace_pool<float>(const Args<float>& a, const AceDev<float>& t, int blocks, cudaStream_t s) {
  pool_dispatch<float, Consts>(&a, t, blocks, s, false);
}

template <> int ace_pool_occupancy<float>(const AceDev<float>& t) {
  return pool_dispatch<float, Consts>(nullptr, t, 0, nullptr, true);
}

}  // namespace apip
