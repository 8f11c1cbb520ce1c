// double instantiation of the body-order-4 ACE kernel (ace_pool.cuh).
#include "apip_internal.h"

namespace apip {
namespace {
__constant__ double c_norm[(kLmaxCap + 1) * (kLmaxCap + 1)];
struct Consts {
  static __device__ __forceinline__ double ynorm(int k) { return c_norm[k]; }
};
}  // namespace
}  // namespace apip

#include "ace_pool.cuh"

namespace apip {

template <> cudaError_t ace_pool_set_norms<double>(const double* norms, int count) {
  return cudaMemcpyToSymbol(c_norm, norms, sizeof(double) * count);
}

template <> void launch_ace_pool<double>(const Args<double>& a, const AceDev<double>& t, int blocks, cudaStream_t s) {
  pool_dispatch<double, Consts>(&a, t, blocks, s, false);
}

template <> int ace_pool_occupancy<double>(const AceDev<double>& t) {
  return pool_dispatch<double, Consts>(nullptr, t, 0, nullptr, true);
}

}  // namespace apip
