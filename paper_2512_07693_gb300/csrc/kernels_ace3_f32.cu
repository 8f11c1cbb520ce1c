// float instantiation of the body-order <= 3 ACE kernel (ace_stream.cuh).
#include <vector>

#include "apip_internal.h"
#include "gaunt_layout.h"

namespace apip {
namespace {
__constant__ float c_norm[(kLmaxCap + 1) * (kLmaxCap + 1)];
__constant__ float c_gaunt[kGauntTotal];
struct Consts {
  static __device__ __forceinline__ float ynorm(int k) { return c_norm[k]; }
  static __device__ __forceinline__ float gaunt(int e) { return c_gaunt[e]; }
};
}  // namespace
}  // namespace apip

#include "ace_stream.cuh"

namespace apip {

template <> cudaError_t ace_stream_set_consts<float>(const double* norms, int count, const double* gaunt) {
  std::vector<float> f(norms, norms + count), gv(gaunt, gaunt + kGauntTotal);
  const cudaError_t e = cudaMemcpyToSymbol(c_norm, f.data(), sizeof(float) * count);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_gaunt, gv.data(), sizeof(float) * kGauntTotal);
}

template <> void launch_ace_stream<float>(const Args<float>& a, const AceDev<float>& t, int blocks, cudaStream_t s) {
  stream_dispatch<float, Consts>(&a, t, blocks, s, false);
}

template <> int ace_stream_occupancy<float>(const AceDev<float>& t) {
  return stream_dispatch<float, Consts>(nullptr, t, 0, nullptr, true);
}

}  // namespace apip
