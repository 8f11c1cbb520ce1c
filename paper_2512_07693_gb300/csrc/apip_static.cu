// Allocation-free variant of the float64 energy reduction.
//
// apip_energy_forces reduces per-atom energies through block partials held in
// context memory that apip_create allocates.  apip_reduce_energy_static does the
// same compensated two-stage reduction of a caller's per-atom energy array, but
// its partials live in one file-scope __device__ array of fixed size, so the call
// allocates nothing.  It is meant for callers that cannot call cudaMalloc, for
// example a host program whose device memory is entirely owned by its own pool
// allocator, or a latency-critical loop that must never enter the allocator.
#include <cuda_runtime.h>

#include <mutex>

#include "apip.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerBlock = APIP_STATIC_ATOMS_PER_BLOCK;   // atoms reduced by one block
constexpr int kMaxBlocks = APIP_STATIC_MAX_BLOCKS;       // capacity of the scratch array

// Scratch: one float64 partial sum per block.  Every GPU that loads the library
// holds these kMaxBlocks * 8 bytes until the process exits.  Host code must not
// pass this name to a kernel: on the host it is only a stand-in for the symbol.
static __device__ __align__(256) double g_partials[kMaxBlocks];

__device__ __forceinline__ void neumaier(double& s, double& c, double v) {
  const double t = s + v;
  c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
  s = t;
}

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// Stage 1: block b sums e[b*kPerBlock, (b+1)*kPerBlock) into partials[b].
__global__ void k_partials(const double* __restrict__ e, int64_t n, double* partials) {
  __shared__ double sh[32];
  const int64_t base = (int64_t)blockIdx.x * kPerBlock;
  const int64_t end = base + kPerBlock < n ? base + kPerBlock : n;
  double s = 0.0, c = 0.0;
  for (int64_t k = base + threadIdx.x; k < end; k += blockDim.x) neumaier(s, c, e[k]);
  const double tot = block_sum(s, sh) + block_sum(c, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// Stage 2: one block sums partials[0, nb) into *out.  Only partials written by
// stage 1 of the same call are read, so nothing has to be cleared beforehand.
__global__ void k_total(const double* partials, int nb, double* out) {
  __shared__ double sh[32];
  double s = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) neumaier(s, c, partials[k]);
  const double tot = block_sum(s, sh) + block_sum(c, sh);
  if (threadIdx.x == 0) *out = tot;
}

// Device address of g_partials per device, looked up once with that device current.
// It belongs to the device's primary context and goes stale if that context is
// destroyed (cudaDeviceReset); the header documents the limit.
constexpr int kMaxDevices = 64;
double* g_addr[kMaxDevices] = {};
std::mutex g_mu;

apip_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return APIP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return APIP_ERR_CUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return APIP_OK;
}

}  // namespace

extern "C" apip_status apip_reduce_energy_static(const double* e_atom, int64_t n, double* e_total, void* stream) {
  if (!e_total || n < 0 || (n > 0 && !e_atom)) return APIP_ERR_ARG;
  if (n > APIP_STATIC_MAX_ATOMS) return APIP_ERR_SIZE;
  double* partials = nullptr;
  const apip_status st = scratch_for_current_device(&partials);
  if (st != APIP_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = n > 0 ? (int)((n + kPerBlock - 1) / kPerBlock) : 0;
  if (nb > 0) k_partials<<<nb, kThreads, 0, s>>>(e_atom, n, partials);
  k_total<<<1, kThreads, 0, s>>>(partials, nb, e_total);
  return cudaGetLastError() == cudaSuccess ? APIP_OK : APIP_ERR_CUDA;
}
