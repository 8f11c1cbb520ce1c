// Measured arithmetic peaks for the roofline of the ACE kernels (float32 pipe)
// and of the float64 path: a register-resident multiply-add loop on every SM,
// timed with CUDA events.  Changes no clock or power setting.
#include <cuda_runtime.h>

#include "apip.h"

namespace {

constexpr int kChains = 8;        // independent multiply-add chains per thread
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_loop(int iters, T seed, T* sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = seed + T(threadIdx.x + c);
  const T m = T(0.999999), b = T(1e-7);
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], m, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(-1) && sink) sink[blockIdx.x] = s;   // never true (every x stays positive); keeps the loop
}

// Device multiply-add rate of T in TFLOP/s (2 flops per multiply-add): the best
// of three launches of blocks_per_sm x SMs blocks.
template <typename T>
cudaError_t measure(int iters, int blocks_per_sm, cudaStream_t s, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * blocks_per_sm;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
  double best = 0.0;
  k_fma_loop<T><<<blocks, kThreads, 0, s>>>(iters / 8, T(1), nullptr);   // warm-up
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    cudaEventRecord(a, s);
    k_fma_loop<T><<<blocks, kThreads, 0, s>>>(iters, T(1), nullptr);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess && ms > 0.f) {
      const double fl = 2.0 * kChains * (double)iters * kThreads * (double)blocks;
      const double t = fl / (ms * 1e-3) / 1e12;
      if (t > best) best = t;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" apip_status apip_measure_peaks(double* fp32_tflops, double* fp64_tflops, void* stream) {
  if (!fp32_tflops || !fp64_tflops) return APIP_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // float32: 8 resident blocks of 256 threads per SM hide the multiply-add latency;
  // float64 runs at a small fraction of that rate, so fewer iterations suffice
  if (measure<float>(1 << 16, 8, s, fp32_tflops) != cudaSuccess) return APIP_ERR_CUDA;
  if (measure<double>(1 << 11, 8, s, fp64_tflops) != cudaSuccess) return APIP_ERR_CUDA;
  return APIP_OK;
}
