// Helpers of the fifth-generation tensor-core kernels (tcgen05.mma with
// accumulators in tensor memory, operands in shared memory): the "chunk-major"
// operand layout, shared-memory and instruction descriptors, MMA issue and
// commit, bounded mbarrier waits, tensor-memory loads and stores.
//
// Operand layout ("chunk-major", no swizzle): an operand with R rows (samples or
// atoms of a tile, or the 64 output rows of a weight matrix) is stored as
// 8-column chunks of R x 16 bytes, element (row, k) at (k / 8) * 16 R + 16 row +
// 2 (k % 8).  Read K-major (rows = M or N) its core matrices are 8 rows x 16
// bytes, the K-adjacent ones 16 R bytes apart (leading byte offset) and the
// 8-row groups 128 bytes apart (stride byte offset); read MN-major (rows = K) the
// 8-row groups along K are 128 bytes apart (leading byte offset) and the 8-column
// groups 16 R bytes apart (stride byte offset).  So a matrix written once, row by
// row, serves both as A (or B) and, transposed, as a gradient operand.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace apip {
namespace tc {

// element (row, k) of a chunk-major operand with `rows` rows
__host__ __device__ constexpr int chunk_off(int row, int k, int rows) {
  return (k >> 3) * (rows * 16) + row * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// An operand for the tensor cores: its shared-memory start, the leading and
// stride byte offsets of its descriptor, and the bytes to advance per K = 16.
struct Opnd {
  uint32_t addr, lbo, sbo, kstep;
};
// 128-sample operands: K-major (samples = M) and MN-major (samples = K)
__device__ __forceinline__ Opnd act_k(const unsigned char* p) { return {smem_u32(p), 2048u, 128u, 4096u}; }
__device__ __forceinline__ Opnd act_mn(const unsigned char* p) { return {smem_u32(p), 128u, 2048u, 256u}; }
// 64-row weights: K-major (forward) and MN-major (the transpose, back-propagation)
__device__ __forceinline__ Opnd wt_k(const unsigned char* p) { return {smem_u32(p), 1024u, 128u, 2048u}; }
__device__ __forceinline__ Opnd wt_mn(const unsigned char* p) { return {smem_u32(p), 128u, 1024u, 256u}; }

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets, the descriptor version of this tensor-core generation, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: float32 D, bfloat16 A and B, M = 128; bits
// 15 / 16 select an MN-major A / B.
__device__ __forceinline__ uint32_t idesc(int N, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D (tensor memory, column d) (+)= A B^T over K, in K = 16 steps (one thread).
__device__ __forceinline__ void mma(uint32_t tmem, uint32_t d, Opnd A, Opnd B, int K, uint32_t id, bool accumulate) {
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = sdesc(A.addr + kk * A.kstep, A.lbo, A.sbo), bd = sdesc(B.addr + kk * B.kstep, B.lbo, B.sbo);
    const uint32_t acc = (accumulate || kk > 0) ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + d),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  }
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the barrier phase with the given parity (two seconds).
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (now_ns() - t0 > 2000000000ull) return false;
  }
}

// 16 consecutive float32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tld16(uint32_t addr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// ... and the reverse: 16 float32 values into this thread's lane.
__device__ __forceinline__ void tst16(uint32_t addr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          addr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// The logistic function (hardware exponential and approximate division: a few
// ulp, far below the bfloat16 rounding of the GEMM operands it feeds).
__device__ __forceinline__ float sig(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

// Operands written by the threads are made visible to the tensor cores, and the
// threads' tensor-memory accesses are ordered before the next MMA.
__device__ __forceinline__ void to_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Eight consecutive float32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tld8(uint32_t addr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

}  // namespace tc
}  // namespace apip
