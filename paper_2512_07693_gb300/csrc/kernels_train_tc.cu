// Training of the learned indicator on the fifth-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory): one fused kernel per batch does
// the forward pass, the loss, the back-propagation and the weight gradients.
//
// The network (32 -> 64 -> 64 -> 64 -> 1, SiLU; inputs x0 = 0.25 G) is trained
// with bfloat16 GEMM operands and float32 accumulation: every matrix product
// takes its inputs (weights, activations, back-propagated gradients) rounded to
// bfloat16 and sums in float32; the elementwise steps (bias, SiLU and its
// derivative, the output layer's dot product, the loss) are float32, the
// pre-activations stay float32 in tensor memory, the master weights and Adam
// are float32.
//
// A CTA of 256 threads loops over 128-sample tiles: sample r of a tile is
// tensor-memory lane r, read by warp r / 32 (lanes) and warp r / 32 + 4, which
// take the first and the second half of each layer's 64 columns.  Per tile, with D = A B^T on the tensor
// cores (M = 128 rows of A, N rows of B, K the shared dimension):
//   z1 = x0 W1^T, z2 = h1 W2^T, z3 = h2 W3^T                (forward, M = samples)
//   dh2 = dz3 W3, dh1 = dz2 W2                              (back-propagation)
//   [dW3 | dW2 | db3 db2] += [dz3^T ; dz2^T] [h2^T ; h1^T ; 1]^T   (one M = 128, N = 144 product
//                                      whose diagonal blocks are the two gradients)
//   [dW1 | dw4 | db1 db4] += [dz1^T ; dg] [x0^T ; h3^T ; 1]^T        (M = 128, N = 112)
// the sample dimension being K of the last two, accumulated over the CTA's tiles
// in tensor memory and added to the global gradient once at the end.  A row of
// ones in B turns a column of D into the bias gradient.
//
// Tensor-memory loads (tcgen05.ld ... .sync.aligned) are executed by whole warps,
// each warp reading its own quarter of the lanes (rows), never under a branch
// that splits a warp.
//
// Operands live in shared memory in the no-swizzle K-major core-matrix layout:
// element (r, k) of an R x K bfloat16 matrix at byte
//   (r / 8) * (16 K) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. 8-row x 16-byte core matrices, the K-adjacent ones 128 bytes apart (the
// descriptor's leading byte offset) and the 8-row groups 16 K bytes apart (its
// stride byte offset).  One thread issues the MMAs and commits them to an
// mbarrier; every thread waits on it (a bounded wait: on time-out the kernel
// records ST_TIMEOUT, waits once more for the MMAs in flight, frees its tensor
// memory and returns).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {
namespace {

constexpr int kIn = APIP_MLP_IN, kW = APIP_MLP_WIDTH;
constexpr int oW1 = 0, oB1 = oW1 + kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + kW * kW, oW3 = oB2 + kW,
              oB3 = oW3 + kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW;
static_assert(oB4 + 1 == APIP_MLP_NPARAM, "parameter layout");
constexpr float kSin = 0.25f;
constexpr int kS = 128;       // samples per tile = tensor-memory lanes
constexpr int kT = 256;       // threads per CTA: two per sample

// shared-memory operands (byte offsets; every one a multiple of 1024)
constexpr int sX0 = 0;                        // [128][32]  A of layer 1
constexpr int sW1 = sX0 + kS * kIn * 2;       // [64][32]   B of layer 1
constexpr int sW2 = sW1 + kW * kIn * 2;       // [64][64]   B of layer 2
constexpr int sW3 = sW2 + kW * kW * 2;        // [64][64]   B of layer 3
constexpr int sW2t = sW3 + kW * kW * 2;       // [64][64]   W2^T, B of dh1
constexpr int sW3t = sW2t + kW * kW * 2;      // [64][64]   W3^T, B of dh2
constexpr int sH1 = sW3t + kW * kW * 2;       // [128][64]  h1 (A of layer 2), then dz3 (A of dh2)
constexpr int sH2 = sH1 + kS * kW * 2;        // [128][64]  h2 (A of layer 3), then dz2 (A of dh1)
constexpr int kNB = 2 * kW + 16;              // 144 rows: h2^T, h1^T, a row of ones, zeros
constexpr int sBW = sH2 + kS * kW * 2;        // [144][128] B of the W3 / W2 gradients
constexpr int sAW = sBW + kNB * kS * 2;       // [128][128] A of the W3 / W2 gradients: dz3^T, dz2^T
constexpr int kNB1 = kIn + kW + 16;           // 112 rows: x0^T, h3^T, a row of ones, zeros
constexpr int sB1 = sAW + kS * kS * 2;        // [112][128] B of the W1 / w4 gradients
constexpr int sA1 = sB1 + kNB1 * kS * 2;      // [128][128] A of the W1 / w4 gradients: dz1^T, dg, zeros
constexpr int sF = sA1 + kS * kS * 2;         // float32: b1, b2, b3, w4, b4 (4 kW + 4), y, g partials (3 kS)
constexpr int kSmem = sF + (4 * kW + 4 + 3 * kS) * 4;
static_assert(sW1 % 1024 == 0 && sH1 % 1024 == 0 && sBW % 1024 == 0 && sAW % 1024 == 0 && sB1 % 1024 == 0 &&
                  sA1 % 1024 == 0 && sF % 16 == 0,
              "operand alignment");
static_assert(kSmem <= 227 * 1024, "shared memory");

// tensor-memory columns (512 allocated: one CTA per SM)
constexpr uint32_t cZ1 = 0, cZ2 = 64, cZ3 = 128, cDH = 192, cW32 = 256, cW1 = cW32 + kNB;
static_assert(cW1 + kNB1 <= 512, "tensor memory");

__device__ __forceinline__ int core(int r, int k, int K) {
  return (r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void put(unsigned char* base, int r, int k, int K, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + core(r, k, K)) = __float2bfloat16_rn(v);
}

// Eight consecutive elements (r, k0 .. k0 + 7) of a row, k0 a multiple of 8: one
// 16-byte store (they form one row of a core matrix).
__device__ __forceinline__ void put8(unsigned char* base, int r, int k0, int K, const float* v) {
  uint4 w;
  uint32_t* u = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    u[q] = *reinterpret_cast<const uint32_t*>(&p);
  }
  *reinterpret_cast<uint4*>(base + core(r, k0, K)) = w;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading byte offset 128
// (K-adjacent core matrices), stride byte offset 16 K (8-row groups), the
// descriptor version of this tensor-core generation, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, int K) {
  return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(((uint32_t)K * 16) >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: float32 D, bfloat16 A and B, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D (tensor memory, column d) (+)= A B^T over K, in K = 16 steps (one thread).
__device__ __forceinline__ void mma(uint32_t tmem, uint32_t d, const unsigned char* A, const unsigned char* B, int K,
                                    int N, bool accumulate) {
  const uint32_t a0 = smem_u32(A), b0 = smem_u32(B), id = idesc(N);
  for (int kk = 0; kk < K / 16; ++kk) {
    const uint64_t ad = sdesc(a0 + kk * 256, K), bd = sdesc(b0 + kk * 256, K);
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
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
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

// The logistic function (hardware exponential and approximate division: a few
// ulp, far below the bfloat16 rounding of the GEMM operands it feeds).
__device__ __forceinline__ float sig(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

// Operands written by the threads are made visible to the tensor cores, and the
// threads' tensor-memory reads are ordered before the next MMA.
__device__ __forceinline__ void to_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__global__ void __launch_bounds__(kT, 1)
    k_train_tc(const __nv_bfloat16* __restrict__ desc, const float* __restrict__ y, int batch,
               const float* __restrict__ params, float* __restrict__ grad, double* loss_acc, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const int r = 32 * quarter + lane;            // this thread's sample row (tensor-memory lane)
  const int c0 = 32 * half;                     // its half of a layer's 64 columns
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // weights (bfloat16 operands) and the constant rows
  for (int e = tid; e < kW * kIn; e += kT) put(sm + sW1, e / kIn, e % kIn, kIn, params[oW1 + e]);
  for (int e = tid; e < kW * kW; e += kT) {
    const int rr = e / kW, k = e % kW;
    put(sm + sW2, rr, k, kW, params[oW2 + e]);
    put(sm + sW3, rr, k, kW, params[oW3 + e]);
    put(sm + sW2t, k, rr, kW, params[oW2 + e]);
    put(sm + sW3t, k, rr, kW, params[oW3 + e]);
  }
  for (int e = tid; e < 16 * kS; e += kT) {
    const int rr = e / kS, ss = e % kS;
    put(sm + sBW, 2 * kW + rr, ss, kS, rr == 0 ? 1.f : 0.f);
    put(sm + sB1, kIn + kW + rr, ss, kS, rr == 0 ? 1.f : 0.f);
  }
  for (int e = tid; e < 63 * kS; e += kT) put(sm + sA1, kW + 1 + e / kS, e % kS, kS, 0.f);
  float* fb = reinterpret_cast<float*>(sm + sF);
  float* ys = fb + 4 * kW + 4;                  // y of the tile's samples
  float* gp = ys + kS;                          // [2][kS] partial sums of the output layer
  for (int k = tid; k < kW; k += kT) {
    fb[k] = params[oB1 + k];
    fb[kW + k] = params[oB2 + k];
    fb[2 * kW + k] = params[oB3 + k];
    fb[3 * kW + k] = params[oW4 + k];
  }
  if (tid == 0) {
    fb[4 * kW] = params[oB4];
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  to_mma();
  const uint32_t tm = tmem_holder;
  const uint32_t lane_addr = tm + ((uint32_t)(32 * quarter) << 16);   // this warp's quarter of the lanes
  const float b4 = fb[4 * kW];
  const float inv_batch = 1.f / (float)batch;
  uint32_t phase = 0;
  double loss = 0.0;
  bool first = true;
  const int ntiles = (batch + kS - 1) / kS;

  // one MMA group: issued by thread 0, then every thread waits for it
  auto run = [&](auto&& issue) -> bool {
    if (tid == 0) {
      issue();
      commit(&bar);
    }
    const bool ok = wait_phase(&bar, phase);
    phase ^= 1u;
    if (!ok) failed = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    return failed == 0;
  };
  // one layer's epilogue over this thread's 32 columns: f(column, z) -> value
  // stored in row r of the A operand `rowbuf` (may be null) and, transposed, in
  // rows tbase + column of `tbuf`
  // (tbase + c0 and c0 are multiples of 8: the addresses are a per-thread base
  // plus compile-time offsets)
  auto epilogue = [&](uint32_t col, unsigned char* rowbuf, unsigned char* tbuf, int tbase, auto&& f) {
    unsigned char* tb = tbuf + core(tbase + c0, r, kS);
    unsigned char* rb = rowbuf ? rowbuf + core(r, c0, kW) : nullptr;
#pragma unroll
    for (int c = 0; c < 32; c += 16) {
      float z[16], o[16];
      tld16(lane_addr + col + c0 + c, z);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        o[q] = f(c0 + c + q, z[q]);
        const int j = c + q;
        *reinterpret_cast<__nv_bfloat16*>(tb + (j >> 3) * (kS * 16) + (j & 7) * 16) = __float2bfloat16_rn(o[q]);
      }
      if (rb) {
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
          uint4 w;
          uint32_t* u = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(o[8 * h8 + 2 * q], o[8 * h8 + 2 * q + 1]);
            u[q] = *reinterpret_cast<const uint32_t*>(&p);
          }
          *reinterpret_cast<uint4*>(rb + ((c + 8 * h8) >> 3) * 128) = w;
        }
      }
    }
  };

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int s = tile * kS + r;
    const bool valid = s < batch;
    // inputs: x0 = 0.25 G (exact in bfloat16), features 16 half .. of row r of the
    // layer-1 A and of column r of the W1-gradient B
    {
      const uint4* src = reinterpret_cast<const uint4*>(desc + (size_t)(valid ? s : 0) * kIn) + 2 * half;
      float x[16];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const uint4 v = valid ? src[q] : make_uint4(0u, 0u, 0u, 0u);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          x[8 * q + e] = kSin * __bfloat162float(h[e]);
          put(sm + sB1, 16 * half + 8 * q + e, r, kS, x[8 * q + e]);
        }
      }
      put8(sm + sX0, r, 16 * half, kIn, x);
      put8(sm + sX0, r, 16 * half + 8, kIn, x + 8);
      if (half == 0) ys[r] = valid ? y[s] : 0.f;
    }
    to_mma();
    if (!run([&] { mma(tm, cZ1, sm + sX0, sm + sW1, kIn, kW, false); })) break;
    // layer 1: h1 = silu(z1 + b1) -> A of layer 2 and rows 64.. of the W-gradient B (h1^T)
    epilogue(cZ1, sm + sH1, sm + sBW, kW, [&](int c, float z) {
      const float zz = z + fb[c];
      return zz * sig(zz);
    });
    to_mma();
    if (!run([&] { mma(tm, cZ2, sm + sH1, sm + sW2, kW, kW, false); })) break;
    // layer 2: h2 -> A of layer 3 and rows 0.. of the W-gradient B (h2^T)
    epilogue(cZ2, sm + sH2, sm + sBW, 0, [&](int c, float z) {
      const float zz = z + fb[kW + c];
      return zz * sig(zz);
    });
    to_mma();
    if (!run([&] { mma(tm, cZ3, sm + sH2, sm + sW3, kW, kW, false); })) break;
    // layer 3 and the output: g = w4 . h3 + b4, its two halves summed through
    // shared memory; h3^T -> rows 32.. of the W1-gradient B
    float gh = 0.f;
    epilogue(cZ3, nullptr, sm + sB1, kIn, [&](int c, float z) {
      const float zz = z + fb[2 * kW + c];
      const float h = zz * sig(zz);
      gh = fmaf(fb[3 * kW + c], h, gh);
      return h;
    });
    gp[half * kS + r] = gh;
    __syncthreads();
    const float g = b4 + gp[r] + gp[kS + r];
    const float res = valid ? g - ys[r] : 0.f;
    if (half == 0) {
      loss += (double)res * (double)res;
      put(sm + sA1, kW, r, kS, 2.f * res * inv_batch);   // row 64 of the W1-gradient A: dg
    }
    const float dg = 2.f * res * inv_batch;
    // dz3 = dg w4 silu'(z3) -> A of dh2 (the h1 buffer) and rows 0.. of the W-gradient A (dz3^T)
    epilogue(cZ3, sm + sH1, sm + sAW, 0, [&](int c, float z) {
      const float zz = z + fb[2 * kW + c];
      const float sg = sig(zz);
      return dg * fb[3 * kW + c] * (sg * (1.f + zz * (1.f - sg)));
    });
    to_mma();
    if (!run([&] { mma(tm, cDH, sm + sH1, sm + sW3t, kW, kW, false); })) break;
    // dz2 = dh2 silu'(z2) -> A of dh1 (the h2 buffer) and rows 64.. of the W-gradient A
    {
      float zs[32];
      tld16(lane_addr + cZ2 + c0, zs);
      tld16(lane_addr + cZ2 + c0 + 16, zs + 16);
      epilogue(cDH, sm + sH2, sm + sAW, kW, [&](int c, float dh) {
        const float zz = zs[c - c0] + fb[kW + c];
        const float sg = sig(zz);
        return valid ? dh * (sg * (1.f + zz * (1.f - sg))) : 0.f;
      });
    }
    to_mma();
    if (!run([&] { mma(tm, cDH, sm + sH2, sm + sW2t, kW, kW, false); })) break;
    // dz1 = dh1 silu'(z1) -> rows 0.. of the W1-gradient A
    {
      float zs[32];
      tld16(lane_addr + cZ1 + c0, zs);
      tld16(lane_addr + cZ1 + c0 + 16, zs + 16);
      epilogue(cDH, nullptr, sm + sA1, 0, [&](int c, float dh) {
        const float zz = zs[c - c0] + fb[c];
        const float sg = sig(zz);
        return valid ? dh * (sg * (1.f + zz * (1.f - sg))) : 0.f;
      });
    }
    to_mma();
    const bool acc = !first;
    if (!run([&] {
          mma(tm, cW32, sm + sAW, sm + sBW, kS, kNB, acc);
          mma(tm, cW1, sm + sA1, sm + sB1, kS, kNB1, acc);
        }))
      break;
    first = false;
  }
  // the accumulated gradients: lane m = row m of the two gradient products, this
  // thread's half of the columns (the loads are warp-wide: every branch below is
  // uniform across a warp)
  if (!first && failed == 0) {
    const int m = r;
    float v[16];
    if (quarter < 2) {                            // rows 0 .. 63: dW3, dW1, db3, db1
      for (int c = 0; c < 32; c += 16) {
        tld16(lane_addr + cW32 + c0 + c, v);
        for (int q = 0; q < 16; ++q) atomicAdd(&grad[oW3 + m * kW + c0 + c + q], v[q]);
      }
      tld16(lane_addr + cW1 + 16 * half, v);
      for (int q = 0; q < 16; ++q) atomicAdd(&grad[oW1 + m * kIn + 16 * half + q], v[q]);
      if (half == 0) {
        tld16(lane_addr + cW32 + 2 * kW, v);
        atomicAdd(&grad[oB3 + m], v[0]);
        tld16(lane_addr + cW1 + kIn + kW, v);
        atomicAdd(&grad[oB1 + m], v[0]);
      }
    } else {                                      // rows 64 .. 127: dW2, db2; row 64 also dw4, db4
      const int j = m - kW;
      for (int c = 0; c < 32; c += 16) {
        tld16(lane_addr + cW32 + kW + c0 + c, v);
        for (int q = 0; q < 16; ++q) atomicAdd(&grad[oW2 + j * kW + c0 + c + q], v[q]);
      }
      if (half == 0) {
        tld16(lane_addr + cW32 + 2 * kW, v);
        atomicAdd(&grad[oB2 + j], v[0]);
      }
      if (quarter == 2) {
        for (int c = 0; c < 32; c += 16) {
          tld16(lane_addr + cW1 + kIn + c0 + c, v);
          if (m == kW)
            for (int q = 0; q < 16; ++q) atomicAdd(&grad[oW4 + c0 + c + q], v[q]);
        }
        if (half == 0) {
          tld16(lane_addr + cW1 + kIn + kW, v);
          if (m == kW) atomicAdd(&grad[oB4], v[0]);
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
  if (lane == 0 && loss != 0.0) atomicAdd(loss_acc, loss);
  if (failed) {
    if (tid == 0) atomicOr(&status[ST_TIMEOUT], 1);
    wait_phase(&bar, phase ^ 1u);   // the MMAs in flight, once more (bounded)
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(512));
}

__global__ void k_train_loss_tc(const double* loss_acc, int batch, float* loss_out) {
  *loss_out = (float)(*loss_acc / batch);
}

}  // namespace

size_t mlp_workspace_floats(int batch) {
  (void)batch;
  return 4;   // the float64 loss accumulator
}

void launch_mlp_loss_grad(const uint16_t* desc, const float* y, int batch, const float* params, float* grad,
                          float* loss, float* ws, int* status, cudaStream_t s) {
  double* acc = reinterpret_cast<double*>(ws);
  cudaMemsetAsync(grad, 0, sizeof(float) * APIP_MLP_NPARAM, s);
  cudaMemsetAsync(acc, 0, sizeof(double), s);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = (batch + kS - 1) / kS;
  const int grid = ntiles < sms ? ntiles : sms;   // one CTA per SM (512 tensor-memory columns each)
  cudaFuncSetAttribute(k_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  k_train_tc<<<grid, kT, kSmem, s>>>(reinterpret_cast<const __nv_bfloat16*>(desc), y, batch, params, grad, acc,
                                     status);
  k_train_loss_tc<<<1, 1, 0, s>>>(acc, batch, loss);
}

}  // namespace apip
