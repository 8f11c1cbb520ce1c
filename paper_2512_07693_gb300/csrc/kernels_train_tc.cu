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
// are float32.  The factor 0.25 of the inputs is moved onto W1 (bfloat16
// scaling by a power of two is exact, so every product is unchanged) and onto
// the W1 gradient at the end; the layer-1 operand is then G itself.
//
// A CTA of 512 threads loops over 128-sample tiles (a persistent grid of one CTA
// per SM).  Sample r of a tile is tensor-memory lane r; warp w reads lanes
// 32 (w % 4) .. + 31 and owns columns 16 (w / 4) .. + 15 of each 64-wide layer.
// Per tile, with D = A B^T on the tensor cores (M = 128 rows of A, N rows of B):
//   z1 = G (W1/4)^T, z2 = h1 W2^T, z3 = h2 W3^T           (forward, M = samples)
//   dh2 = dz3 W3, dh1 = dz2 W2                          (back-propagation)
//   [dW3 | dW2 | db3 db2] += [dz3 ; dz2]^T [h2 | h1 | 1]  (M = 128, N = 144, K = samples;
//                                                       the diagonal blocks are the gradients)
//   [dW1 | db1] += dz1^T [G | 1]                         (M = 128 of which 64 are used, N = 48)
// The forward epilogues leave silu'(z) in the tensor-memory columns of z for the
// back-propagation.  The gradient products accumulate over the CTA's tiles in
// tensor memory; the output layer's gradient (dw4, db4) is summed by the
// threads.  Each CTA writes its sums once and a second kernel adds the CTAs'
// sums in a fixed order, so the gradient is the same bit for bit on every call.
//
// Operand layout ("chunk-major", no swizzle): an operand with 128 samples is
// stored as 8-feature chunks of 128 x 16 bytes, element (sample s, feature f) at
//   (f / 8) * 2048 + s * 16 + (f % 8) * 2.
// Read as a K-major operand (samples = M, features = K) its core matrices are 8
// samples x 16 bytes, the K-adjacent ones 2048 bytes apart (leading byte offset)
// and the 8-sample groups 128 bytes apart (stride byte offset).  Read as an
// MN-major operand (features = M or N, samples = K) its core matrices are 8
// samples x 8 features: the 8-sample groups (along K) 128 bytes apart (leading
// byte offset) and the 8-feature groups 2048 bytes apart (stride byte offset).
// So every activation a thread writes once, row by row, serves both the next
// layer's product and the transposed gradient product; nothing is transposed.
// The weights are stored the same way with 64 rows (chunks of 1024 bytes): K-major
// for the forward products and, the same bytes read MN-major, transposed for the
// back-propagation; each CTA converts them from the float32 parameters once.  The
// per-tile inputs G arrive by TMA (four 8 x 128 boxes, zero-filled past the
// batch), double-buffered: the next tile's load is in flight while this tile
// computes.
//
// Tensor-memory loads and stores (tcgen05.ld / st ... .sync.aligned) are executed
// by whole warps, each warp on its own quarter of the lanes, never under a branch
// that splits a warp.  One thread issues the MMAs and the copies; MMAs are
// committed to an mbarrier that every thread waits on itself.  Every wait is
// bounded (two seconds): on time-out the kernel records ST_TIMEOUT, stops issuing,
// leaves the tile loop at the next CTA barrier, waits once more for the MMAs and
// copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "tc_common.cuh"

namespace apip {
namespace {

using namespace tc;

constexpr int kIn = APIP_MLP_IN, kW = APIP_MLP_WIDTH;
constexpr int oW1 = 0, oB1 = oW1 + kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + kW * kW, oW3 = oB2 + kW,
              oB3 = oW3 + kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW;
static_assert(oB4 + 1 == APIP_MLP_NPARAM, "parameter layout");
static_assert(kIn == 32 && kW == 64, "the tile layout below is written for a 32-64-64-64-1 network");
static_assert((kW * kIn) % 512 == 0 && (kW * kW) % 512 == 0 && 4 * kW + 4 <= 512, "weight conversion");
constexpr float kSin = 0.25f;
constexpr int kS = 128;                 // samples per tile = tensor-memory lanes
constexpr int kT = 512;                 // threads per CTA: four per sample
constexpr int kC = 16;                  // columns of a 64-wide layer per thread
constexpr int kChunk = kS * 16;         // bytes of an 8-feature chunk of a 128-sample operand

// shared memory (byte offsets)
constexpr int kXBuf = 6 * kChunk;       // G (4 chunks, by TMA), a chunk of ones, a chunk of zeros
constexpr int sX = 0;                   // two input buffers
constexpr int sWt1 = sX + 2 * kXBuf;    // W1 / 4: [4 K-chunks][64 rows][16 B]
constexpr int sWt2 = sWt1 + kW * kIn * 2;
constexpr int sWt3 = sWt2 + kW * kW * 2;
constexpr int sFp = sWt3 + kW * kW * 2; // float32 b1, b2, b3, w4, b4, 3 pad
constexpr int kNF = 4 * kW + 4;
constexpr int sGp = sFp + kNF * 4;      // float32 [4][128]: the output layer's partial sums
constexpr int sH2 = 48 * 1024;          // h2 | h1 | ones | zeros: B of the big gradient product
constexpr int sH1 = sH2 + 8 * kChunk;
constexpr int sOnes = sH1 + 8 * kChunk;
constexpr int sDZ1 = sOnes + 2 * kChunk;  // dz1 | dz3 | dz2: A of the W1 gradient (16 chunks from dz1),
constexpr int sDZ3 = sDZ1 + 8 * kChunk;   //   A of the big gradient product (dz3 | dz2),
constexpr int sDZ2 = sDZ3 + 8 * kChunk;   //   A of dh2 (dz3) and of dh1 (dz2)
constexpr int kSmem = sDZ2 + 8 * kChunk;
static_assert(sGp + kS * 4 * 4 <= sH2, "shared-memory map");
static_assert(sWt1 % 1024 == 0 && sH2 % 1024 == 0 && sDZ1 % 1024 == 0 && sFp % 16 == 0, "alignment");
// per-CTA gradient sums in the workspace: the parameters padded to 16 bytes
constexpr int kPart = (APIP_MLP_NPARAM + 3) / 4 * 4;
static_assert(oW1 % 4 == 0 && oW2 % 4 == 0 && oW3 % 4 == 0, "16-byte aligned weight rows");
static_assert(kSmem <= 227 * 1024, "shared memory");

// tensor-memory columns (512 allocated: one CTA per SM)
constexpr uint32_t cZ1 = 0, cZ2 = 64, cZ3 = 128, cDH = 192, cW32 = 256, cW1 = 400;
constexpr int kNB = 2 * kW + 16, kNB1 = kIn + 16;
static_assert(cW32 + kNB <= cW1 && cW1 + kNB1 <= 512, "tensor memory");

// G rows 128 tile .. + 127 into an input buffer: four boxes of 8 features x 128
// samples (TMA; rows past the batch read as zeros), completing on `bar`.
__device__ __forceinline__ void load_tile(const CUtensorMap* map, unsigned char* dst, uint64_t* bar, int tile) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(4 * kChunk)
               : "memory");
#pragma unroll
  for (int c = 0; c < 4; ++c)
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst + c * kChunk)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(8 * c), "r"(tile * kS), "r"(smem_u32(bar))
        : "memory");
}

// Sixteen float32 values as bfloat16 into row r of a chunk-major operand at
// column c0 (a multiple of 8): two 16-byte stores.
__device__ __forceinline__ void put16(unsigned char* base, int r, int c0, const float* v) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint4 w;
    uint32_t* u = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 p = __floats2bfloat162_rn(v[8 * h + 2 * q], v[8 * h + 2 * q + 1]);
      u[q] = *reinterpret_cast<const uint32_t*>(&p);
    }
    *reinterpret_cast<uint4*>(base + chunk_off(r, c0 + 8 * h, kS)) = w;
  }
}

__global__ void __launch_bounds__(kT, 1)
    k_train_tc(const __grid_constant__ CUtensorMap gmap, const float* __restrict__ y, int batch,
               const float* __restrict__ params, float* __restrict__ part, double* loss_part, int* status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar, tbar[2];
  __shared__ uint32_t tmem_holder;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, cg = warp >> 2;
  const int r = 32 * quarter + lane;            // this thread's sample row (tensor-memory lane)
  const int c0 = kC * cg;                       // its columns of a 64-wide layer
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the constant chunks (16-byte words): a chunk of ones (feature 0 of every
  // sample 1, for the bias gradients) and a chunk of zeros, after each input
  // buffer and after h1
  {
    const uint4 one = make_uint4(0x3f80u, 0u, 0u, 0u), zero = make_uint4(0u, 0u, 0u, 0u);
    for (int e = tid; e < 2 * kS; e += kT) {
      const int s = e & (kS - 1), wch = e >> 7;
      const uint4 v = wch == 0 ? one : zero;
      *reinterpret_cast<uint4*>(sm + sX + 4 * kChunk + wch * kChunk + s * 16) = v;
      *reinterpret_cast<uint4*>(sm + sX + kXBuf + 4 * kChunk + wch * kChunk + s * 16) = v;
      *reinterpret_cast<uint4*>(sm + sOnes + wch * kChunk + s * 16) = v;
    }
  }
  const int ntiles = (batch + kS - 1) / kS;
  const int stride = gridDim.x;
  // input copies (thread 0 only): issued and waited-for counts per buffer; the
  // k-th copy into a buffer completes phase k of its barrier
  uint32_t tissued0 = 0, tissued1 = 0, twaited0 = 0, twaited1 = 0;
  auto tload = [&](int b, int tile) {
    load_tile(&gmap, sm + sX + b * kXBuf, &tbar[b], tile);
    ++(b ? tissued1 : tissued0);
  };
  auto twait = [&](int b) -> bool {
    uint32_t& k = b ? twaited1 : twaited0;
    return wait_phase(&tbar[b], k++ & 1u);
  };
  // everything below may read what the previous kernel wrote
  pdl_begin();
  if (tid == 0) {
    tload(0, blockIdx.x);
    if (blockIdx.x + stride < ntiles) tload(1, blockIdx.x + stride);
  }
  // the weight operands from the float32 parameters (coalesced reads): W1 / 4, W2,
  // W3 as bfloat16 in the chunk-major layout with 64 rows; biases and w4 as float32
#pragma unroll
  for (int k = 0; k < kW * kIn / kT; ++k) {
    const int e = tid + k * kT;
    *reinterpret_cast<__nv_bfloat16*>(sm + sWt1 + chunk_off(e / kIn, e % kIn, kW)) =
        __float2bfloat16_rn(kSin * params[oW1 + e]);
  }
#pragma unroll
  for (int k = 0; k < kW * kW / kT; ++k) {
    const int e = tid + k * kT;
    const int o = chunk_off(e / kW, e % kW, kW);
    *reinterpret_cast<__nv_bfloat16*>(sm + sWt2 + o) = __float2bfloat16_rn(params[oW2 + e]);
    *reinterpret_cast<__nv_bfloat16*>(sm + sWt3 + o) = __float2bfloat16_rn(params[oW3 + e]);
  }
  if (tid < 4 * kW + 4) {
    const int q = tid / kW, c = tid % kW;
    const int src = q == 0 ? oB1 : q == 1 ? oB2 : q == 2 ? oB3 : oW4;
    reinterpret_cast<float*>(sm + sFp)[tid] = tid < 4 * kW ? params[src + c] : (tid == 4 * kW ? params[oB4] : 0.f);
  }
  to_mma();
  const uint32_t tm = tmem_holder;
  const uint32_t lane_addr = tm + ((uint32_t)(32 * quarter) << 16);   // this warp's quarter of the lanes
  const float* fb = reinterpret_cast<const float*>(sm + sFp);
  float* gp = reinterpret_cast<float*>(sm + sGp);
  const float b4 = fb[4 * kW];
  const float inv_batch = 1.f / (float)batch;
  const uint32_t id64 = idesc(kW, false, false), id_bwd = idesc(kW, false, true);
  const uint32_t id_w32 = idesc(kNB, true, true), id_w1 = idesc(kNB1, true, true);
  uint32_t phase = 0;
  double loss = 0.0;
  float aw4[kC], ab4 = 0.f;   // this thread's share of dw4 (its columns) and of db4 (cg == 0)
#pragma unroll
  for (int q = 0; q < kC; ++q) aw4[q] = 0.f;
  bool first = true;

  // one MMA group: issued by thread 0, then every thread waits for it itself (no
  // CTA barrier: the next step's shared-memory writes touch no operand in use).
  // After a time-out nothing more is issued; `failed` is read uniformly right
  // after the CTA barrier of each to_mma(), where the tile loop is left.
  int fail_par = -1;   // parity of a group this thread saw time out
  auto run = [&](auto&& issue) {
    if (!failed) {
      if (tid == 0) {
        issue();
        commit(&bar);
      }
      if (!wait_phase(&bar, phase)) {
        failed = 1;
        fail_par = (int)phase;
      }
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  };
  // one forward layer's epilogue on this thread's 16 columns: h = silu(z + b)
  // into row r of `dst`, silu'(z + b) back into the tensor-memory columns of z
  auto forward = [&](uint32_t col, const float* bias, unsigned char* dst) {
    float z[kC], d[kC];
    tld16(lane_addr + col + c0, z);
#pragma unroll
    for (int q = 0; q < kC; ++q) {
      const float zz = z[q] + bias[c0 + q];
      const float sg = sig(zz);
      d[q] = sg * (1.f + zz * (1.f - sg));
      z[q] = zz * sg;
    }
    put16(dst, r, c0, z);
    tst16(lane_addr + col + c0, d);
  };
  // one backward epilogue: dz = dh silu'(z) (zero for samples past the batch)
  auto backward = [&](uint32_t dcol, unsigned char* dst, bool valid) {
    float dh[kC], d[kC];
    tld16(lane_addr + cDH + c0, dh);
    tld16(lane_addr + dcol + c0, d);
#pragma unroll
    for (int q = 0; q < kC; ++q) dh[q] = valid ? dh[q] * d[q] : 0.f;
    put16(dst, r, c0, dh);
  };

  // layer 1 of the first tile
  run([&] {
    if (!twait(0)) failed = 1;
    else mma(tm, cZ1, act_k(sm + sX), wt_k(sm + sWt1), kIn, id64, false);
  });
  for (int it = 0;; ++it) {
    const int tile = blockIdx.x + it * stride;
    if (tile >= ntiles) break;
    const int b = it & 1;
    const int s = tile * kS + r;
    const bool valid = s < batch;
    const float yv = valid ? y[s] : 0.f;
    forward(cZ1, fb, sm + sH1);
    to_mma();
    if (failed) break;
    run([&] { mma(tm, cZ2, act_k(sm + sH1), wt_k(sm + sWt2), kW, id64, false); });
    forward(cZ2, fb + kW, sm + sH2);
    to_mma();
    if (failed) break;
    run([&] { mma(tm, cZ3, act_k(sm + sH2), wt_k(sm + sWt3), kW, id64, false); });
    // layer 3 and the output g = w4 . h3 + b4 (the four column groups' partial sums
    // through shared memory), then dz3 = dg w4 silu'(z3)
    {
      float h3[kC], d3[kC], gh = 0.f;
      tld16(lane_addr + cZ3 + c0, h3);
#pragma unroll
      for (int q = 0; q < kC; ++q) {
        const float zz = h3[q] + fb[2 * kW + c0 + q];
        const float sg = sig(zz);
        d3[q] = sg * (1.f + zz * (1.f - sg));
        h3[q] = zz * sg;
        gh = fmaf(fb[3 * kW + c0 + q], h3[q], gh);
      }
      gp[cg * kS + r] = gh;
      __syncthreads();
      const float g = b4 + ((gp[r] + gp[kS + r]) + (gp[2 * kS + r] + gp[3 * kS + r]));
      const float res = valid ? g - yv : 0.f;
      const float dg = 2.f * res * inv_batch;
      const float dgb = bf16r(dg);
      if (cg == 0) {
        loss += (double)res * (double)res;
        ab4 += dgb;
      }
#pragma unroll
      for (int q = 0; q < kC; ++q) {
        aw4[q] = fmaf(dgb, bf16r(h3[q]), aw4[q]);
        d3[q] = dg * fb[3 * kW + c0 + q] * d3[q];
      }
      put16(sm + sDZ3, r, c0, d3);
    }
    to_mma();
    if (failed) break;
    run([&] { mma(tm, cDH, act_k(sm + sDZ3), wt_mn(sm + sWt3), kW, id_bwd, false); });
    backward(cZ2, sm + sDZ2, valid);
    to_mma();
    if (failed) break;
    run([&] { mma(tm, cDH, act_k(sm + sDZ2), wt_mn(sm + sWt2), kW, id_bwd, false); });
    backward(cZ1, sm + sDZ1, valid);
    to_mma();
    if (failed) break;
    // the gradient products of this tile, and layer 1 of the next tile (its input
    // buffer is the other one; its output columns hold nothing needed any more)
    const bool acc = !first;
    const bool next = tile + stride < ntiles;
    run([&] {
      mma(tm, cW32, act_mn(sm + sDZ3), act_mn(sm + sH2), kS, id_w32, acc);
      mma(tm, cW1, act_mn(sm + sDZ1), act_mn(sm + sX + b * kXBuf), kS, id_w1, acc);
      if (next) {
        if (!twait(b ^ 1)) failed = 1;
        else mma(tm, cZ1, act_k(sm + sX + (b ^ 1) * kXBuf), wt_k(sm + sWt1), kIn, id64, false);
      }
    });
    first = false;
    // this tile's input buffer is free again: the tile after next goes there
    if (tid == 0 && !failed && tile + 2 * stride < ntiles) tload(b, tile + 2 * stride);
  }
  __syncthreads();   // `failed` is uniform from here on
  // this CTA's gradient sums, part[blockIdx.x][parameter]: lane m = row m of the
  // two gradient products; zero if the CTA had no tile or a wait gave up.  Every
  // branch below is uniform across a warp.
  float* out = part + (size_t)blockIdx.x * kPart;
  const bool have = !first && failed == 0;
  // 16 values of a row as four 16-byte stores (the rows start 16-byte aligned)
  auto put_row = [&](float* dst, const float* v, float scale) {
#pragma unroll
    for (int q = 0; q < 16; q += 4)
      *reinterpret_cast<float4*>(dst + q) =
          have ? make_float4(scale * v[q], scale * v[q + 1], scale * v[q + 2], scale * v[q + 3])
               : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  {
    const int m = r;
    float v[16];
    if (quarter < 2) {                            // rows 0 .. 63: dW3, db3; dW1, db1
      if (have) tld16(lane_addr + cW32 + c0, v);
      put_row(out + oW3 + m * kW + c0, v, 1.f);
      if (cg < 2) {
        if (have) tld16(lane_addr + cW1 + c0, v);
        put_row(out + oW1 + m * kIn + c0, v, kSin);
      } else if (cg == 2) {
        if (have) tld16(lane_addr + cW32 + 2 * kW, v);
        out[oB3 + m] = have ? v[0] : 0.f;
      } else {
        if (have) tld16(lane_addr + cW1 + kIn, v);
        out[oB1 + m] = have ? v[0] : 0.f;
      }
    } else {                                      // rows 64 .. 127: dW2, db2
      const int j = m - kW;
      if (have) tld16(lane_addr + cW32 + kW + c0, v);
      put_row(out + oW2 + j * kW + c0, v, 1.f);
      if (cg == 0) {
        if (have) tld16(lane_addr + cW32 + 2 * kW, v);
        out[oB2 + j] = have ? v[0] : 0.f;
      }
    }
  }
  // dw4, db4 and the loss: warp sums, then the warps in a fixed order
  {
    __shared__ float red[kT / 32][kC + 1];
    __shared__ double lred[kT / 32];
#pragma unroll
    for (int q = 0; q < kC; ++q)
      for (int o = 16; o > 0; o >>= 1) aw4[q] += __shfl_xor_sync(0xffffffffu, aw4[q], o);
    for (int o = 16; o > 0; o >>= 1) {
      ab4 += __shfl_xor_sync(0xffffffffu, ab4, o);
      loss += __shfl_xor_sync(0xffffffffu, loss, o);
    }
    if (lane == 0) {
      for (int q = 0; q < kC; ++q) red[warp][q] = aw4[q];
      red[warp][kC] = ab4;
      lred[warp] = loss;
    }
    __syncthreads();
    if (tid < kW) {                               // column tid: the warps 4 (tid / 16) + quarter
      const int g4 = tid / kC, q = tid % kC;
      const float t = (red[4 * g4][q] + red[4 * g4 + 1][q]) + (red[4 * g4 + 2][q] + red[4 * g4 + 3][q]);
      out[oW4 + tid] = have ? t : 0.f;
    } else if (tid == kW) {
      const float t = (red[0][kC] + red[1][kC]) + (red[2][kC] + red[3][kC]);
      out[oB4] = have ? t : 0.f;
    } else if (tid == kW + 1) {
      double t = 0.0;
      for (int w = 0; w < kT / 32; ++w) t += lred[w];
      loss_part[blockIdx.x] = t;
    }
  }
  if (failed && tid == 0) {
    atomicOr(&status[ST_TIMEOUT], 1);
    // the MMAs and input copies still in flight, once more (bounded)
    if (fail_par >= 0) wait_phase(&bar, (uint32_t)fail_par);
    while (twaited0 < tissued0 && twait(0)) {}
    while (twaited1 < tissued1 && twait(1)) {}
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(512));
}

// grad[p] = sum over the CTAs of part[b][p] in a fixed order (eight interleaved
// partial sums over b, then those in order); the loss likewise.  A block takes 128
// parameters, a lane four consecutive ones (16-byte loads).
constexpr int kRedWarps = 8;
__global__ void __launch_bounds__(32 * kRedWarps)
    k_train_reduce(const float* __restrict__ part, const double* __restrict__ loss_part, int nb, int batch,
                   float* __restrict__ grad, float* __restrict__ loss_out) {
  pdl_begin();
  __shared__ float4 red[kRedWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p = 4 * (blockIdx.x * 32 + lane);   // first of this lane's parameters
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (p < kPart) {
#pragma unroll 4
    for (int b = w; b < nb; b += kRedWarps) {
      const float4 v = *reinterpret_cast<const float4*>(part + (size_t)b * kPart + p);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  red[w][lane] = acc;
  __syncthreads();
  if (w == 0 && p < APIP_MLP_NPARAM) {
    float t[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < kRedWarps; ++k) {
      const float4 v = red[k][lane];
      t[0] += v.x;
      t[1] += v.y;
      t[2] += v.z;
      t[3] += v.w;
    }
    for (int q = 0; q < 4 && p + q < APIP_MLP_NPARAM; ++q) grad[p + q] = t[q];
  }
  if (blockIdx.x == 0 && threadIdx.x == 32) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += loss_part[b];
    *loss_out = (float)(t / batch);
  }
}

int train_grid_max() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}
size_t loss_floats(int g) { return (2 * (size_t)g + 3) / 4 * 4; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

}  // namespace

// Workspace (floats, from a 16-byte aligned base): the loss partials (float64, one
// per CTA, padded to 16 bytes), then the CTAs' gradient sums (kPart floats each).
size_t mlp_workspace_floats(int batch) {
  (void)batch;
  const int g = train_grid_max();
  return loss_floats(g) + (size_t)g * kPart;
}

bool launch_mlp_loss_grad(const uint16_t* desc, const float* y, int batch, const float* params, float* grad,
                          float* loss, float* ws, int* status, cudaStream_t s) {
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_tiled();
  if (!encode || (reinterpret_cast<uintptr_t>(desc) & 15u) != 0) return false;
  // G as a [batch][32] bfloat16 tensor read in boxes of 8 features x 128 samples
  CUtensorMap gmap;
  const cuuint64_t dims[2] = {(cuuint64_t)kIn, (cuuint64_t)batch};
  const cuuint64_t strides[1] = {(cuuint64_t)kIn * 2};
  const cuuint32_t box[2] = {8u, (cuuint32_t)kS};
  const cuuint32_t estr[2] = {1u, 1u};
  if (encode(&gmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(desc), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const int gmax = train_grid_max();
  double* loss_part = reinterpret_cast<double*>(ws);
  float* part = ws + loss_floats(gmax);
  const int ntiles = (batch + kS - 1) / kS;
  const int grid = ntiles < gmax ? ntiles : gmax;   // one CTA per SM (512 tensor-memory columns each)
  cudaFuncSetAttribute(k_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  launch_pdl(k_train_tc, grid, kT, kSmem, s, gmap, y, batch, params, part, loss_part, status);
  launch_pdl(k_train_reduce, (kPart / 4 + 31) / 32, 32 * kRedWarps, 0, s, (const float*)part,
             (const double*)loss_part, grid, batch, grad, loss);
  return true;
}

}  // namespace apip
