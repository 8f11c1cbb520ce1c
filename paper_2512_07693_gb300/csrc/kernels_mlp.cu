// Learned switching quantity: radial descriptors, the indicator MLP (forward,
// input gradient for the forces, and batched training with Adam).
//
// g_k of Eq. 6 may be any differentiable function of interatomic distances (main
// text after Eq. 5).  Here g_k = MLP(G_k) with G_km = sum_j phi_m(r_kj), so the
// grad-lambda force needs -grad sum_k c_k g_k = -sum_k c_k sum_m dg_k/dG_km grad G_km,
// with c_k = sum_i Et_i w(r_ik) accumulated by the ACE kernel exactly as for CSP^list.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {
namespace {

constexpr int kIn = APIP_MLP_IN, kW = APIP_MLP_WIDTH;
constexpr int oW1 = 0, oB1 = oW1 + kW * kIn, oW2 = oB1 + kW, oB2 = oW2 + kW * kW, oW3 = oB2 + kW,
              oB3 = oW3 + kW * kW, oW4 = oB3 + kW, oB4 = oW4 + kW;
static_assert(oB4 + 1 == APIP_MLP_NPARAM, "parameter layout");
constexpr double kMu0 = 1.5, kDmu = (5.0 - 1.5) / (kIn - 1), kEta = 1.0 / (2.0 * 0.15 * 0.15), kSin = 0.25;

// SiLU and its derivative (float32: the hardware exponential, as for the EAM terms)
template <typename T> __device__ __forceinline__ T silu(T z) { return z / (T(1) + fexp(-z)); }
template <typename T> __device__ __forceinline__ T silu_d(T z) {
  const T s = T(1) / (T(1) + fexp(-z));
  return s * (T(1) + z * (T(1) - s));
}

// phi_m(r) = exp(-eta (r - mu_m)^2) fc(r) for m = 0..31 (and d phi_m/dr), from
// the Gaussian nearest to r outward with the ratio recurrence
//   e_{m+1} = e_m rho_m, rho_{m+1} = rho_m kappa;  e_{m-1} = e_m sig_m, sig_{m-1} = sig_m kappa,
// rho_m = exp(-eta dmu^2 + 2 eta dmu x_m), sig_m = exp(-eta dmu^2 - 2 eta dmu x_m),
// kappa = exp(-2 eta dmu^2), x_m = r - mu_m: three exponentials per neighbour,
// and values only shrink away from the centre (no overflow).
template <typename T, bool DERIV>
__device__ __forceinline__ void features(T r, T fc, T dfc, T* phi, T* dphi) {
  const T dmu = T(kDmu), eta = T(kEta);
  int m0 = (int)rint((r - T(kMu0)) / dmu);
  m0 = m0 < 0 ? 0 : (m0 > kIn - 1 ? kIn - 1 : m0);
  const T x0 = r - (T(kMu0) + T(m0) * dmu);
  const T e0 = exp(-eta * x0 * x0);
  const T kappa = exp(T(-2) * eta * dmu * dmu);
  const T base = -eta * dmu * dmu, slope = T(2) * eta * dmu * x0;
  T up = e0, rho = exp(base + slope);
#pragma unroll
  for (int m = 0; m < kIn; ++m) {
    if (m > m0) { up *= rho; rho *= kappa; }
    if (m >= m0) phi[m] = up;
  }
  T dn = e0, sig = exp(base - slope);
#pragma unroll
  for (int m = kIn - 1; m >= 0; --m) {
    if (m < m0) { dn *= sig; sig *= kappa; phi[m] = dn; }
  }
#pragma unroll
  for (int m = 0; m < kIn; ++m) {
    if (DERIV) {
      const T x = r - (T(kMu0) + T(m) * dmu);
      dphi[m] = phi[m] * (T(-2) * eta * x * fc + dfc);
    }
    phi[m] *= fc;
  }
}

// Descriptors of atom i over its neighbour list (r < rc of the ACE).
template <typename T>
__device__ __forceinline__ void descriptors_of(const Args<T>& a, int i, T* G) {
#pragma unroll
  for (int m = 0; m < kIn; ++m) G[m] = T(0);
  const auto si = a.pv.self(i);
  const T rc2 = a.ace_rc * a.ace_rc, inv_w = T(1) / (a.ace_rc - a.ace_rc_lo);
  const int cnt = a.nnb[i];
  for (int s = 0; s < cnt; ++s) {
    const int j = a.nbl[(size_t)s * a.nmax + i];
    const auto d = a.pv.vec(si, j);
    const T r2 = dot3(d, d);
    if (!(r2 < rc2)) continue;
    const T r = sqrt(r2);
    T dfc;
    const T fc = ftrans(r, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
    T phi[kIn];
    features<T, false>(r, fc, dfc, phi, nullptr);
#pragma unroll
    for (int m = 0; m < kIn; ++m) G[m] += phi[m];
  }
}

// Forward pass; z (optional) receives z1, z2, z3 (3 x 64) for a backward pass.
template <typename T>
__device__ __forceinline__ T mlp_forward(const T* __restrict__ w, const T* G, T* z) {
  T x0[kIn];
#pragma unroll
  for (int k = 0; k < kIn; ++k) x0[k] = T(kSin) * G[k];
  T h1[kW], h2[kW];
#pragma unroll 4
  for (int j = 0; j < kW; ++j) {
    T s = w[oB1 + j];
#pragma unroll
    for (int k = 0; k < kIn; ++k) s += w[oW1 + j * kIn + k] * x0[k];
    if (z) z[j] = s;
    h1[j] = silu(s);
  }
#pragma unroll 4
  for (int j = 0; j < kW; ++j) {
    T s = w[oB2 + j];
#pragma unroll
    for (int k = 0; k < kW; ++k) s += w[oW2 + j * kW + k] * h1[k];
    if (z) z[kW + j] = s;
    h2[j] = silu(s);
  }
  T g = w[oB4];
#pragma unroll 4
  for (int j = 0; j < kW; ++j) {
    T s = w[oB3 + j];
#pragma unroll
    for (int k = 0; k < kW; ++k) s += w[oW3 + j * kW + k] * h2[k];
    if (z) z[2 * kW + j] = s;
    g += w[oW4 + j] * silu(s);
  }
  return g;
}

// d = dg_out * dg/d(z1, z2, z3) given the pre-activations z (3 x 64); writes d (3 x 64).
template <typename T>
__device__ __forceinline__ void mlp_backward_z(const T* __restrict__ w, const T* z, T dg, T* d) {
#pragma unroll 4
  for (int j = 0; j < kW; ++j) d[2 * kW + j] = dg * w[oW4 + j] * silu_d(z[2 * kW + j]);
#pragma unroll 4
  for (int k = 0; k < kW; ++k) {
    T s = T(0);
    for (int j = 0; j < kW; ++j) s += w[oW3 + j * kW + k] * d[2 * kW + j];
    d[kW + k] = s * silu_d(z[kW + k]);
  }
#pragma unroll 4
  for (int k = 0; k < kW; ++k) {
    T s = T(0);
    for (int j = 0; j < kW; ++j) s += w[oW2 + j * kW + k] * d[kW + j];
    d[k] = s * silu_d(z[k]);
  }
}

// Pass 1 of the learned switch: EAM density, energy and xi' (as k_pass1) and
// g_i = MLP(G_i), also into posg[i] in the FP32 path.  Weights are staged in
// shared memory per block.
template <typename T>
__global__ void __launch_bounds__(kLearnedBlock) k_pass1_learned(Args<T> a) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);
  __shared__ double sh[32];
  for (int k = threadIdx.x; k < APIP_MLP_NPARAM; k += blockDim.x) w[k] = a.mlp_w[k];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double e_out = 0.0;
  if (i < a.n) {
    const auto si = a.pv.self(i);
    const T rcE2 = a.k.eam_rc2;
    const T rc2 = a.ace_rc * a.ace_rc, inv_w = T(1) / (a.ace_rc - a.ace_rc_lo);
    Acc<T> zeta, pair;
    T G[kIn];
#pragma unroll
    for (int m = 0; m < kIn; ++m) G[m] = T(0);
    const int cnt = a.nnb[i];
    for (int s = 0; s < cnt; ++s) {
      const int j = a.nbl[(size_t)s * a.nmax + i];
      const auto d = a.pv.vec(si, j);
      const T r2 = dot3(d, d);
      if (!(r2 < rc2) && !(r2 < rcE2)) continue;
      const T r = sqrt(r2);
      if (r2 < rcE2) {
        T rho, phi;
        eam_terms(a.k, r, &rho, &phi);
        zeta.add(rho);
        pair.add(phi);
      }
      if (r2 < rc2) {
        T dfc;
        const T fc = ftrans(r, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
        T ph[kIn];
        features<T, false>(r, fc, dfc, ph, nullptr);
#pragma unroll
        for (int m = 0; m < kIn; ++m) G[m] += ph[m];
      }
    }
    const T zz = zeta.value();
    const T sz = zz > T(0) ? sqrt(zz) : T(0);
    const T e = -sz + T(0.5) * pair.value();
    a.zeta[i] = zz;
    a.xi_p[i] = zz > T(0) ? T(-0.5) / sz : T(0);
    a.e_eam[i] = e;
    const double e_ind = ind_energy(a, i);   // the external indenter, if any
    if (a.e_atom) a.e_atom[i] = (double)e + (double)e_ind;
    e_out = (double)e + (double)e_ind;
    const T g = mlp_forward<T>(w, G, nullptr);
    a.g[i] = g;
    if constexpr (sizeof(T) == 4) a.posg[i] = make_uint4(si.q.x, si.q.y, si.q.z, __float_as_uint(g));
  }
  const double tot = block_sum(e_out, sh);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
}

// ------------------------------------------------ pass 1, learned, float32
// The network on the tensor cores: mma.sync m16n8k16 with bfloat16 operands and
// float32 accumulation, a warp per tile of 32 atoms (two 16-row tiles).  Float32
// accuracy from bfloat16 products: every operand x is split as
// x = x_hi + x_mid + x_lo (each part the bfloat16 rounding of what the previous
// parts leave, 8 significant bits each, so 24 in all), and a product is the sum of
// the six part products whose orders add to at most 2 (hi hi, hi mid, mid hi,
// hi lo, mid mid, lo hi); the three dropped ones are below 2^-24 of the product.
// Part products are exact in float32 and accumulate in float32.
//
// Fragment layouts (PTX ISA, mma.m16n8k16 .bf16): with g = lane / 4, t = lane % 4,
// A (16 x 16, row-major) regs a0 = A[g][2t, 2t+1], a1 = A[g+8][2t, 2t+1],
// a2 = A[g][2t+8, 2t+9], a3 = A[g+8][2t+8, 2t+9]; B (16 x 8, k x n) regs
// b0 = B[2t, 2t+1][g], b1 = B[2t+8, 2t+9][g]; C (16 x 8) c0 = C[g][2t],
// c1 = C[g][2t+1], c2 = C[g+8][2t], c3 = C[g+8][2t+1]; the lower column sits in
// the low 16 bits of a pair.  The C fragments of n-tiles 2kb and 2kb+1 of one
// layer are the A fragment of k-block kb of the next: activations stay in
// registers from layer to layer.

// Compensated float32 dot product (the Dot2 scheme of Ogita, Rump and Oishi): s
// is the running sum, c the sum of the exact rounding errors of every product
// (from an FMA) and every addition (TwoSum); the value s + c is as accurate as a
// twice-as-wide accumulation.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v, bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ void fma(float a, float b) {
    const float p = a * b;
    c += fmaf(a, b, -p);
    add(p);
  }
  __device__ __forceinline__ void merge(float s2, float c2) {
    add(s2);
    c += c2;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// uint2 offsets of the layers within a split: layer 1 (2 k-blocks), 2 and 3 (4 each)
constexpr int kTcOff1 = 0, kTcOff2 = 2 * 8 * 32, kTcOff3 = kTcOff2 + 4 * 8 * 32;
constexpr int kTcSplit = kTcOff3 + 4 * 8 * 32;                              // 2560 uint2 per split
constexpr int kTcFrag = 3 * kTcSplit;                                       // hi, mid, lo
constexpr int kTcWarps = 8;
constexpr int kTcXs = 33;        // staging row stride (floats) of the layer-1 input: odd, so that
                                 // lanes adding at nearby Gaussian indices hit different banks
constexpr int kTcBias = 3 * kW + kW + 4;   // b1, b2, b3, w4, b4 (+ pad)

__device__ __forceinline__ uint32_t bf2(float lo_col, float hi_col) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// (x, y) -> the hi, mid, lo bfloat16 pairs of the three-way split.
__device__ __forceinline__ void split3(float x, float y, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(h);
  const float rx = x - hf.x, ry = y - hf.y;     // exact
  const __nv_bfloat162 m = __floats2bfloat162_rn(rx, ry);
  const float2 mf = __bfloat1622float2(m);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  mid = *reinterpret_cast<const uint32_t*>(&m);
  lo = bf2(rx - mf.x, ry - mf.y);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

// One k-block of a layer for all 8 n-tiles: acc[nt] += A_kb W^T, A given as its
// three parts (4 regs each), the weights' fragments from shared memory (layer
// offset lo_off, k-block kb); small part products first.  Product-major order:
// consecutive mma instructions update different n-tiles, so they overlap
// instead of waiting on one accumulator.
__device__ __forceinline__ void tc_kblock(float (*acc)[4], const uint32_t* ah, const uint32_t* am, const uint32_t* al,
                                          const uint2* sf, int lo_off, int kb, int lane) {
  const uint2* f = sf + lo_off + kb * 8 * 32 + lane;
  const uint32_t* const as[6] = {am, ah, al, ah, am, ah};
  constexpr int ws[6] = {1, 2, 0, 1, 0, 0};   // weight part: 0 hi, 1 mid, 2 lo
#pragma unroll
  for (int p = 0; p < 6; ++p)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[nt], as[p], f[ws[p] * kTcSplit + nt * 32]);
}

// acc (layer output, 8 n-tiles) -> bias + SiLU in place.
__device__ __forceinline__ void tc_bias_silu(float (*acc)[4], const float* b, int t) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[nt][q] = silu(acc[nt][q] + b[8 * nt + 2 * t + (q & 1)]);
}

// A 64-wide hidden layer: out = in W^T (in holds the previous activations).
__device__ __forceinline__ void tc_hidden(float (*in)[4], float (*out)[4], const uint2* sf, int lo_off, int lane) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int q = 0; q < 4; ++q) out[nt][q] = 0.f;
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    uint32_t ah[4], am[4], al[4];
    split3(in[2 * kb][0], in[2 * kb][1], ah[0], am[0], al[0]);
    split3(in[2 * kb][2], in[2 * kb][3], ah[1], am[1], al[1]);
    split3(in[2 * kb + 1][0], in[2 * kb + 1][1], ah[2], am[2], al[2]);
    split3(in[2 * kb + 1][2], in[2 * kb + 1][3], ah[3], am[3], al[3]);
    tc_kblock(out, ah, am, al, sf, lo_off, kb, lane);
  }
}

// The fragments of the split weights: thread f of kTcFrag writes uint2 f
// (split, layer, k-block, n-tile, lane) from the float32 weights.
__global__ void k_mlp_frags(const float* __restrict__ w, uint2* __restrict__ frag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= kTcFrag) return;
  const int sp = f / kTcSplit, r = f % kTcSplit;
  const int layer = r < kTcOff2 ? 0 : (r < kTcOff3 ? 1 : 2);
  const int q = r - (layer == 0 ? kTcOff1 : (layer == 1 ? kTcOff2 : kTcOff3));
  const int lane = q % 32, nt = (q / 32) % 8, kb = q / 256;
  const int K = layer == 0 ? kIn : kW;
  const float* W = w + (layer == 0 ? oW1 : (layer == 1 ? oW2 : oW3));
  const int n = 8 * nt + lane / 4, k0 = 16 * kb + 2 * (lane % 4);
  uint32_t v[2];
  for (int h = 0; h < 2; ++h) {
    uint32_t p[3];
    split3(W[n * K + k0 + 8 * h], W[n * K + k0 + 8 * h + 1], p[0], p[1], p[2]);
    v[h] = p[sp];
  }
  frag[f] = make_uint2(v[0], v[1]);
}

// Adds phi_m(r) (fc folded in) to row[m] for the Gaussians within kWin spacings
// of the nearest one, |r - mu_m| < 8.5 dmu = 0.96 A; the others are below
// exp(-eta (8.5 dmu)^2) = 1.3e-9 of the largest, under float32 rounding of the
// sum.  Same ratio recurrence as features() outward from the nearest Gaussian.
constexpr int kWin = 8;
__device__ __forceinline__ void add_features_window(float r, float fc, float kappa, float* row) {
  const float dmu = float(kDmu), eta = float(kEta);
  int m0 = __float2int_rn((r - float(kMu0)) / dmu);
  m0 = m0 < 0 ? 0 : (m0 > kIn - 1 ? kIn - 1 : m0);
  const float x0 = r - (float(kMu0) + float(m0) * dmu);
  const float base = -eta * dmu * dmu, slope = 2.f * eta * dmu * x0;
  const float e0 = __expf(-eta * x0 * x0) * fc;
  float rho = __expf(base + slope), sig = __expf(base - slope), up = e0, dn = e0;
  row[m0] += e0;
#pragma unroll
  for (int k = 1; k <= kWin; ++k) {
    up *= rho;
    rho *= kappa;
    dn *= sig;
    sig *= kappa;
    if (m0 + k < kIn) row[m0 + k] += up;
    if (m0 - k >= 0) row[m0 - k] += dn;
  }
}

// Pass 1 with the learned switch, float32: as k_pass1_learned (EAM density,
// energy, xi'; descriptors; g = MLP(G)) with the network on the tensor cores.
// Persistent blocks of 8 warps; warp w of block b takes the tiles of 32 atoms
// b * 8 + w, + 8 gridDim, ...; one energy partial per block.
__global__ void __launch_bounds__(kTcWarps * 32) k_pass1_learned_tc(Args<float> a, const uint2* __restrict__ frag) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint2* sf = reinterpret_cast<uint2*>(smem_raw);
  float* sb = reinterpret_cast<float*>(sf + kTcFrag);
  float* sx = sb + kTcBias;
  __shared__ double sh[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
  for (int k = tid; k < kTcFrag / 2; k += blockDim.x)
    reinterpret_cast<uint4*>(sf)[k] = reinterpret_cast<const uint4*>(frag)[k];
  for (int k = tid; k < kW; k += blockDim.x) {
    sb[k] = a.mlp_w[oB1 + k];
    sb[kW + k] = a.mlp_w[oB2 + k];
    sb[2 * kW + k] = a.mlp_w[oB3 + k];
    sb[3 * kW + k] = a.mlp_w[oW4 + k];
  }
  if (tid == 0) sb[4 * kW] = a.mlp_w[oB4];
  __syncthreads();
  float* xs = sx + warp * (32 * kTcXs + 32);   // [32][kTcXs] layer-1 input, then g of the 32 atoms
  float* gs = xs + 32 * kTcXs;
  const float rcE2 = a.k.eam_rc2;
  const float rc2 = a.ace_rc * a.ace_rc, inv_w = 1.f / (a.ace_rc - a.ace_rc_lo);
  const float kappa = __expf(-2.f * float(kEta) * float(kDmu) * float(kDmu));
  float* xrow = xs + lane * kTcXs;   // this lane's atom: descriptors accumulate here
  double e_out = 0.0;
  const int ntiles = (a.n + 31) / 32;
  for (int tile = blockIdx.x * kTcWarps + warp; tile < ntiles; tile += gridDim.x * kTcWarps) {
    const int i = tile * 32 + lane;
    const bool act = i < a.n;
#pragma unroll
    for (int m = 0; m < kIn; ++m) xrow[m] = 0.f;
    if (act) {
      const auto si = a.pv.self(i);
      Acc<float> zeta, pair;
      walk_list(a.nbl + i, a.nmax, 0, a.nnb[i], [&](int j) { return a.pv.fetch(j); },
                [&](int, const uint4& o) {
                  const auto d = a.pv.vec_of(si, o);
                  const float r2 = dot3(d, d);
                  if (!(r2 < rc2) && !(r2 < rcE2)) return;
                  const float r = sqrtf(r2);
                  if (r2 < rcE2) {
                    float rho, phi;
                    eam_terms(a.k, r, &rho, &phi);
                    zeta.add(rho);
                    pair.add(phi);
                  }
                  if (r2 < rc2) {
                    float dfc;
                    const float fc = ftrans(r, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
                    add_features_window(r, fc, kappa, xrow);
                  }
                });
      const float zz = zeta.value();
      const float sz = zz > 0.f ? sqrtf(zz) : 0.f;
      const float e = -sz + 0.5f * pair.value();
      a.zeta[i] = zz;
      a.xi_p[i] = zz > 0.f ? -0.5f / sz : 0.f;
      a.e_eam[i] = e;
      const double e_ind = ind_energy(a, i);   // the external indenter, if any
      if (a.e_atom) a.e_atom[i] = (double)e + (double)e_ind;
      e_out += (double)e + (double)e_ind;
    }
#pragma unroll
    for (int m = 0; m < kIn; ++m) xrow[m] *= float(kSin);
    __syncwarp();
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = 16 * mt + gq, r1 = r0 + 8;
      float h1[8][4], h2[8][4];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) h1[nt][q] = 0.f;
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        const int c = 16 * kb + 2 * tq;
        uint32_t ah[4], am[4], al[4];
        split3(xs[r0 * kTcXs + c], xs[r0 * kTcXs + c + 1], ah[0], am[0], al[0]);
        split3(xs[r1 * kTcXs + c], xs[r1 * kTcXs + c + 1], ah[1], am[1], al[1]);
        split3(xs[r0 * kTcXs + c + 8], xs[r0 * kTcXs + c + 9], ah[2], am[2], al[2]);
        split3(xs[r1 * kTcXs + c + 8], xs[r1 * kTcXs + c + 9], ah[3], am[3], al[3]);
        tc_kblock(h1, ah, am, al, sf, kTcOff1, kb, lane);
      }
      tc_bias_silu(h1, sb, tq);
      tc_hidden(h1, h2, sf, kTcOff2, lane);
      tc_bias_silu(h2, sb + kW, tq);
      tc_hidden(h2, h1, sf, kTcOff3, lane);
      // output: g = b4 + sum_j w4_j SiLU(z3_j + b3_j), rows r0 (q = 0, 1) and r1 (q = 2, 3),
      // a compensated dot product: each product split exactly (FMA) and each sum
      // with its rounding error (TwoSum) carried in a second float, so that the
      // cancelling terms of the output layer add no rounding of their own
      Dot2 d0, d1;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int col = 8 * nt + 2 * tq + (q & 1);
          const float w = sb[3 * kW + col], h = silu(h1[nt][q] + sb[2 * kW + col]);
          if (q < 2) d0.fma(w, h); else d1.fma(w, h);
        }
#pragma unroll
      for (int o = 1; o <= 2; o <<= 1) {
        d0.merge(__shfl_xor_sync(0xffffffffu, d0.s, o), __shfl_xor_sync(0xffffffffu, d0.c, o));
        d1.merge(__shfl_xor_sync(0xffffffffu, d1.s, o), __shfl_xor_sync(0xffffffffu, d1.c, o));
      }
      if (tq == 0) {
        d0.merge(sb[4 * kW], 0.f);
        d1.merge(sb[4 * kW], 0.f);
        gs[r0] = d0.value();
        gs[r1] = d1.value();
      }
    }
    __syncwarp();
    if (act) {
      const float g = gs[lane];
      a.g[i] = g;
      const uint4 q = a.posq[i];
      a.posg[i] = make_uint4(q.x, q.y, q.z, __float_as_uint(g));
    }
    __syncwarp();   // xs and gs are rewritten by the next tile
  }
  const double tot = block_sum(e_out, sh);
  if (tid == 0) a.partials[blockIdx.x] = tot;
}

size_t tc_smem_bytes() {
  return sizeof(uint2) * kTcFrag + sizeof(float) * (kTcBias + kTcWarps * (32 * kTcXs + 32));
}

// -grad sum_k c_k g_k for the atoms with c_k != 0 (learned counterpart of
// k_csp_force): dG_km = c_k dg_k/dG_km by back-propagation, then for each
// neighbour j: v = sum_m dG_km phi_m'(r_kj), F_j -= v e_kj, F_k += v e_kj.
// Here for one atom k of the compacted list; resets c_k.
template <typename T>
__device__ __forceinline__ void mlp_force_atom(const Args<T>& a, int k) {
  const double c = a.cvec[k];
  a.cvec[k] = 0.0;
  T G[kIn];
  descriptors_of(a, k, G);
  T z[3 * kW], d[3 * kW];
  mlp_forward<T>(a.mlp_w, G, z);
  mlp_backward_z<T>(a.mlp_w, z, T(c), d);
  T dG[kIn];
#pragma unroll 4
  for (int m = 0; m < kIn; ++m) {
    T s = T(0);
    for (int j = 0; j < kW; ++j) s += a.mlp_w[oW1 + j * kIn + m] * d[j];
    dG[m] = T(kSin) * s;
  }
  const auto sk = a.pv.self(k);
  const T rc2 = a.ace_rc * a.ace_rc, inv_w = T(1) / (a.ace_rc - a.ace_rc_lo);
  const int cnt = a.nnb[k];
  double fk[3] = {0.0, 0.0, 0.0};
  for (int s = 0; s < cnt; ++s) {
    const int j = a.nbl[(size_t)s * a.nmax + k];
    const auto dv = a.pv.vec(sk, j);
    const T r2 = dot3(dv, dv);
    if (!(r2 < rc2)) continue;
    const T r = sqrt(r2);
    T dfc;
    const T fc = ftrans(r, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
    T phi[kIn], dphi[kIn];
    features<T, true>(r, fc, dfc, phi, dphi);
    T v = T(0);
#pragma unroll
    for (int m = 0; m < kIn; ++m) v += dG[m] * dphi[m];
    const T ir = T(1) / r;
    const double f0 = (double)(v * dv.x * ir), f1 = (double)(v * dv.y * ir), f2 = (double)(v * dv.z * ir);
    atomicAdd(&a.force[3 * j], -f0);
    atomicAdd(&a.force[3 * j + 1], -f1);
    atomicAdd(&a.force[3 * j + 2], -f2);
    fk[0] += f0; fk[1] += f1; fk[2] += f2;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) atomicAdd(&a.force[3 * k + q], fk[q]);
}

// The atoms with c_k != 0 in warp-ballot order (counts[1] of them), so that the
// force kernel's warps are full: c is nonzero only near the transition region.
template <typename T>
__global__ void __launch_bounds__(256) k_cvec_compact(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool pred = i < a.n && a.cvec[i] != 0.0;
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(&a.counts[1], __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) a.clist[base + __popc(mask & ((1u << lane) - 1u))] = i;
}

template <typename T>
__global__ void __launch_bounds__(128) k_mlp_force(Args<T> a) {
  pdl_begin();
  const int count = a.counts[1];
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
    mlp_force_atom(a, a.clist[q]);
}

template <typename T>
__global__ void k_descriptors(Args<T> a, __nv_bfloat16* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  T G[kIn];
  descriptors_of(a, i, G);
#pragma unroll
  for (int m = 0; m < kIn; ++m) out[(size_t)i * kIn + m] = __float2bfloat16_rn((float)G[m]);
}

template <typename T>
__global__ void k_cast_params(const float* src, T* dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < APIP_MLP_NPARAM) dst[k] = (T)src[k];
}

// ------------------------------------------------------------------ Adam
__global__ void k_adam(float* p, const float* g, float* m, float* v, int t, float lr) {
  pdl_begin();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= APIP_MLP_NPARAM) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / (1.0f - powf(b1, (float)t));
  const float vh = vk / (1.0f - powf(b2, (float)t));
  p[k] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

// float64: the per-thread network, one 128-atom block per partial; float32: the
// tensor-core kernel on a.n_part_p1 persistent blocks (learned_tc_grid)
template <typename T> void launch_pass1_learned(const Args<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    const size_t bytes = tc_smem_bytes();
    cudaFuncSetAttribute(k_pass1_learned_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    launch_pdl(k_pass1_learned_tc, a.n_part_p1, kTcWarps * 32, bytes, s, a, a.mlp_frag);
  } else {
    const size_t bytes = sizeof(T) * APIP_MLP_NPARAM;
    cudaFuncSetAttribute(k_pass1_learned<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    launch_pdl(k_pass1_learned<T>, (a.n + kLearnedBlock - 1) / kLearnedBlock, kLearnedBlock, bytes, s, a);
  }
}

int learned_tc_slots() {
  const size_t bytes = tc_smem_bytes();
  if (cudaFuncSetAttribute(k_pass1_learned_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return 0;
  int occ = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pass1_learned_tc, kTcWarps * 32, bytes) != cudaSuccess)
    return 0;
  return occ * sms;
}

int learned_tc_blocks(int n, int slots) {
  const int need = (n + kTcWarps * 32 - 1) / (kTcWarps * 32);
  return need < 1 ? 1 : (need < slots ? need : slots);
}

void launch_mlp_frags(const float* w, void* frag, cudaStream_t s) {
  k_mlp_frags<<<(kTcFrag + 255) / 256, 256, 0, s>>>(w, reinterpret_cast<uint2*>(frag));
}

size_t mlp_frag_bytes() { return sizeof(uint2) * kTcFrag; }

template <typename T> void launch_mlp_force(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_cvec_compact<T>, (a.n + 255) / 256, 256, 0, s, a);
  int blocks = (a.n + 127) / 128;   // the list holds at most n atoms; a grid-stride loop covers it
  if (blocks > 2048) blocks = 2048;
  launch_pdl(k_mlp_force<T>, blocks, 128, 0, s, a);
}

template <typename T> void launch_descriptors(const Args<T>& a, uint16_t* out, cudaStream_t s) {
  k_descriptors<T><<<(a.n + 127) / 128, 128, 0, s>>>(a, reinterpret_cast<__nv_bfloat16*>(out));
}

template <typename T> void launch_cast_params(const float* src, T* dst, cudaStream_t s) {
  k_cast_params<T><<<(APIP_MLP_NPARAM + 255) / 256, 256, 0, s>>>(src, dst);
}

void launch_mlp_adam(float* p, const float* g, float* m, float* v, int t, float lr, cudaStream_t s) {
  launch_pdl(k_adam, (APIP_MLP_NPARAM + 255) / 256, 256, 0, s, p, g, m, v, t, lr);
}

template void launch_pass1_learned<float>(const Args<float>&, cudaStream_t);
template void launch_pass1_learned<double>(const Args<double>&, cudaStream_t);
template void launch_mlp_force<float>(const Args<float>&, cudaStream_t);
template void launch_mlp_force<double>(const Args<double>&, cudaStream_t);
template void launch_descriptors<float>(const Args<float>&, uint16_t*, cudaStream_t);
template void launch_descriptors<double>(const Args<double>&, uint16_t*, cudaStream_t);
template void launch_cast_params<float>(const float*, float*, cudaStream_t);
template void launch_cast_params<double>(const float*, double*, cudaStream_t);

}  // namespace apip
