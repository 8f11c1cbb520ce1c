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
#include "tc_common.cuh"

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
  const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
  for (int s = 0; s < cnt; ++s) {
    const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
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
    const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
    for (int s = 0; s < cnt; ++s) {
      const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
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

// ------------------------------------- learned switch, float32, tensor cores
// The network on the fifth-generation tensor cores (tcgen05.mma, bfloat16
// operands, float32 accumulation in tensor memory), one kernel for both uses:
//   pass 1 (FORCE = false): for every atom the EAM density, energy and xi'
//     (as k_pass1) and g = MLP(G) (also into posg);
//   the grad-lambda force (FORCE = true): for the atoms with c_k != 0 (the list
//     k_cvec_compact builds), dG_k = c_k dg/dG by back-propagation through the
//     same network, then F_j -= v e_kj, F_k += v e_kj per neighbour with
//     v = sum_m dG_km phi_m'(r_kj) (Eq. 6 with a general g: -grad sum_k c_k g_k).
// Float32 accuracy from bfloat16 products: every operand x (activation or
// weight) is split as x = x_hi + x_mid + x_lo, each part the bfloat16 rounding of
// what the previous parts leave (8 significant bits each, 24 in all), and a
// product is the sum of the six part products whose orders add to at most 2
// (mid mid, hi lo, lo hi, hi mid, mid hi, hi hi, small ones first); the three
// dropped ones are below 2^-24 of the product.  Part products are exact in
// float32 and accumulate in float32 in tensor memory.
//
// A persistent CTA of 512 threads per SM loops over tiles of 128 atoms: atom row
// r of a tile is tensor-memory lane r; thread (warp w, lane l) owns row
// r = 32 (w % 4) + l and quarter cg = w / 4 of the work of that row: neighbour
// entries cg, cg + 4, ... of the atom's list, descriptor columns 8 cg .. + 7 and
// columns 16 cg .. + 15 of each 64-wide layer.  Per tile, with D = A B^T:
//   z1 = x0 W1^T, z2 = h1 W2^T, z3 = h2 W3^T                (forward)
//   dh2 = dz3 W3, dh1 = dz2 W2, dG = dz1 W1                 (FORCE: back-propagation;
//                                                            the weights read MN-major)
// The forward epilogues keep silu'(z) in the tensor-memory columns of z for the
// back-propagation.  The output layer g = b4 + sum_j w4_j silu(z3_j + b3_j) is a
// compensated dot product on the CUDA cores.  The weight images (three parts,
// chunk-major with 64 rows; tc_common.cuh) are built once per apip_set_mlp by
// k_mlp_images and copied into shared memory by each CTA.
//
// Every tensor-memory load and store is executed by whole warps on their own
// quarter of the lanes, never under a branch that splits a warp.  One thread
// issues the MMAs, committed to an mbarrier that every thread waits on; every
// wait is bounded (two seconds): on time-out the kernel records ST_TIMEOUT, stops
// issuing, leaves the tile loop, waits once more for the MMAs in flight, frees
// its tensor memory and returns.
namespace lt {
using namespace tc;
constexpr int kT = 512;                    // threads per CTA: four per atom
constexpr int kRows = 128;                 // atoms per tile = tensor-memory lanes
constexpr int kImgW1 = kW * kIn * 2, kImgW2 = kW * kW * 2;   // bytes of a weight image part
constexpr int kImgPart = kImgW1 + 2 * kImgW2;                // W1 | W2 | W3 of one part
constexpr int kImg = 3 * kImgPart;                           // hi, mid, lo
constexpr int kXPart = kRows * kIn * 2, kHPart = kRows * kW * 2;
constexpr int kPs = kIn + 1;               // stride (floats) of a descriptor partial row
// shared memory (byte offsets)
constexpr int sW = 0;                      // weight images
constexpr int sX = sW + kImg;              // x0 = G / 4, three parts
constexpr int sH = sX + 3 * kXPart;        // a 64-wide activation or gradient, three parts
constexpr int sP = sH + 3 * kHPart;        // descriptor partials [4][128][33]; FORCE: dG rows [128][33]
constexpr int sF = sP + 4 * kRows * kPs * 4;   // float32 b1, b2, b3, w4, b4 (+ pad)
constexpr int kNF = 4 * kW + 4;
constexpr int sE = sF + kNF * 4;           // pass 1: EAM partials [4][128][4]; FORCE: c of each row
constexpr int sG = sE + 4 * kRows * 4 * 4; // output-layer partials [4][128][2]
constexpr int kSmem = sG + 4 * kRows * 2 * 4;
static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(kImgPart % 1024 == 0 && sX % 1024 == 0 && sH % 1024 == 0 && sP % 16 == 0, "alignment");
// pass 1 (network only; the descriptors come from k_learned_desc): weights, one
// 64-wide activation region (which also holds the split x0 before layer 1 and
// the output-layer partials after layer 3), the float32 parameters; two CTAs per
// SM, 256 tensor-memory columns each
constexpr int sHm = sW + kImg;
constexpr int sFm = sHm + 3 * kHPart;
constexpr int kSmemM = sFm + kNF * 4;
static_assert(2 * (kSmemM + 2048) <= 228 * 1024, "two CTAs per SM");
static_assert(3 * kXPart <= 3 * kHPart && 4 * kRows * 2 * 4 <= 3 * kHPart, "aliases within the activation region");
// tensor-memory columns
constexpr uint32_t cZ1 = 0, cZ2 = 64, cZ3 = 128, cDH = 192, cDG = 256;
}  // namespace lt

// Weight images for the tensor-core kernel: part p of W1, W2, W3 (bfloat16,
// chunk-major with 64 rows) at p * kImgPart; thread e converts the pair of
// elements (row, 2c), (row, 2c + 1) of one matrix.
__global__ void k_mlp_images(const float* __restrict__ w, unsigned char* __restrict__ img) {
  using namespace lt;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  constexpr int n1 = kW * kIn / 2, n2 = kW * kW / 2;
  if (e >= n1 + 2 * n2) return;
  int m, q;   // matrix (0: W1, 1: W2, 2: W3), pair index within it
  if (e < n1) { m = 0; q = e; } else if (e < n1 + n2) { m = 1; q = e - n1; } else { m = 2; q = e - n1 - n2; }
  const int K = m == 0 ? kIn : kW;
  const int row = (2 * q) / K, col = (2 * q) % K;
  const float* W = w + (m == 0 ? oW1 : (m == 1 ? oW2 : oW3));
  uint32_t part[3];
  split3(W[row * K + col], W[row * K + col + 1], part[0], part[1], part[2]);
  const int off = (m == 0 ? 0 : (m == 1 ? kImgW1 : kImgW1 + kImgW2)) + tc::chunk_off(row, col, kW);
#pragma unroll
  for (int p = 0; p < 3; ++p) *reinterpret_cast<uint32_t*>(img + p * kImgPart + off) = part[p];
}

// Sixteen float32 values, split in three, into row r of the three parts of a
// 128-row chunk-major operand at column c0 (a multiple of 8): two 16-byte stores
// per part.
__device__ __forceinline__ void put16_split(unsigned char* base, int part_bytes, int r, int c0, const float* v) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint4 w[3];
    uint32_t* u0 = reinterpret_cast<uint32_t*>(&w[0]);
    uint32_t* u1 = reinterpret_cast<uint32_t*>(&w[1]);
    uint32_t* u2 = reinterpret_cast<uint32_t*>(&w[2]);
#pragma unroll
    for (int q = 0; q < 4; ++q) split3(v[8 * h + 2 * q], v[8 * h + 2 * q + 1], u0[q], u1[q], u2[q]);
    const int off = tc::chunk_off(r, c0 + 8 * h, lt::kRows);
#pragma unroll
    for (int p = 0; p < 3; ++p) *reinterpret_cast<uint4*>(base + p * part_bytes + off) = w[p];
  }
}

// D (column d) = A B^T with both operands given as three parts (addresses of
// part 0; parts pa_bytes / pb_bytes apart): the six part products, small first.
__device__ __forceinline__ void mma_split(uint32_t tmem, uint32_t d, tc::Opnd A, int pa_bytes, tc::Opnd B,
                                          int pb_bytes, int K, uint32_t id) {
  constexpr int ap[6] = {1, 0, 2, 0, 1, 0}, bp[6] = {1, 2, 0, 1, 0, 0};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    tc::Opnd a = A, b = B;
    a.addr += ap[q] * pa_bytes;
    b.addr += bp[q] * pb_bytes;
    tc::mma(tmem, d, a, b, K, id, q > 0);
  }
}

// phi_m(r) (fc folded in) for the Gaussians within kWin spacings of the nearest
// one, as add_features_window, and their derivatives contracted with dG:
// returns v = sum_m dG[m] d phi_m / dr (the other Gaussians are below 1.3e-9 of
// the largest).
__device__ __forceinline__ float dfeatures_window(float r, float fc, float dfc, float kappa, const float* dG) {
  const float dmu = float(kDmu), eta = float(kEta);
  int m0 = __float2int_rn((r - float(kMu0)) / dmu);
  m0 = m0 < 0 ? 0 : (m0 > kIn - 1 ? kIn - 1 : m0);
  const float x0 = r - (float(kMu0) + float(m0) * dmu);
  const float base = -eta * dmu * dmu, slope = 2.f * eta * dmu * x0;
  const float e0 = __expf(-eta * x0 * x0);
  float rho = __expf(base + slope), sig = __expf(base - slope), up = e0, dn = e0;
  const float a2 = -2.f * eta * fc;
  float v = dG[m0] * e0 * (a2 * x0 + dfc);
#pragma unroll
  for (int k = 1; k <= kWin; ++k) {
    up *= rho;
    rho *= kappa;
    dn *= sig;
    sig *= kappa;
    if (m0 + k < kIn) v += dG[m0 + k] * up * (a2 * (x0 - float(k) * dmu) + dfc);
    if (m0 - k >= 0) v += dG[m0 - k] * dn * (a2 * (x0 + float(k) * dmu) + dfc);
  }
  return v;
}

// Pass 1 of the learned switch, float32, CUDA-core part: one thread per atom
// walks its list for the EAM density, energy and xi' (as k_pass1) and the radial
// descriptors, accumulated in the thread's shared-memory row (odd stride: the
// lanes add at nearby Gaussian indices in different banks), and writes
// x0 = G / 4 (float32, 32 per atom) for the network (k_learned_tc<false>).
__global__ void __launch_bounds__(kBlock) k_learned_desc(Args<float> a, float* __restrict__ x0) {
  pdl_begin();
  __shared__ float rows[kBlock * (kIn + 1)];
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float* row = rows + threadIdx.x * (kIn + 1);
#pragma unroll
  for (int m = 0; m < kIn; ++m) row[m] = 0.f;
  double e_out = 0.0;
  if (i < a.n) {
    const auto si = a.pv.self(i);
    const float rcE2 = a.k.eam_rc2;
    const float rc2 = a.ace_rc * a.ace_rc, inv_w = 1.f / (a.ace_rc - a.ace_rc_lo);
    const float kappa = __expf(-2.f * float(kEta) * float(kDmu) * float(kDmu));
    Acc<float> zeta, pair;
    walk_list(a.nbl + i, a.nmax, 0, APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1), a.status, a.n, [&](int j) { return a.pv.fetch(j); },
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
                  add_features_window(r, fc, kappa, row);
                }
              });
    const float zz = zeta.value();
    const float sz = zz > 0.f ? sqrtf(zz) : 0.f;
    const float e = -sz + 0.5f * pair.value();
    a.zeta[i] = zz;
    a.xi_p[i] = zz > 0.f ? -0.5f / sz : 0.f;
    a.e_eam[i] = e;
    const double e_ind = ind_energy(a, i);   // the external indenter, if any
    if (a.e_atom) a.e_atom[i] = (double)e + e_ind;
    e_out = (double)e + e_ind;
    float4* xo = reinterpret_cast<float4*>(x0 + (size_t)i * kIn);
#pragma unroll
    for (int m = 0; m < kIn / 4; ++m)
      xo[m] = make_float4(kSin * row[4 * m], kSin * row[4 * m + 1], kSin * row[4 * m + 2], kSin * row[4 * m + 3]);
  }
  const double tot = block_sum(e_out, sh);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
}

// FORCE = false: pass 1's network on x0 from k_learned_desc, two CTAs per SM
// (256 tensor-memory columns each; the split x0 and the output-layer partials
// share the activation region); FORCE = true: descriptors, network and
// back-propagation for the compacted atoms, one CTA per SM (512 columns).
template <bool FORCE>
__global__ void __launch_bounds__(lt::kT, FORCE ? 1 : 2)
    k_learned_tc(Args<float> a, const uint4* __restrict__ img, const float* __restrict__ x0) {
  using namespace lt;
  constexpr int oX = FORCE ? sX : sHm, oH = FORCE ? sH : sHm, oF = FORCE ? sF : sFm, oG = FORCE ? sG : sHm;
  constexpr uint32_t kCols = FORCE ? 512u : 256u;
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_holder;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, cg = warp >> 2;
  const int r = 32 * quarter + lane;    // this thread's atom row (tensor-memory lane)
  const int c0 = 16 * cg;               // its columns of a 64-wide layer
  // everything below may read what the previous kernel wrote
  pdl_begin();
  const int count = FORCE ? a.counts[1] : a.n;
  const int ntiles = (count + kRows - 1) / kRows;
  if ((int)blockIdx.x >= ntiles) return;   // no tile for this CTA (uniform): nothing allocated
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int k = tid; k < kImg / 16; k += kT) reinterpret_cast<uint4*>(sm + sW)[k] = img[k];
  float* fb = reinterpret_cast<float*>(sm + oF);
  if (tid < kNF) {
    const int q = tid / kW, c = tid % kW;
    const int src = q == 0 ? oB1 : q == 1 ? oB2 : q == 2 ? oB3 : oW4;
    fb[tid] = tid < 4 * kW ? a.mlp_w[src + c] : (tid == 4 * kW ? a.mlp_w[oB4] : 0.f);
  }
  to_mma();
  const uint32_t tm = tmem_holder;
  const uint32_t lane_addr = tm + ((uint32_t)(32 * quarter) << 16);
  float* P = reinterpret_cast<float*>(sm + sP);           // FORCE: descriptor partials [cg][row][kPs], then dG rows
  float* C1 = reinterpret_cast<float*>(sm + sE);          // FORCE: c of each row
  float* G2 = reinterpret_cast<float*>(sm + oG);          // pass 1: output-layer partials [cg][row][2]
  const uint32_t id64 = idesc(kW, false, false), id_b64 = idesc(kW, false, true), id_b32 = idesc(kIn, false, true);
  const float rc2 = a.ace_rc * a.ace_rc, inv_w = 1.f / (a.ace_rc - a.ace_rc_lo);
  const float kappa = __expf(-2.f * float(kEta) * float(kDmu) * float(kDmu));
  uint32_t phase = 0;
  int fail_par = -1;
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
  // forward epilogue of one layer: h = silu(z + b) (split) into the activation
  // region; FORCE keeps silu'(z + b) in the tensor-memory columns of z
  auto forward = [&](uint32_t col, const float* bias) {
    float z[16], d[16];
    tld16(lane_addr + col + c0, z);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float u = z[q] + bias[c0 + q];
      const float sg = 1.f / (1.f + __expf(-u));
      d[q] = sg * (1.f + u * (1.f - sg));
      z[q] = u * sg;
    }
    put16_split(sm + oH, kHPart, r, c0, z);
    if (FORCE) tst16(lane_addr + col + c0, d);
  };
  // backward epilogue: dz = dh silu'(z) (split) into the activation region
  auto backward = [&](uint32_t zcol) {
    float dh[16], d[16];
    tld16(lane_addr + cDH + c0, dh);
    tld16(lane_addr + zcol + c0, d);
#pragma unroll
    for (int q = 0; q < 16; ++q) dh[q] *= d[q];
    put16_split(sm + oH, kHPart, r, c0, dh);
  };
  // x0 columns 8 cg .. + 7 of row r, split, into the layer-1 operand
  auto put_x0 = [&](const float* x) {
    uint4 w[3];
    uint32_t* u0 = reinterpret_cast<uint32_t*>(&w[0]);
    uint32_t* u1 = reinterpret_cast<uint32_t*>(&w[1]);
    uint32_t* u2 = reinterpret_cast<uint32_t*>(&w[2]);
#pragma unroll
    for (int m = 0; m < 4; ++m) split3(x[2 * m], x[2 * m + 1], u0[m], u1[m], u2[m]);
    const int off = chunk_off(r, 8 * cg, kRows);
#pragma unroll
    for (int p = 0; p < 3; ++p) *reinterpret_cast<uint4*>(sm + oX + p * kXPart + off) = w[p];
  };

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int q = tile * kRows + r;
    const bool valid = q < count;
    const int i = valid ? (FORCE ? APIP_CHK(a.status, BND_COMPACT, a.clist[q], a.n) : q) : -1;
    if constexpr (!FORCE) {
      // x0 of this row from the descriptor kernel (zero past the atoms)
      float x[8];
      const float4* xi = reinterpret_cast<const float4*>(x0 + (size_t)(valid ? i : 0) * kIn + 8 * cg);
      const float4 v0 = valid ? xi[0] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 v1 = valid ? xi[1] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w; x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
      put_x0(x);
    } else {
      // ---- descriptors over this thread's entries
      float* prow = P + (cg * kRows + r) * kPs;
#pragma unroll
      for (int m = 0; m < kIn; ++m) prow[m] = 0.f;
      if (valid) {
        const auto si = a.pv.self(i);
        const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
        for (int s = cg; s < cnt; s += 4) {
          const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
          const auto d = a.pv.vec(si, j);
          const float r2 = dot3(d, d);
          if (!(r2 < rc2)) continue;
          const float rr = sqrtf(r2);
          float dfc;
          const float fc = ftrans(rr, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
          add_features_window(rr, fc, kappa, prow);
        }
      }
      if (cg == 0) {
        float c = 0.f;
        if (valid) {
          c = (float)fix_get(&a.cvec[i], a.det);
          a.cvec[i] = 0.0;
        }
        C1[r] = c;
      }
      __syncthreads();
      // G columns 8 cg .. + 7: the four partial rows in a fixed order; x0 = G / 4
      float x[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float* pr = P + r * kPs + 8 * cg + m;
        x[m] = kSin * ((pr[0] + pr[kRows * kPs]) + (pr[2 * kRows * kPs] + pr[3 * kRows * kPs]));
      }
      put_x0(x);
    }
    // ---- forward
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cZ1, act_k(sm + oX), kXPart, wt_k(sm + sW), kImgPart, kIn, id64); });
    forward(cZ1, fb);
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cZ2, act_k(sm + oH), kHPart, wt_k(sm + sW + kImgW1), kImgPart, kW, id64); });
    forward(cZ2, fb + kW);
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cZ3, act_k(sm + oH), kHPart, wt_k(sm + sW + kImgW1 + kImgW2), kImgPart, kW, id64); });
    {
      // layer 3 and this quarter's part of the output layer (compensated); FORCE:
      // dz3 = c w4 silu'(z3 + b3) (split) into the activation region
      float z[16];
      tld16(lane_addr + cZ3 + c0, z);
      Dot2 dg;
      float dz[16];
      const float c = FORCE ? C1[r] : 0.f;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float u = z[k] + fb[2 * kW + c0 + k];
        const float sg = 1.f / (1.f + __expf(-u));
        const float w4 = fb[3 * kW + c0 + k];
        if (FORCE) dz[k] = c * w4 * (sg * (1.f + u * (1.f - sg)));
        else dg.fma(w4, u * sg);
      }
      if (FORCE) {
        put16_split(sm + oH, kHPart, r, c0, dz);
      } else {
        G2[(cg * kRows + r) * 2] = dg.s;
        G2[(cg * kRows + r) * 2 + 1] = dg.c;
      }
    }
    if constexpr (!FORCE) {
      __syncthreads();
      if (cg == 0 && valid) {
        Dot2 t;
        t.merge(fb[4 * kW], 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) t.merge(G2[(k * kRows + r) * 2], G2[(k * kRows + r) * 2 + 1]);
        const float g = t.value();
        a.g[i] = g;
        const uint4 pq = a.posq[i];
        a.posg[i] = make_uint4(pq.x, pq.y, pq.z, __float_as_uint(g));
      }
      __syncthreads();   // the next tile rewrites the partials' region (its x0)
      continue;
    }
    // ---- back-propagation (FORCE)
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cDH, act_k(sm + oH), kHPart, wt_mn(sm + sW + kImgW1 + kImgW2), kImgPart, kW, id_b64); });
    backward(cZ2);
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cDH, act_k(sm + oH), kHPart, wt_mn(sm + sW + kImgW1), kImgPart, kW, id_b64); });
    backward(cZ1);
    to_mma();
    if (failed) break;
    run([&] { mma_split(tm, cDG, act_k(sm + oH), kHPart, wt_mn(sm + sW), kImgPart, kW, id_b32); });
    {
      // dG columns 8 cg .. + 7 (times the input scale) into row r of the dG rows
      float v[8];
      tld8(lane_addr + cDG + 8 * cg, v);
#pragma unroll
      for (int m = 0; m < 8; ++m) P[r * kPs + 8 * cg + m] = kSin * v[m];
    }
    __syncthreads();
    if (valid) {
      // the force of this thread's neighbour entries
      const float* dG = P + r * kPs;
      const auto sk = a.pv.self(i);
      const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
      double fk[3] = {0.0, 0.0, 0.0};
      for (int s = cg; s < cnt; s += 4) {
        const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
        const auto d = a.pv.vec(sk, j);
        const float r2 = dot3(d, d);
        if (!(r2 < rc2)) continue;
        const float rr = sqrtf(r2);
        float dfc;
        const float fc = ftrans(rr, a.ace_rc_lo, a.ace_rc, inv_w, &dfc);
        const float v = dfeatures_window(rr, fc, dfc, kappa, dG) / rr;
        const double f0 = (double)(v * d.x), f1 = (double)(v * d.y), f2 = (double)(v * d.z);
        scatter_add(&a.force[3 * j], -f0, a.det);
        scatter_add(&a.force[3 * j + 1], -f1, a.det);
        scatter_add(&a.force[3 * j + 2], -f2, a.det);
        fk[0] += f0; fk[1] += f1; fk[2] += f2;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) scatter_add(&a.force[3 * i + k], fk[k], a.det);
    }
    __syncthreads();   // the next tile rewrites the dG rows (partial rows) and c
  }
  __syncthreads();   // `failed` is uniform from here on
  if (failed && tid == 0) {
    atomicOr(&a.status[ST_TIMEOUT], 1);
    if (fail_par >= 0) wait_phase(&bar, (uint32_t)fail_par);   // the MMAs in flight, once more (bounded)
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kCols));
}

// -grad sum_k c_k g_k for the atoms with c_k != 0 (learned counterpart of
// k_csp_force): dG_km = c_k dg_k/dG_km by back-propagation, then for each
// neighbour j: v = sum_m dG_km phi_m'(r_kj), F_j -= v e_kj, F_k += v e_kj.
// Here for one atom k of the compacted list; resets c_k.
template <typename T>
__device__ __forceinline__ void mlp_force_atom(const Args<T>& a, int k) {
  const double c = fix_get(&a.cvec[k], a.det);
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
  const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[k], a.max_nb + 1);
  double fk[3] = {0.0, 0.0, 0.0};
  for (int s = 0; s < cnt; ++s) {
    const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + k], a.n);
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
    scatter_add(&a.force[3 * j], -f0, a.det);
    scatter_add(&a.force[3 * j + 1], -f1, a.det);
    scatter_add(&a.force[3 * j + 2], -f2, a.det);
    fk[0] += f0; fk[1] += f1; fk[2] += f2;
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) scatter_add(&a.force[3 * k + q], fk[q], a.det);
}

// The atoms with c_k != 0 in warp-ballot order (counts[1] of them), so that the
// force kernel's warps are full: c is nonzero only near the transition region.
template <typename T>
__global__ void __launch_bounds__(256) k_cvec_compact(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool pred = i < a.n && (__double_as_longlong(a.cvec[i]) << 1) != 0;   // c != +-0, on the bits
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
    mlp_force_atom(a, APIP_CHK(a.status, BND_COMPACT, a.clist[q], a.n));
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
// descriptor kernel (one thread per atom, one partial per block), then the
// tensor-core network on persistent CTAs (two per SM)
template <typename T> void launch_pass1_learned(const Args<T>& a, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    launch_pdl(k_learned_desc, (a.n + kBlock - 1) / kBlock > 0 ? (a.n + kBlock - 1) / kBlock : 1, kBlock, 0, s, a,
               a.mlp_x0);
    cudaFuncSetAttribute(k_learned_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt::kSmemM);
    launch_pdl(k_learned_tc<false>, a.learned_grid1, lt::kT, lt::kSmemM, s, a, a.mlp_img, (const float*)a.mlp_x0);
  } else {
    const size_t bytes = sizeof(T) * APIP_MLP_NPARAM;
    cudaFuncSetAttribute(k_pass1_learned<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    launch_pdl(k_pass1_learned<T>, (a.n + kLearnedBlock - 1) / kLearnedBlock, kLearnedBlock, bytes, s, a);
  }
}

// Resident CTAs of the tensor-core learned kernels on this device: the force
// kernel one per SM (512 tensor-memory columns), pass 1's network (into
// *grid_pass1) two per SM (256 columns each); 0 if they do not fit.
int learned_tc_slots(int* grid_pass1) {
  int dev = 0, sms = 0, o1 = 0, o0 = 0;
  *grid_pass1 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the whole unified memory of an SM as shared memory: two pass-1 CTAs need 2 x 111 KB
  if (cudaFuncSetAttribute(k_learned_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt::kSmemM) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_learned_tc<false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
      cudaFuncSetAttribute(k_learned_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt::kSmem) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_learned_tc<true>, lt::kT, lt::kSmem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o0, k_learned_tc<false>, lt::kT, lt::kSmemM) != cudaSuccess)
    return 0;
  if (o1 < 1 || o0 < 1) return 0;
  // two per SM (their shared memory and registers fit twice, tensor memory holds
  // two); the tile loop is persistent, so a CTA that finds no room waits its turn
  *grid_pass1 = 2 * sms;
  return sms;
}

void launch_mlp_images(const float* w, void* img, cudaStream_t s) {
  constexpr int pairs = (kW * kIn + 2 * kW * kW) / 2;
  k_mlp_images<<<(pairs + 255) / 256, 256, 0, s>>>(w, reinterpret_cast<unsigned char*>(img));
}

size_t mlp_img_bytes() { return lt::kImg; }

template <typename T> void launch_mlp_force(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_cvec_compact<T>, (a.n + 255) / 256, 256, 0, s, a);
  if constexpr (sizeof(T) == 4) {
    // persistent CTAs over the tiles of the compacted list (its length is on the device)
    cudaFuncSetAttribute(k_learned_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lt::kSmem);
    launch_pdl(k_learned_tc<true>, a.learned_grid, lt::kT, lt::kSmem, s, a, a.mlp_img, (const float*)nullptr);
  } else {
    int blocks = (a.n + 127) / 128;   // the list holds at most n atoms; a grid-stride loop covers it
    if (blocks > 2048) blocks = 2048;
    launch_pdl(k_mlp_force<T>, blocks, 128, 0, s, a);
  }
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
