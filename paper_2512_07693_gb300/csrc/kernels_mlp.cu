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

template <typename T> __device__ __forceinline__ T silu(T z) { return z / (T(1) + exp(-z)); }
template <typename T> __device__ __forceinline__ T silu_d(T z) {
  const T s = T(1) / (T(1) + exp(-z));
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
    const T e_ind = ind_energy(a, i);   // the external indenter, if any
    if (a.e_atom) a.e_atom[i] = (double)e + (double)e_ind;
    e_out = (double)e + (double)e_ind;
    const T g = mlp_forward<T>(w, G, nullptr);
    a.g[i] = g;
    if constexpr (sizeof(T) == 4) a.posg[i] = make_uint4(si.q.x, si.q.y, si.q.z, __float_as_uint(g));
  }
  const double tot = block_sum(e_out, sh);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
}

// -grad sum_k c_k g_k for the atoms with c_k != 0 (learned counterpart of
// k_csp_force): dG_km = c_k dg_k/dG_km by back-propagation, then for each
// neighbour j: v = sum_m dG_km phi_m'(r_kj), F_j -= v e_kj, F_k += v e_kj.
template <typename T>
__global__ void __launch_bounds__(128) k_mlp_force(Args<T> a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  const double c = a.cvec[k];
  if (c == 0.0) return;
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

// ---------------------------------------------------------------- training
// Per sample: forward (z -> ws_z), loss term, back-propagation to d (-> ws_d).
__global__ void __launch_bounds__(128) k_train_fwd_bwd(const __nv_bfloat16* __restrict__ desc,
                                                       const float* __restrict__ y, int batch,
                                                       const float* __restrict__ params, float* ws_z,
                                                       float* ws_d, float* dg_out, float* loss_part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* w = reinterpret_cast<float*>(smem_raw);
  __shared__ double sh[32];
  for (int k = threadIdx.x; k < APIP_MLP_NPARAM; k += blockDim.x) w[k] = params[k];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (s < batch) {
    float G[kIn];
#pragma unroll
    for (int m = 0; m < kIn; ++m) G[m] = __bfloat162float(desc[(size_t)s * kIn + m]);
    float* z = ws_z + (size_t)s * 3 * kW;
    float* d = ws_d + (size_t)s * 3 * kW;
    const float g = mlp_forward<float>(w, G, z);
    const float r = g - y[s];
    l = (double)r * (double)r;
    const float dg = 2.0f * r / (float)batch;
    dg_out[s] = dg;
    mlp_backward_z<float>(w, z, dg, d);
  }
  const double tot = block_sum(l, sh);
  if (threadIdx.x == 0) loss_part[blockIdx.x] = tot;
}

// Weight gradients: one thread per parameter, summed over a chunk of samples,
// chunks combined with atomics into grad (zeroed beforehand).
__global__ void k_train_wgrad(const __nv_bfloat16* __restrict__ desc, int batch, const float* __restrict__ ws_z,
                              const float* __restrict__ ws_d, const float* __restrict__ dg, float* grad,
                              int chunk) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= APIP_MLP_NPARAM) return;
  const int s0 = blockIdx.y * chunk, s1 = min(batch, s0 + chunk);
  float acc = 0.0f;
  if (p < oB1) {                          // W1[j][k]: d1_j x0_k
    const int j = (p - oW1) / kIn, k = (p - oW1) % kIn;
    for (int s = s0; s < s1; ++s)
      acc += ws_d[(size_t)s * 3 * kW + j] * (float)kSin * __bfloat162float(desc[(size_t)s * kIn + k]);
  } else if (p < oW2) {                   // b1[j]
    const int j = p - oB1;
    for (int s = s0; s < s1; ++s) acc += ws_d[(size_t)s * 3 * kW + j];
  } else if (p < oB2) {                   // W2[j][k]: d2_j h1_k
    const int j = (p - oW2) / kW, k = (p - oW2) % kW;
    for (int s = s0; s < s1; ++s) acc += ws_d[(size_t)s * 3 * kW + kW + j] * silu(ws_z[(size_t)s * 3 * kW + k]);
  } else if (p < oW3) {                   // b2[j]
    const int j = p - oB2;
    for (int s = s0; s < s1; ++s) acc += ws_d[(size_t)s * 3 * kW + kW + j];
  } else if (p < oB3) {                   // W3[j][k]: d3_j h2_k
    const int j = (p - oW3) / kW, k = (p - oW3) % kW;
    for (int s = s0; s < s1; ++s)
      acc += ws_d[(size_t)s * 3 * kW + 2 * kW + j] * silu(ws_z[(size_t)s * 3 * kW + kW + k]);
  } else if (p < oW4) {                   // b3[j]
    const int j = p - oB3;
    for (int s = s0; s < s1; ++s) acc += ws_d[(size_t)s * 3 * kW + 2 * kW + j];
  } else if (p < oB4) {                   // w4[j]: dg h3_j
    const int j = p - oW4;
    for (int s = s0; s < s1; ++s) acc += dg[s] * silu(ws_z[(size_t)s * 3 * kW + 2 * kW + j]);
  } else {                                // b4
    for (int s = s0; s < s1; ++s) acc += dg[s];
  }
  atomicAdd(&grad[p], acc);
}

__global__ void k_train_loss(const float* loss_part, int nb, int batch, float* loss_out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) s += loss_part[k];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) *loss_out = (float)(tot / batch);
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int t, float lr) {
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

template <typename T> void launch_pass1_learned(const Args<T>& a, cudaStream_t s) {
  const size_t bytes = sizeof(T) * APIP_MLP_NPARAM;
  cudaFuncSetAttribute(k_pass1_learned<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_pass1_learned<T><<<(a.n + kLearnedBlock - 1) / kLearnedBlock, kLearnedBlock, bytes, s>>>(a);
}

template <typename T> void launch_mlp_force(const Args<T>& a, cudaStream_t s) {
  k_mlp_force<T><<<(a.n + 127) / 128, 128, 0, s>>>(a);
}

template <typename T> void launch_descriptors(const Args<T>& a, uint16_t* out, cudaStream_t s) {
  k_descriptors<T><<<(a.n + 127) / 128, 128, 0, s>>>(a, reinterpret_cast<__nv_bfloat16*>(out));
}

template <typename T> void launch_cast_params(const float* src, T* dst, cudaStream_t s) {
  k_cast_params<T><<<(APIP_MLP_NPARAM + 255) / 256, 256, 0, s>>>(src, dst);
}

void launch_mlp_loss_grad(const uint16_t* desc, const float* y, int batch, const float* params, float* grad,
                          float* loss, float* ws, cudaStream_t s) {
  const int nb = (batch + 127) / 128;
  float* ws_z = ws;
  float* ws_d = ws + (size_t)batch * 3 * kW;
  float* dg = ws_d + (size_t)batch * 3 * kW;
  float* loss_part = dg + batch;
  const size_t bytes = sizeof(float) * APIP_MLP_NPARAM;
  cudaFuncSetAttribute(k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  const __nv_bfloat16* d = reinterpret_cast<const __nv_bfloat16*>(desc);
  k_train_fwd_bwd<<<nb, 128, bytes, s>>>(d, y, batch, params, ws_z, ws_d, dg, loss_part);
  cudaMemsetAsync(grad, 0, sizeof(float) * APIP_MLP_NPARAM, s);
  const int chunk = 256;
  dim3 grid((APIP_MLP_NPARAM + 255) / 256, (batch + chunk - 1) / chunk);
  k_train_wgrad<<<grid, 256, 0, s>>>(d, batch, ws_z, ws_d, dg, grad, chunk);
  k_train_loss<<<1, 256, 0, s>>>(loss_part, nb, batch, loss);
}

size_t mlp_workspace_floats(int batch) { return (size_t)batch * (6 * kW + 1) + (batch + 127) / 128; }

void launch_mlp_adam(float* p, const float* g, float* m, float* v, int t, float lr, cudaStream_t s) {
  k_adam<<<(APIP_MLP_NPARAM + 255) / 256, 256, 0, s>>>(p, g, m, v, t, lr);
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
