// ACE forward and adjoint on the compacted atoms with lam > 0, one warp per
// atom, with the lam-dependent part of the EAM force and the weighting-function
// part of the grad-lambda force fused into the same neighbour loop.
//
// For atom i (warp):
//  1. A_nlm = a_scale sum_j R_n(r_ij) Y_lm(rhat_ij): lanes evaluate R and Y for 32
//     neighbours at a time into shared memory, then lanes own components of A.
//  2. phi_c = sum_t K_c[t] prod_q A[idx_q(t)] over the folded term lists (lanes
//     stride the terms); E_i^ACE = phi_1 + (phi_2^2 + eps^2)^(1/4) - sqrt(eps).
//  3. omega = dE_i/dA from the derivative entries of the terms, sorted by target
//     A index: a segmented warp scan per 32 entries, no atomics; then scaled by
//     a_scale lam_i.
//  4. Lane = neighbour j: f_ij = sum_nlm omega_nlm grad(R_n Y_lm)(r_ij) (Eq. S14 /
//     A1 force contribution); plus, for the fast-model weights (1 - lam), the part
//     -lam_i a_ij e_ij of S12 that pass 2 left out; plus, when dlam_i != 0, the
//     weighting-function part of the grad-lambda force (Eq. S18-S21)
//        Et_i (g_j - d_i - d0) w'(r_ij) e_ij,  Et_i = (E_i^prec - E_i^EAM) dlam_i / wbar_i,
//     and c_j += Et_i w(r_ij) for the CSP part (applied by k_csp_force).
//     F_j -= f, F_i += f: every contribution is pairwise antisymmetric (A1).
#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {

__constant__ double c_norm_d[(kLmaxCap + 1) * (kLmaxCap + 1)];
__constant__ float c_norm_f[(kLmaxCap + 1) * (kLmaxCap + 1)];

template <typename T> __device__ __forceinline__ T ynorm(int k);
template <> __device__ __forceinline__ double ynorm<double>(int k) { return c_norm_d[k]; }
template <> __device__ __forceinline__ float ynorm<float>(int k) { return c_norm_f[k]; }

// Real spherical harmonics Y_lm(u) = N_lm Pi_l^m(z) {C_m, S_m}(x, y) for a unit
// vector u, where C_m + i S_m = (x + i y)^m and Pi_l^m obeys the associated
// Legendre recurrence (no Condon-Shortley phase).  Calls f(index, Y, dPx, dPy,
// dPz) with the gradient of that polynomial expression in (x, y, z); the
// gradient of Y(r/|r|) is (grad P - (u . grad P) u) / |r|.
template <typename T, int L, bool GRAD, typename F>
__device__ __forceinline__ void for_each_ylm(T x, T y, T z, F&& f) {
  T C[L + 1], S[L + 1];
  C[0] = T(1);
  S[0] = T(0);
#pragma unroll
  for (int m = 1; m <= L; ++m) {
    C[m] = x * C[m - 1] - y * S[m - 1];
    S[m] = x * S[m - 1] + y * C[m - 1];
  }
#pragma unroll
  for (int m = 0; m <= L; ++m) {
    T dfact = T(1);
#pragma unroll
    for (int k = 1; k <= m; ++k) dfact *= T(2 * k - 1);
    T p1 = T(0), p2 = T(0), d1 = T(0), d2 = T(0);
#pragma unroll
    for (int l = m; l <= L; ++l) {
      T P, dP;
      if (l == m) { P = dfact; dP = T(0); }
      else if (l == m + 1) { P = T(2 * m + 1) * z * dfact; dP = T(2 * m + 1) * dfact; }
      else {
        const T inv = T(1) / T(l - m);
        P = (T(2 * l - 1) * z * p1 - T(l + m - 1) * p2) * inv;
        dP = (T(2 * l - 1) * (p1 + z * d1) - T(l + m - 1) * d2) * inv;
      }
      p2 = p1; p1 = P; d2 = d1; d1 = dP;
      if (m == 0) {
        const T nrm = ynorm<T>(l * l + l);
        f(l * l + l, nrm * P, T(0), T(0), GRAD ? nrm * dP : T(0));
      } else {
        const T nrm = ynorm<T>(l * l + l + m);
        const T np = nrm * P;
        if (GRAD) {
          f(l * l + l + m, np * C[m], np * T(m) * C[m - 1], -np * T(m) * S[m - 1], nrm * dP * C[m]);
          f(l * l + l - m, np * S[m], np * T(m) * S[m - 1], np * T(m) * C[m - 1], nrm * dP * S[m]);
        } else {
          f(l * l + l + m, np * C[m], T(0), T(0), T(0));
          f(l * l + l - m, np * S[m], T(0), T(0), T(0));
        }
      }
    }
  }
}

// R_n(r) = T_{n-1}(1 - 2r/rc) fc(r) and dR/dr, n = 1..n_max (index n-1).
template <typename T>
__device__ __forceinline__ void radial(T r, const AceDev<T>& t, T* R, T* dR) {
  T dfc;
  const T fc = ftrans(r, t.rc_lo, t.rc, T(1) / (t.rc - t.rc_lo), &dfc);
  const T x = T(1) - T(2) * r / t.rc;
  const T dxdr = T(-2) / t.rc;
  T tm2 = T(1), tm1 = x, dm2 = T(0), dm1 = T(1);
#pragma unroll
  for (int n = 0; n < kNmaxCap; ++n) {
    T Tn, dTn;
    if (n == 0) { Tn = T(1); dTn = T(0); }
    else if (n == 1) { Tn = x; dTn = T(1); }
    else {
      Tn = T(2) * x * tm1 - tm2;
      dTn = T(2) * tm1 + T(2) * x * dm1 - dm2;
      tm2 = tm1; tm1 = Tn; dm2 = dm1; dm1 = dTn;
    }
    R[n] = Tn * fc;
    dR[n] = dTn * dxdr * fc + Tn * dfc;
  }
}

template <typename T, int LMAX>
__global__ void __launch_bounds__(kAceWarps * 32) k_ace(Args<T> a, AceDev<T> t) {
  constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nA = t.nA;
  const int nAp = (nA + 1 + 3) & ~3;
  const int per_warp = 2 * nAp + 32 * (kNmaxCap + NLM);
  T* A = reinterpret_cast<T*>(smem_raw) + warp * per_warp;
  T* W = A + nAp;
  T* Rs = W + nAp;
  T* Ys = Rs + 32 * kNmaxCap;

  const int count = a.counts[0];
  const int gw = blockIdx.x * kAceWarps + warp;
  const int nw = gridDim.x * kAceWarps;
  const T rc2 = t.rc * t.rc;
  const T rcE2 = T(a.eam.rc * a.eam.rc), rcE = T(a.eam.rc), rcE_lo = T(a.eam.rc_lo);
  const T rcE_inv = T(a.eam.inv_w);
  const T rw2 = T(a.sw.r_w * a.sw.r_w), rw = T(a.sw.r_w), rw_lo = T(a.sw.r_w_lo);
  const T rw_inv = T(a.sw.inv_w);
  const bool eam_corr = !a.precise_adds_eam && a.eam_force;
  const int n_max = t.n_max;
  double e_part = 0.0;

  for (int tt = gw; tt < count; tt += nw) {
    const int i = a.ace_list[tt];
    const auto si = a.pv.self(i);
    const int cnt = a.nnb[i];
    for (int c = lane; c <= nA; c += 32) {
      A[c] = (c == nA) ? T(1) : T(0);
      W[c] = T(0);
    }
    __syncwarp();

    // 1. atomic density A_nlm
    for (int base = 0; base < cnt; base += 32) {
      const int s = base + lane;
      T* Rl = Rs + lane * kNmaxCap;
      T* Yl = Ys + lane * NLM;
      bool in = false;
      V3<T> d{T(0), T(0), T(0)};
      T r2 = T(0);
      if (s < cnt) {
        const int j = a.nbl[(size_t)s * a.nmax + i];
        d = a.pv.vec(si, j);
        r2 = dot3(d, d);
        in = r2 < rc2;
      }
      if (in) {
        const T r = sqrt(r2);
        const T ir = T(1) / r;
        T R[kNmaxCap], dR[kNmaxCap];
        radial(r, t, R, dR);
#pragma unroll
        for (int n = 0; n < kNmaxCap; ++n) Rl[n] = R[n];
        for_each_ylm<T, LMAX, false>(d.x * ir, d.y * ir, d.z * ir,
                                     [&](int k, T y, T, T, T) { Yl[k] = y; });
      } else {
#pragma unroll
        for (int n = 0; n < kNmaxCap; ++n) Rl[n] = T(0);
#pragma unroll
        for (int k = 0; k < NLM; ++k) Yl[k] = T(0);
      }
      __syncwarp();
      const int kmax = min(32, cnt - base);
      for (int c = lane; c < nA; c += 32) {
        const int n = c / NLM, lm = c - n * NLM;
        T acc = T(0);
        for (int k = 0; k < kmax; ++k) acc += Rs[k * kNmaxCap + n] * Ys[k * NLM + lm];
        A[c] += acc;
      }
      __syncwarp();
    }
    for (int c = lane; c < nA; c += 32) A[c] *= t.a_scale;
    __syncwarp();

    // 2. embedding channels
    Acc<T> s1, s2;     // compensated in FP32
    for (int q = lane; q < t.n3; q += 32) {
      const uint32_t k = t.key3[q];
      const T x = A[k & 255u] * A[(k >> 8) & 255u] * A[(k >> 16) & 255u];
      s1.add(t.k3a[q] * x);
      s2.add(t.k3b[q] * x);
    }
    for (int q = lane; q < t.n4; q += 32) {
      const uint32_t k = t.key4[q];
      const T x = A[k & 255u] * A[(k >> 8) & 255u] * A[(k >> 16) & 255u] * A[k >> 24];
      s1.add(t.k4a[q] * x);
      s2.add(t.k4b[q] * x);
    }
    const T p1 = warp_sum(s1.value());
    const T p2 = warp_sum(s2.value());
    const T q2 = sqrt(p2 * p2 + t.eps * t.eps);
    const T e_ace = p1 + sqrt(q2) - t.sqrt_eps;
    const T dfs = T(0.5) * p2 / (q2 * sqrt(q2));

    // 3. omega = dE/dA from the derivative entries (sorted by target): 32
    //    consecutive entries per step, a segmented warp scan over equal targets,
    //    and one plain shared-memory update per distinct target.
    for (int base = 0; base < t.nd; base += 32) {
      const int q = base + lane;
      int tgt = -1 - lane;
      T v = T(0);
      if (q < t.nd) {
        const uint32_t k = t.keyd[q];
        tgt = (int)(k >> 24);
        v = (t.kda[q] + dfs * t.kdb[q]) * A[k & 255u] * A[(k >> 8) & 255u] * A[(k >> 16) & 255u];
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const T vo = __shfl_up_sync(0xffffffffu, v, o);
        const int to = __shfl_up_sync(0xffffffffu, tgt, o);
        if (lane >= o && to == tgt) v += vo;
      }
      const int tn = __shfl_down_sync(0xffffffffu, tgt, 1);
      if (q < t.nd && (lane == 31 || tn != tgt)) W[tgt] += v;
      __syncwarp();
    }

    const T lam_i = a.lam[i];
    const T e_eam_i = a.e_eam[i];
    const T e_prec = e_ace + (a.precise_adds_eam ? e_eam_i : T(0));
    const T delta = e_prec - e_eam_i;
    const T dlam_i = a.dlam[i];
    const bool trans = a.grad_lambda && a.lam_mode == APIP_LAM_PAPER && dlam_i != T(0);
    const T Et = trans ? delta * dlam_i / a.wbar[i] : T(0);
    const T Di = a.dd[i] + T(a.sw.d0);
    const T xi_i = a.xi_p[i];
    const T wscale = t.a_scale * lam_i;
    for (int c = lane; c < nA; c += 32) W[c] *= wscale;
    __syncwarp();

    // 4. pair forces
    Acc<T> fx, fy, fz;
    for (int base = 0; base < cnt; base += 32) {
      const int s = base + lane;
      if (s >= cnt) continue;
      const int j = a.nbl[(size_t)s * a.nmax + i];
      const V3<T> d = a.pv.vec(si, j);
      const T r2 = dot3(d, d);
      const bool in_a = r2 < rc2;
      const bool in_e = eam_corr && r2 < rcE2;
      const bool in_w = trans && r2 < rw2;
      if (!(in_a || in_e || in_w)) continue;
      const T r = sqrt(r2);
      const T ir = T(1) / r;
      const T ex = d.x * ir, ey = d.y * ir, ez = d.z * ir;
      T sr = T(0);                 // coefficient of e_ij
      T gx = T(0), gy = T(0), gz = T(0);   // sum v_lm grad P_lm
      if (in_a) {
        T R[kNmaxCap], dR[kNmaxCap];
        radial(r, t, R, dR);
        for_each_ylm<T, LMAX, true>(ex, ey, ez, [&](int k, T y, T px, T py, T pz) {
          T u = T(0), v = T(0);
#pragma unroll
          for (int n = 0; n < kNmaxCap; ++n) {
            if (n < n_max) {
              const T w = W[n * NLM + k];
              u += w * dR[n];
              v += w * R[n];
            }
          }
          sr += u * y;
          gx += v * px;
          gy += v * py;
          gz += v * pz;
        });
        const T eg = ex * gx + ey * gy + ez * gz;
        gx = (gx - eg * ex) * ir;
        gy = (gy - eg * ey) * ir;
        gz = (gz - eg * ez) * ir;
      }
      if (in_e) {
        T dfc;
        const T fc = ftrans(r, rcE_lo, rcE, rcE_inv, &dfc);
        const T er = T(a.eam.A) * exp(-T(a.eam.beta) * (r - T(a.eam.re)));
        const T drho = er * (dfc - T(a.eam.beta) * fc);
        const T x = exp(-T(a.eam.alpha) * (r - T(a.eam.r0)));
        const T dphi = T(a.eam.D) * (T(2) * T(a.eam.alpha) * (x - x * x) * fc + (x * x - T(2) * x) * dfc);
        sr -= lam_i * (xi_i * drho + T(0.5) * dphi);
      }
      if (in_w) {
        T dw;
        const T w = ftrans(r, rw_lo, rw, rw_inv, &dw);
        sr += Et * (a.g[j] - Di) * dw;
        atomicAdd(&a.cvec[j], (double)(Et * w));
      }
      const T f0 = sr * ex + gx, f1 = sr * ey + gy, f2 = sr * ez + gz;
      atomicAdd(&a.force[3 * j], -(double)f0);
      atomicAdd(&a.force[3 * j + 1], -(double)f1);
      atomicAdd(&a.force[3 * j + 2], -(double)f2);
      fx.add(f0);
      fy.add(f1);
      fz.add(f2);
    }
    const T sx = warp_sum(fx.value()), sy = warp_sum(fy.value()), sz = warp_sum(fz.value());
    if (lane == 0) {
      atomicAdd(&a.force[3 * i], (double)sx);
      atomicAdd(&a.force[3 * i + 1], (double)sy);
      atomicAdd(&a.force[3 * i + 2], (double)sz);
      if (trans) atomicAdd(&a.cvec[i], (double)Et);
      a.e_ace[i] = e_ace;
      const double ed = (double)lam_i * (double)delta;
      e_part += ed;
      if (a.e_atom) a.e_atom[i] += ed;
    }
    __syncwarp();
  }
  if (lane == 0) a.partials[a.n_part_p1 + gw] = e_part;
}

template <typename T> void ace_set_norms(const double* norms, int count) {
  if (sizeof(T) == 8) {
    cudaMemcpyToSymbol(c_norm_d, norms, sizeof(double) * count);
  } else {
    float f[(kLmaxCap + 1) * (kLmaxCap + 1)];
    for (int k = 0; k < count; ++k) f[k] = (float)norms[k];
    cudaMemcpyToSymbol(c_norm_f, f, sizeof(float) * count);
  }
}

template <typename T, int LMAX>
static void launch_l(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  const int nAp = (t.nA + 1 + 3) & ~3;
  const size_t bytes = sizeof(T) * (size_t)kAceWarps * (2 * nAp + 32 * (kNmaxCap + NLM));
  cudaFuncSetAttribute(k_ace<T, LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_ace<T, LMAX><<<blocks, kAceWarps * 32, bytes, s>>>(a, t);
}

template <typename T> void launch_ace(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  switch (t.l_max) {
    case 0: launch_l<T, 0>(a, t, blocks, s); break;
    case 1: launch_l<T, 1>(a, t, blocks, s); break;
    case 2: launch_l<T, 2>(a, t, blocks, s); break;
    case 3: launch_l<T, 3>(a, t, blocks, s); break;
    default: launch_l<T, 4>(a, t, blocks, s); break;
  }
}

template void ace_set_norms<double>(const double*, int);
template void ace_set_norms<float>(const double*, int);
template void launch_ace<double>(const Args<double>&, const AceDev<double>&, int, cudaStream_t);
template void launch_ace<float>(const Args<float>&, const AceDev<float>&, int, cudaStream_t);

}  // namespace apip
