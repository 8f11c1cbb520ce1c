// ACE forward and adjoint on the compacted atoms with lam > 0, with the
// lam-dependent part of the EAM force and the weighting-function part of the
// grad-lambda force fused into the same neighbour loop.  Included by one
// translation unit per precision (kernels_ace_f32.cu, kernels_ace_f64.cu), each
// of which defines ynorm<T> (the real Y_lm normalisation in constant memory).
//
// One thread block (8 warps) handles a group of KA compacted atoms at a time,
// with the per-atom pool X = [1 | A | C] and its adjoint in shared memory
// (layout [pool index][KA]):
//  1. A_nlm = a_scale sum_j R_n(r_ij) Y_lm(rhat_ij): one thread per (atom,
//     neighbour) pair evaluates R and Y into shared memory, then threads own
//     (component, atom) entries of A.
//  2. C_{(p1 p2) L M} = sum G(l1 m1, l2 m2, L M) A_{p1 m1} A_{p2 m2} (a thread per
//     component); then phi_c = sum_b c_cb X_{s1(b)} . X_{s2(b)} over the
//     basis records (a thread per record, compensated sums per atom) and
//     E_i^ACE = phi_1 + (phi_2^2 + eps^2)^(1/4) - sqrt(eps).
//  3. The adjoint dE/dX: a thread per pool value gathers its segment's reverse
//     row (sum of k_b X_partner, k_b = c1_b + F'(phi_2) c2_b); then dE/dC goes
//     back onto A through the Gaunt entries, grouped by target A component and
//     cut into pieces whose partial sums are reduced per target.  No atomics.
//     omega = dE/dA a_scale lam_i.
//  4. One thread per pair: f_ij = sum_nlm omega_nlm grad(R_n Y_lm)(r_ij) (the ACE
//     force contribution of Eq. S14 / A1); plus, when the fast weights are 1 - lam,
//     the part -lam_i a_ij e_ij of S12 that pass 2 left out; plus, when
//     dlam_i != 0, the weighting-function part of the grad-lambda force
//     (Eq. S18-S21) Et_i (g_j - d_i - d0) w'(r_ij) e_ij with
//     Et_i = (E_i^prec - E_i^EAM) dlam_i / wbar_i, and c_j += Et_i w(r_ij) for the
//     CSP part (applied by k_csp_force).  F_j -= f, F_i += f (float64 atomics):
//     every contribution is pairwise antisymmetric (Eq. A1).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {

template <typename T> __device__ __forceinline__ T ynorm(int k);

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

// Elements of T in one pool of npool values for KA atoms, padded to 16 bytes.
template <typename T>
__host__ __device__ __forceinline__ int pool_elems(int npool, int KA) {
  return (int)(((size_t)npool * KA * sizeof(T) + 15) / 16 * 16 / sizeof(T));
}

// Dynamic shared memory of k_ace: the pool X, its adjoint (which also holds the
// per-pair R, Y rows of step 1), and the block reduction.
template <typename T, int LMAX, int KA>
__host__ __device__ inline size_t ace_smem_bytes(int npool) {
  constexpr size_t ry = (size_t)kAceThreads * (kNmaxCap + (LMAX + 1) * (LMAX + 1));
  const size_t px = (size_t)pool_elems<T>(npool, KA);
  return sizeof(T) * (px + (px > ry ? px : ry) + (size_t)2 * kAceWarps * KA);
}

template <int KA>
__device__ __forceinline__ int atom_of_pair(int p, const int* off) {
  int k = 0;
#pragma unroll
  for (int q = 1; q < KA; ++q) k += (p >= off[q]) ? 1 : 0;
  return k;
}

template <typename T, int LMAX, int KA>
__global__ void __launch_bounds__(kAceThreads) k_ace(Args<T> a, AceDev<T> t) {
  constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  constexpr int RYS = kNmaxCap + NLM;
  constexpr int RY_ELEMS = kAceThreads * RYS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_atom[KA], s_off[KA + 1], s_trans[KA];
  __shared__ T s_dfs[KA], s_e[KA], s_lam[KA], s_delta[KA], s_et[KA], s_D[KA], s_xi[KA];
  __shared__ double s_ep[KA];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nA = t.nA, npool = t.npool, c0 = 1 + nA;
  const int px = pool_elems<T>(npool, KA);
  T* X = reinterpret_cast<T*>(smem_raw);   // X[q * KA + k]
  T* G = X + px;                           // dE/dX, same layout
  T* RY = G;                               // step 1 staging
  T* red = G + (px > RY_ELEMS ? px : RY_ELEMS);
  T* A = X + KA;                           // A[c * KA + k] = X[(1 + c) * KA + k]
  T* W = G + KA;                           // omega, same layout as A

  const int count = a.counts[0];
  const int ngroups = (count + KA - 1) / KA;
  const T rc2 = t.rc * t.rc;
  const T rcE2 = T(a.eam.rc * a.eam.rc), rcE = T(a.eam.rc), rcE_lo = T(a.eam.rc_lo), rcE_inv = T(a.eam.inv_w);
  const T rw2 = T(a.sw.r_w * a.sw.r_w), rw = T(a.sw.r_w), rw_lo = T(a.sw.r_w_lo), rw_inv = T(a.sw.inv_w);
  const bool eam_corr = !a.precise_adds_eam && a.eam_force;
  const int n_max = t.n_max;
  double e_part = 0.0;

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    if (tid < KA) {
      const int idx = grp * KA + tid;
      s_atom[tid] = idx < count ? a.ace_list[idx] : -1;
    }
    __syncthreads();
    if (tid == 0) {
      s_off[0] = 0;
      for (int k = 0; k < KA; ++k) s_off[k + 1] = s_off[k] + (s_atom[k] >= 0 ? a.nnb[s_atom[k]] : 0);
    }
    for (int c = tid; c < c0 * KA; c += kAceThreads) X[c] = (c < KA) ? T(1) : T(0);
    __syncthreads();
    const int total = s_off[KA];

    // 1. atomic densities
    for (int base = 0; base < total; base += kAceThreads) {
      const int p = base + tid;
      T* ry = RY + tid * RYS;
      bool in = false;
      V3<T> d{T(0), T(0), T(0)};
      T r2 = T(0);
      if (p < total) {
        const int k = atom_of_pair<KA>(p, s_off);
        const int i = s_atom[k];
        const int j = a.nbl[(size_t)(p - s_off[k]) * a.nmax + i];
        d = a.pv.vec(a.pv.self(i), j);
        r2 = dot3(d, d);
        in = r2 < rc2;
      }
      if (in) {
        const T r = sqrt(r2);
        const T ir = T(1) / r;
        T R[kNmaxCap], dR[kNmaxCap];
        radial(r, t, R, dR);
#pragma unroll
        for (int n = 0; n < kNmaxCap; ++n) ry[n] = R[n];
        for_each_ylm<T, LMAX, false>(d.x * ir, d.y * ir, d.z * ir,
                                     [&](int k, T y, T, T, T) { ry[kNmaxCap + k] = y; });
      } else {
#pragma unroll
        for (int q = 0; q < RYS; ++q) ry[q] = T(0);
      }
      __syncthreads();
      const int hp = min(total - base, kAceThreads);
      for (int item = tid; item < nA * KA; item += kAceThreads) {
        const int c = item / KA, k = item - c * KA;
        const int n = c / NLM, lm = c - n * NLM;
        const int lo = max(s_off[k] - base, 0), hi = min(s_off[k + 1] - base, hp);
        T acc = T(0);
        for (int q = lo; q < hi; ++q) acc += RY[q * RYS + n] * RY[q * RYS + kNmaxCap + lm];
        A[item] += acc;
      }
      __syncthreads();
    }
    for (int item = tid; item < nA * KA; item += kAceThreads) A[item] *= t.a_scale;
    __syncthreads();

    // 2a. Gaunt couplings of pairs of A segments
    for (int c = tid; c < t.nC; c += kAceThreads) {
      const uint2 cp = t.comp[c];
      const T* x1 = X + (cp.x & 0xffffu) * KA;
      const T* x2 = X + (cp.x >> 16) * KA;
      const int g0 = (int)(cp.y >> 8), g1 = g0 + (int)(cp.y & 255u);
      T acc[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) acc[k] = T(0);
      for (int e = g0; e < g1; ++e) {
        const Ent<T> g = t.gent[e];
        const T* u = x1 + (g.key & 255u) * KA;
        const T* v = x2 + (g.key >> 8) * KA;
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] += g.v * u[k] * v[k];
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) X[(c0 + c) * KA + k] = acc[k];
    }
    __syncthreads();

    // 2b. embedding channels: one dot product of two pool segments per record
    {
      Acc<T> f1[KA], f2[KA];
      for (int r = tid; r < t.nf; r += kAceThreads) {
        const Rec<T> rc = t.frec[r];
        const T* u = X + (rc.key & 0xffffu) * KA;
        const T* v = X + (rc.key >> 16) * KA;
        T dot[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) dot[k] = T(0);
        for (int m = 0; m < (int)rc.len; ++m) {
#pragma unroll
          for (int k = 0; k < KA; ++k) dot[k] += u[m * KA + k] * v[m * KA + k];
        }
#pragma unroll
        for (int k = 0; k < KA; ++k) {
          f1[k].add(rc.k1 * dot[k]);
          f2[k].add(rc.k2 * dot[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) {
        const T v1 = warp_sum(f1[k].value()), v2 = warp_sum(f2[k].value());
        if (lane == 0) {
          red[(2 * warp) * KA + k] = v1;
          red[(2 * warp + 1) * KA + k] = v2;
        }
      }
    }
    __syncthreads();
    if (tid < KA) {
      T p1 = T(0), p2 = T(0);
      for (int w = 0; w < kAceWarps; ++w) {
        p1 += red[(2 * w) * KA + tid];
        p2 += red[(2 * w + 1) * KA + tid];
      }
      const T q2 = sqrt(p2 * p2 + t.eps * t.eps);
      const T e_ace = p1 + sqrt(q2) - t.sqrt_eps;
      s_e[tid] = e_ace;
      s_dfs[tid] = T(0.5) * p2 / (q2 * sqrt(q2));
      const int i = s_atom[tid];
      T lam = T(0), delta = T(0), et = T(0), D = T(0), xi = T(0);
      int trans = 0;
      if (i >= 0) {
        lam = a.lam[i];
        const T e_eam = a.e_eam[i];
        delta = e_ace + (a.precise_adds_eam ? e_eam : T(0)) - e_eam;
        const T dl = a.dlam[i];
        trans = (a.grad_lambda && (a.lam_mode == APIP_LAM_PAPER || a.lam_mode == APIP_LAM_LEARNED) &&
                 dl != T(0)) ? 1 : 0;
        et = trans ? delta * dl / a.wbar[i] : T(0);
        D = a.dd[i] + T(a.sw.d0);
        xi = a.xi_p[i];
      }
      s_lam[tid] = lam; s_delta[tid] = delta; s_et[tid] = et; s_D[tid] = D; s_xi[tid] = xi; s_trans[tid] = trans;
    }
    __syncthreads();

    // 3a. dE/dX: each pool value gathers the reverse row of its segment
    {
      T dfs[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) dfs[k] = s_dfs[k];
      for (int q = 1 + tid; q < npool; q += kAceThreads) {
        const int4 qr = t.qrow[q];
        T acc[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] = T(0);
        for (int e = qr.x; e < qr.y; ++e) {
          const Rec<T> rc = t.arec[e];
          const T* v = X + (rc.key + qr.z) * KA;
#pragma unroll
          for (int k = 0; k < KA; ++k) acc[k] += (rc.k1 + dfs[k] * rc.k2) * v[k];
        }
#pragma unroll
        for (int k = 0; k < KA; ++k) G[q * KA + k] = acc[k];
      }
    }
    __syncthreads();

    // 3b. dE/dC back onto A: partial sums of the pieces, kept in the C part of X
    //     (not read again for this group)
    for (int pc = tid; pc < t.npc; pc += kAceThreads) {
      T acc[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) acc[k] = T(0);
      const int e1 = t.poff[pc + 1];
      for (int e = t.poff[pc]; e < e1; ++e) {
        const Ent<T> b = t.bent[e];
        const T* gc = G + (b.key & 0xffffu) * KA;
        const T* xo = X + (b.key >> 16) * KA;
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] += b.v * gc[k] * xo[k];
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) X[(c0 + pc) * KA + k] = acc[k];
    }
    __syncthreads();
    for (int item = tid; item < nA * KA; item += kAceThreads) {
      const int c = item / KA, k = item - c * KA;
      T s = W[item];
      const int p1 = t.tpiece[c + 1];
      for (int pc = t.tpiece[c]; pc < p1; ++pc) s += X[(c0 + pc) * KA + k];
      W[item] = s * t.a_scale * s_lam[k];
    }
    __syncthreads();
    // 4. pair forces
    for (int base = 0; base < total; base += kAceThreads) {
      const int p = base + tid;
      if (p >= total) continue;
      const int k = atom_of_pair<KA>(p, s_off);
      const int i = s_atom[k];
      const int j = a.nbl[(size_t)(p - s_off[k]) * a.nmax + i];
      const V3<T> d = a.pv.vec(a.pv.self(i), j);
      const T r2 = dot3(d, d);
      const bool trans = s_trans[k] != 0;
      const bool in_a = r2 < rc2;
      const bool in_e = eam_corr && r2 < rcE2;
      const bool in_w = trans && r2 < rw2;
      if (!(in_a || in_e || in_w)) continue;
      const T r = sqrt(r2);
      const T ir = T(1) / r;
      const T ex = d.x * ir, ey = d.y * ir, ez = d.z * ir;
      T sr = T(0);
      T gx = T(0), gy = T(0), gz = T(0);
      if (in_a) {
        T R[kNmaxCap], dR[kNmaxCap];
        radial(r, t, R, dR);
        const T* Wk = W + k;
        for_each_ylm<T, LMAX, true>(ex, ey, ez, [&](int c, T y, T px, T py, T pz) {
          T u = T(0), v = T(0);
#pragma unroll
          for (int n = 0; n < kNmaxCap; ++n) {
            if (n < n_max) {
              const T w = Wk[(n * NLM + c) * KA];
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
        sr -= s_lam[k] * (s_xi[k] * drho + T(0.5) * dphi);
      }
      if (in_w) {
        T dw;
        const T w = ftrans(r, rw_lo, rw, rw_inv, &dw);
        sr += s_et[k] * (a.g[j] - s_D[k]) * dw;
        atomicAdd(&a.cvec[j], (double)(s_et[k] * w));
      }
      const double f0 = (double)(sr * ex + gx), f1 = (double)(sr * ey + gy), f2 = (double)(sr * ez + gz);
      atomicAdd(&a.force[3 * j], -f0);
      atomicAdd(&a.force[3 * j + 1], -f1);
      atomicAdd(&a.force[3 * j + 2], -f2);
      atomicAdd(&a.force[3 * i], f0);
      atomicAdd(&a.force[3 * i + 1], f1);
      atomicAdd(&a.force[3 * i + 2], f2);
    }
    if (tid < KA) {
      const int i = s_atom[tid];
      if (i >= 0) {
        if (s_trans[tid]) atomicAdd(&a.cvec[i], (double)s_et[tid]);
        a.e_ace[i] = s_e[tid];
        const double ed = (double)s_lam[tid] * (double)s_delta[tid];
        e_part += ed;
        if (a.e_atom) a.e_atom[i] += ed;
      }
    }
    __syncthreads();
  }
  if (tid < KA) s_ep[tid] = e_part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < KA; ++k) s += s_ep[k];
    a.partials[a.n_part_p1 + blockIdx.x] = s;
  }
}

template <typename T, int LMAX, int KA>
void launch_lk(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  const size_t bytes = ace_smem_bytes<T, LMAX, KA>(t.npool);
  cudaFuncSetAttribute(k_ace<T, LMAX, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  k_ace<T, LMAX, KA><<<blocks, kAceThreads, bytes, s>>>(a, t);
}

// Resident blocks per SM of k_ace for this pool size (0 if it does not fit).
template <typename T, int LMAX, int KA>
int occupancy_lk(int npool, size_t* bytes) {
  *bytes = ace_smem_bytes<T, LMAX, KA>(npool);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (*bytes + (size_t)1024 > (size_t)optin) return 0;
  if (cudaFuncSetAttribute(k_ace<T, LMAX, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*bytes) !=
      cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ace<T, LMAX, KA>, kAceThreads, *bytes) != cudaSuccess)
    return 0;
  return occ;
}

template <typename T, int KA>
void launch_k(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  switch (t.l_max) {
    case 0: launch_lk<T, 0, KA>(a, t, blocks, s); break;
    case 1: launch_lk<T, 1, KA>(a, t, blocks, s); break;
    case 2: launch_lk<T, 2, KA>(a, t, blocks, s); break;
    case 3: launch_lk<T, 3, KA>(a, t, blocks, s); break;
    default: launch_lk<T, 4, KA>(a, t, blocks, s); break;
  }
}

template <typename T, int KA>
int occupancy_k(int l_max, int npool, size_t* bytes) {
  switch (l_max) {
    case 0: return occupancy_lk<T, 0, KA>(npool, bytes);
    case 1: return occupancy_lk<T, 1, KA>(npool, bytes);
    case 2: return occupancy_lk<T, 2, KA>(npool, bytes);
    case 3: return occupancy_lk<T, 3, KA>(npool, bytes);
    default: return occupancy_lk<T, 4, KA>(npool, bytes);
  }
}

template <typename T>
void launch_ace_impl(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  switch (t.group) {
    case 8: launch_k<T, 8>(a, t, blocks, s); break;
    case 4: launch_k<T, 4>(a, t, blocks, s); break;
    case 2: launch_k<T, 2>(a, t, blocks, s); break;
    default: launch_k<T, 1>(a, t, blocks, s); break;
  }
}

template <typename T>
int ace_occupancy_impl(int l_max, int group, int npool, size_t* bytes) {
  switch (group) {
    case 8: return occupancy_k<T, 8>(l_max, npool, bytes);
    case 4: return occupancy_k<T, 4>(l_max, npool, bytes);
    case 2: return occupancy_k<T, 2>(l_max, npool, bytes);
    default: return occupancy_k<T, 1>(l_max, npool, bytes);
  }
}

}  // namespace apip
