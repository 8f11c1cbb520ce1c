// Device code shared by the two ACE kernels (ace_pool.cuh for body order 4,
// ace_stream.cuh for body order <= 3): real spherical harmonics, the radial
// basis, table loads, and the per-block steps that do not depend on how the
// product basis is evaluated:
//  1. A_nlm = a_scale sum_j R_n(r_ij) Y_lm(rhat_ij) for a group of NAT compacted
//     atoms: one thread per (atom, neighbour) pair evaluates R and Y into shared
//     memory, then threads own (component, atom) entries of A (layout [c][NAT]).
//  -  the per-atom scalars after the embedding channels phi_1, phi_2:
//     E_i^ACE = phi_1 + (phi_2^2 + eps^2)^(1/4) - sqrt(eps) and F'(phi_2);
//  4. one thread per pair: f_ij = sum_nlm omega_nlm grad(R_n Y_lm)(r_ij) (the ACE
//     force contribution of Eq. S14 / A1); plus, when the fast weights are 1 - lam,
//     the part -lam_i a_ij e_ij of S12 that pass 2 left out; plus, when
//     dlam_i != 0, the weighting-function part of the grad-lambda force
//     (Eq. S18-S21) Et_i (g_j - d_i - d0) w'(r_ij) e_ij with
//     Et_i = (E_i^prec - E_i^EAM) dlam_i / wbar_i, and c_j += Et_i w(r_ij) for the
//     CSP or MLP part (applied by k_csp_force / k_mlp_force).  F_j -= f, F_i += f
//     (float64 atomics): every contribution is pairwise antisymmetric (Eq. A1).
//
// K is the translation unit's constant accessor: K::ynorm(k) (the real Y_lm
// normalisation) and, for the streamed kernel, K::gaunt(e).
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {

// Real spherical harmonics Y_lm(u) = N_lm Pi_l^m(z) {C_m, S_m}(x, y) for a unit
// vector u, where C_m + i S_m = (x + i y)^m and Pi_l^m obeys the associated
// Legendre recurrence (no Condon-Shortley phase).  Calls f(index, Y, dPx, dPy,
// dPz) with the gradient of that polynomial expression in (x, y, z); the
// gradient of Y(r/|r|) is (grad P - (u . grad P) u) / |r|.
template <typename T, typename K, int L, bool GRAD, typename F>
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
        const T nrm = K::ynorm(l * l + l);
        f(l * l + l, nrm * P, T(0), T(0), GRAD ? nrm * dP : T(0));
      } else {
        const T nrm = K::ynorm(l * l + l + m);
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
  const T fc = ftrans(r, t.rc_lo, t.rc, t.inv_width, &dfc);
  const T x = T(1) - t.two_over_rc * r;
  const T dxdr = -t.two_over_rc;
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

// Read-only loads of the table entries (through the non-coherent data cache).
__device__ __forceinline__ Rec<float> ld(const Rec<float>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {__float_as_uint(v.x), __float_as_uint(v.y), v.z, v.w};
}
__device__ __forceinline__ Rec<double> ld(const Rec<double>* p) {
  const uint2 h = __ldg(reinterpret_cast<const uint2*>(p));
  const double* d = reinterpret_cast<const double*>(p) + 1;
  return {h.x, h.y, __ldg(d), __ldg(d + 1)};
}
__device__ __forceinline__ Ent<float> ld(const Ent<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, __float_as_uint(v.y)};
}
__device__ __forceinline__ Ent<double> ld(const Ent<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, (uint32_t)__double_as_longlong(v.y)};
}

// n elements of T for KA atoms, rounded up to a multiple of 16 bytes.
template <typename T>
__host__ __device__ __forceinline__ int pool_elems(int n, int KA) {
  return (int)(((size_t)n * KA * sizeof(T) + 15) / 16 * 16 / sizeof(T));
}

// Row stride of the per-pair R, Y staging of step 1: n_max radial values and the
// (l_max+1)^2 harmonics, padded to an odd number of words so that the rows of
// consecutive pairs start in different banks.
template <int LMAX>
__host__ __device__ constexpr int ry_stride() { return (kNmaxCap + (LMAX + 1) * (LMAX + 1)) | 1; }
template <int LMAX>
__host__ __device__ constexpr int ry_elems() { return kAceThreads * ry_stride<LMAX>(); }

// Per-atom state of a group, in static shared memory.
template <typename T, int NAT>
struct AceGroup {
  int atom[NAT], off[NAT + 1], trans[NAT];
  T dfs[NAT], e[NAT], lam[NAT], delta[NAT], et[NAT], D[NAT], xi[NAT];
  double ep[NAT];
};

// Atom of pair p of the group (off = exclusive prefix of the neighbour counts).
template <int NAT>
__device__ __forceinline__ int atom_of_pair(int p, const int* off) {
  if (NAT <= 8) {
    int k = 0;
#pragma unroll
    for (int q = 1; q < NAT; ++q) k += (p >= off[q]) ? 1 : 0;
    return k;
  }
  int lo = 0, hi = NAT - 1;   // the largest k with off[k] <= p
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Atoms of group grp and their pair offsets (a warp scan of the neighbour
// counts); ends with a barrier.
template <typename T, int NAT>
__device__ __forceinline__ void group_setup(const Args<T>& a, int grp, int count, AceGroup<T, NAT>& g) {
  static_assert(NAT <= 32, "one warp holds the group");
  const int tid = threadIdx.x;
  if (tid < 32) {
    const int idx = grp * NAT + tid;
    const int i = (tid < NAT && idx < count) ? APIP_CHK(a.status, BND_COMPACT, a.ace_list[idx], a.n) : -1;
    const int nn = i >= 0 ? APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1) : 0;
    int inc = nn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (tid >= o) inc += y;
    }
    if (tid < NAT) {
      g.atom[tid] = i;
      g.off[tid + 1] = inc;
    }
    if (tid == 0) g.off[0] = 0;
  }
  __syncthreads();
}

// Float32 path: the switch of the group's transition atoms (dlam != 0 after pass
// 2), recomputed with accurate pair distances and sums of Eq. 6.  Pass 2 takes
// w-bar_i and sum_k g_k w(r_ik) in float32 from float32 distances, whose
// reciprocal square root is biased at ~1e-7; through dlam/dd and E^prec - E^EAM
// (several eV for a pure-ACE precise model) that would be ~1e-5 eV of energy.
// Only atoms with 0 < lam < 1 need it (elsewhere lam is 0 or 1 up to terms cubic
// in the float error), and they are all compacted.  One warp per transition atom,
// lanes over its neighbour list: r in float-float from the exact fixed-point
// separation (error-free squares and sums, a correctly rounded square root and one
// correction), the t of Eq. S1 in float-float, the quintic in float32, the sums in
// float-float; then d, lam = 1 - f_trans(d) and dlam in float64 (a few operations
// per atom).  The results replace the atom's lam, dlam, w-bar and d (read by
// atom_scalars).  Ends with a barrier.
template <typename T, int NAT>
__device__ __forceinline__ void refine_switch(const Args<T>& a, const AceGroup<T, NAT>& g) {
  if constexpr (sizeof(T) == 4) {
    if (a.lam_mode == APIP_LAM_PAPER || a.lam_mode == APIP_LAM_LEARNED) {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const SwFF& sw = a.swff;
      for (int k = warp; k < NAT; k += kAceWarps) {
        const int i = g.atom[k];
        if (i < 0 || a.dlam[i] == T(0)) continue;   // not transitional (constant-lam atoms: dlam = 0)
        const uint4 qi = a.pv.q[i];
        const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
        FF wsum{0.f, 0.f}, gsum{0.f, 0.f};
        // one neighbour record (fixed-point position, g in .w: pass 1's posg)
        auto add = [&](const uint4& qj) {
          const FF x = ff_coord((int)(qj.x - qi.x), sw.u_hi[0], sw.u_lo[0]);
          const FF y = ff_coord((int)(qj.y - qi.y), sw.u_hi[1], sw.u_lo[1]);
          const FF z = ff_coord((int)(qj.z - qi.z), sw.u_hi[2], sw.u_lo[2]);
          // r^2: exact squares of the high parts plus the cross terms
          FF r2 = ff_prod(x.hi, x.hi);
          r2.lo = __fmaf_rn(2.f * x.hi, x.lo, r2.lo);
          FF t2 = ff_prod(y.hi, y.hi);
          t2.lo = __fmaf_rn(2.f * y.hi, y.lo, t2.lo);
          r2 = ff_add(r2, t2);
          t2 = ff_prod(z.hi, z.hi);
          t2.lo = __fmaf_rn(2.f * z.hi, z.lo, t2.lo);
          r2 = ff_add(r2, t2);
          if (!(r2.hi < sw.rw2)) return;
          float w = 1.f;
          if (r2.hi > sw.rw_lo2) {
            // r = sqrt(r2): the rounded root r_h leaves r2 - r_h^2 exact (FMA)
            const float rh = __fsqrt_rn(r2.hi);
            const float rl = __fdividef(__fadd_rn(__fmaf_rn(-rh, rh, r2.hi), r2.lo), 2.f * rh);
            // t = (r_w + r_w_lo - 2r) / width: c_hi - 2 r_h is exact (Sterbenz)
            // (clamped: the bounds above are rounded outwards)
            const float t = fminf(1.f, fmaxf(-1.f, __fmul_rn(__fadd_rn(__fsub_rn(sw.c_hi, 2.f * rh),
                                                                         __fsub_rn(sw.c_lo, 2.f * rl)),
                                                               sw.inv_w)));
            const float p = 1.f + t;
            w = 0.0625f * p * p * p * (8.f + t * (-9.f + 3.f * t));
          }
          wsum = ff_add(wsum, FF{w, 0.f});
          gsum = ff_add(gsum, ff_prod(__uint_as_float(qj.w), w));
        };
        // two list entries per lane and round, their loads issued before the arithmetic
        for (int s = lane; s < cnt; s += 64) {
          const bool two = s + 32 < cnt;
          const int j0 = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
          const int j1 = two ? APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)(s + 32) * a.nmax + i], a.n) : j0;
          const uint4 q0 = a.posg[j0], q1 = a.posg[j1];
          add(q0);
          if (two) add(q1);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          wsum = ff_add(wsum, FF{__shfl_xor_sync(0xffffffffu, wsum.hi, o), __shfl_xor_sync(0xffffffffu, wsum.lo, o)});
          gsum = ff_add(gsum, FF{__shfl_xor_sync(0xffffffffu, gsum.hi, o), __shfl_xor_sync(0xffffffffu, gsum.lo, o)});
        }
        if (lane == 0) {
          const double wb = 1.0 + ((double)wsum.hi + (double)wsum.lo);   // the self term, w(0) = 1
          const double d = ((double)gsum.hi + (double)gsum.lo + (double)a.g[i]) / wb - a.sw.d0;
          double dl;
          const double lam = ftrans_c(d, a.sw.d_lo, a.sw.d_hi, a.sw.inv_d, &dl);
          a.lam[i] = (T)lam;
          a.dlam[i] = (T)dl;
          a.wbar[i] = (T)wb;
          a.dd[i] = (T)d;
        }
      }
    }
  }
  __syncthreads();
}

// Step 1: A[c * NAT + k] += a_scale sum_j R Y (A zeroed by the caller; RY is a
// staging area of ry_elems<LMAX>() elements).  The pairs are taken 256 at a
// time; after their R, Y rows are staged, the (atom, component) sums are formed
// only for the atoms that have pairs in that chunk, the components of one atom
// on consecutive threads (which then read the same staged rows).  Ends with a
// barrier.
template <typename T, typename K, int LMAX, int NAT>
__device__ __forceinline__ void densities(const Args<T>& a, const AceDev<T>& t, const AceGroup<T, NAT>& g,
                                          T* A, T* RY) {
  constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  constexpr int RYS = ry_stride<LMAX>();
  const int tid = threadIdx.x;
  const int nA = t.nA;
  const T rc2 = t.rc * t.rc;
  const int total = g.off[NAT];
  for (int base = 0; base < total; base += kAceThreads) {
    const int p = base + tid;
    T* ry = RY + tid * RYS;
    bool in = false;
    V3<T> d{T(0), T(0), T(0)};
    T r2 = T(0);
    if (p < total) {
      const int k = atom_of_pair<NAT>(p, g.off);
      const int i = g.atom[k];
      const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)(p - g.off[k]) * a.nmax + i], a.n);
      d = a.pv.vec(a.pv.self(i), j);
      r2 = dot3(d, d);
      in = r2 < rc2;
    }
    if (in) {
      T r, ir;
      len_inv(r2, &r, &ir);
      T R[kNmaxCap], dR[kNmaxCap];
      radial(r, t, R, dR);
#pragma unroll
      for (int n = 0; n < kNmaxCap; ++n) ry[n] = R[n];
      for_each_ylm<T, K, LMAX, false>(d.x * ir, d.y * ir, d.z * ir,
                                      [&](int c, T y, T, T, T) { ry[kNmaxCap + c] = y; });
    } else {
#pragma unroll
      for (int q = 0; q < RYS; ++q) ry[q] = T(0);
    }
    __syncthreads();
    const int hp = min(total - base, kAceThreads);
    const int k0 = atom_of_pair<NAT>(base, g.off), k1 = atom_of_pair<NAT>(base + hp - 1, g.off);
    const int items = nA * (k1 - k0 + 1);
    for (int item = tid; item < items; item += kAceThreads) {
      const int k = k0 + item / nA, c = item - (k - k0) * nA;
      const int n = c / NLM, lm = c - n * NLM;
      const int lo = max(g.off[k] - base, 0), hi = min(g.off[k + 1] - base, hp);
      T acc = T(0);
      for (int q = lo; q < hi; ++q) acc += RY[q * RYS + n] * RY[q * RYS + kNmaxCap + lm];
      A[c * NAT + k] += acc;
    }
    __syncthreads();
  }
  for (int item = tid; item < nA * NAT; item += kAceThreads) A[item] *= t.a_scale;
  __syncthreads();
}

// Per-atom scalars of group slot k from the channels (p1, p2) (one thread per slot).
template <typename T, int NAT>
__device__ __forceinline__ void atom_scalars(const Args<T>& a, const AceDev<T>& t, int k, T p1, T p2,
                                             AceGroup<T, NAT>& g) {
  const T q2 = sqrt(p2 * p2 + t.eps * t.eps);
  const T e_ace = p1 + sqrt(q2) - t.sqrt_eps;
  g.e[k] = e_ace;
  g.dfs[k] = T(0.5) * p2 / (q2 * sqrt(q2));
  const int i = g.atom[k];
  T lam = T(0), delta = T(0), et = T(0), D = T(0), xi = T(0);
  int trans = 0;
  if (i >= 0) {
    lam = a.lam[i];
    const T e_eam = a.e_eam[i];
    // E^prec - E^EAM: E^ACE alone when the precise model adds the EAM (no float
    // cancellation of E^EAM against itself), minus the precise model's energy zero
    delta = (a.precise_adds_eam ? e_ace : e_ace - e_eam) - a.k.prec_shift;
    const T dl = a.dlam[i];
    trans = (a.grad_lambda && (a.lam_mode == APIP_LAM_PAPER || a.lam_mode == APIP_LAM_LEARNED) && dl != T(0))
                ? 1 : 0;
    et = trans ? delta * dl / a.wbar[i] : T(0);
    D = a.dd[i] + a.k.sw_d0;
    xi = a.xi_p[i];
  }
  g.lam[k] = lam; g.delta[k] = delta; g.et[k] = et; g.D[k] = D; g.xi[k] = xi; g.trans[k] = trans;
}

// Step 4 with omega W[c * NAT + k], then the per-atom energies; returns this
// thread's energy contribution (non-zero only for tid < NAT).  Ends with a barrier.
template <typename T, typename K, int LMAX, int NAT>
__device__ __forceinline__ double pair_forces(const Args<T>& a, const AceDev<T>& t, const AceGroup<T, NAT>& g,
                                              const T* W) {
  constexpr int NLM = (LMAX + 1) * (LMAX + 1);
  const int tid = threadIdx.x;
  const T rc2 = t.rc * t.rc;
  const T rcE2 = a.k.eam_rc2, rcE = a.k.eam_rc, rcE_lo = a.k.eam_rc_lo, rcE_inv = a.k.eam_inv_w;
  const T rw2 = a.k.sw_r_w2, rw = a.k.sw_r_w, rw_lo = a.k.sw_r_w_lo, rw_inv = a.k.sw_inv_w;
  // (force mixing weights the EAM force per atom in pass 2: no correction here)
  const bool eam_corr = !a.precise_adds_eam && a.eam_force && !a.force_mix;
  const int n_max = t.n_max;
  const int total = g.off[NAT];
  for (int base = 0; base < total; base += kAceThreads) {
    const int p = base + tid;
    if (p >= total) continue;
    const int k = atom_of_pair<NAT>(p, g.off);
    const int i = g.atom[k];
    const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)(p - g.off[k]) * a.nmax + i], a.n);
    const V3<T> d = a.pv.vec(a.pv.self(i), j);
    const T r2 = dot3(d, d);
    const bool trans = g.trans[k] != 0;
    const bool in_a = r2 < rc2;
    const bool in_e = eam_corr && r2 < rcE2;
    const bool in_w = trans && r2 < rw2;
    if (!(in_a || in_e || in_w)) continue;
    T r, ir;
    len_inv(r2, &r, &ir);
    const T ex = d.x * ir, ey = d.y * ir, ez = d.z * ir;
    T sr = T(0);
    T gx = T(0), gy = T(0), gz = T(0);
    if (in_a) {
      T R[kNmaxCap], dR[kNmaxCap];
      radial(r, t, R, dR);
      const T* Wk = W + k;
      for_each_ylm<T, K, LMAX, true>(ex, ey, ez, [&](int c, T y, T px, T py, T pz) {
        T u = T(0), v = T(0);
#pragma unroll
        for (int n = 0; n < kNmaxCap; ++n) {
          if (n < n_max) {
            const T w = Wk[(n * NLM + c) * NAT];
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
      const T er = a.k.eam_A * fexp(-a.k.eam_beta * (r - a.k.eam_re));
      const T drho = er * (dfc - a.k.eam_beta * fc);
      const T x = fexp(-a.k.eam_alpha * (r - a.k.eam_r0));
      const T dphi = a.k.eam_D * (T(2) * a.k.eam_alpha * (x - x * x) * fc + (x * x - T(2) * x) * dfc);
      sr -= g.lam[k] * (g.xi[k] * drho + T(0.5) * dphi);
    }
    if (in_w) {
      T dw;
      const T w = ftrans(r, rw_lo, rw, rw_inv, &dw);
      sr += g.et[k] * (a.g[j] - g.D[k]) * dw;
      scatter_add(&a.cvec[j], (double)(g.et[k] * w), a.det);
    }
    const T fx = sr * ex + gx, fy = sr * ey + gy, fz = sr * ez + gz;
    if (!a.force_mix) {
      // AP (Eq. 5): omega already carries lam_i, and the pair term is antisymmetric
      const double f0 = (double)fx, f1 = (double)fy, f2 = (double)fz;
      scatter_add(&a.force[3 * j], -f0, a.det);
      scatter_add(&a.force[3 * j + 1], -f1, a.det);
      scatter_add(&a.force[3 * j + 2], -f2, a.det);
      scatter_add(&a.force[3 * i], f0, a.det);
      scatter_add(&a.force[3 * i + 1], f1, a.det);
      scatter_add(&a.force[3 * i + 2], f2, a.det);
    } else {
      // force mixing (Eq. 3): each receiving atom takes its own lam of the precise
      // model's force (omega without lam)
      const T wj = a.lam[j], wi = g.lam[k];
      if (wj != T(0)) {
        atomicAdd(&a.force[3 * j], -(double)(wj * fx));
        atomicAdd(&a.force[3 * j + 1], -(double)(wj * fy));
        atomicAdd(&a.force[3 * j + 2], -(double)(wj * fz));
      }
      if (wi != T(0)) {
        atomicAdd(&a.force[3 * i], (double)(wi * fx));
        atomicAdd(&a.force[3 * i + 1], (double)(wi * fy));
        atomicAdd(&a.force[3 * i + 2], (double)(wi * fz));
      }
    }
  }
  double e_part = 0.0;
  if (tid < NAT) {
    const int i = g.atom[tid];
    if (i >= 0) {
      if (g.trans[tid]) scatter_add(&a.cvec[i], (double)g.et[tid], a.det);
      a.e_ace[i] = g.e[tid];
      const double ed = (double)g.lam[tid] * (double)g.delta[tid];
      e_part = ed;
      if (a.e_atom) a.e_atom[i] += ed;
    }
  }
  __syncthreads();
  return e_part;
}

// The block's energy partial: the sum over its group slots of all its groups.
template <typename T, int NAT>
__device__ __forceinline__ void block_energy(const Args<T>& a, AceGroup<T, NAT>& g, double e_part) {
  const int tid = threadIdx.x;
  if (tid < NAT) g.ep[tid] = e_part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < NAT; ++k) s += g.ep[k];
    a.partials[a.n_part_p1 + blockIdx.x] = s;
  }
}

}  // namespace apip
