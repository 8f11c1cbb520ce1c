// ACE evaluation for body order 4 (the pool kernel).  One thread block (8 warps)
// handles a group of KA compacted atoms at a time, with the per-atom pool
// X = [1 | A | C] and its adjoint in shared memory (layout [pool index][KA]):
//  1. A (ace_device.cuh);
//  2. C_{(p1 p2) L M} = sum G(l1 m1, l2 m2, L M) A_{p1 m1} A_{p2 m2} (a thread per
//     component); then phi_c = sum_b c_cb X_{s1(b)} . X_{s2(b)} over the basis
//     records (a thread per record, compensated sums per atom);
//  3. the adjoint dE/dX: a thread per pool value gathers its segment's reverse
//     row (sum of k_b X_partner, k_b = c1_b + F'(phi_2) c2_b); then dE/dC goes
//     back onto A through the Gaunt entries, grouped by target A component and
//     cut into pieces whose partial sums are reduced per target.  No atomics.
//     omega = dE/dA a_scale lam_i;
//  4. pair forces (ace_device.cuh).
#pragma once

#include "ace_device.cuh"

namespace apip {

// Dynamic shared memory of k_ace_pool: the pool X, its adjoint (which also holds
// the per-pair R, Y rows of step 1), and the block reduction.
template <typename T, int LMAX, int KA>
__host__ __device__ inline size_t ace_pool_smem(int npool) {
  const size_t ry = (size_t)ry_elems<LMAX>();
  const size_t px = (size_t)pool_elems<T>(npool, KA);
  return sizeof(T) * (px + (px > ry ? px : ry) + (size_t)2 * kAceWarps * KA);
}

template <typename T, typename K, int LMAX, int KA>
__global__ void __launch_bounds__(kAceThreads) k_ace_pool(Args<T> a, AceDev<T> t) {
  pdl_begin();
  // every list-build kernel of this call has completed: block 0 clears the
  // trigger (and, after a build, the binning counts) for the next step
  if (blockIdx.x == 0) end_list_build(a.flags, a.cell_count, a.ncell);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ AceGroup<T, KA> g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nA = t.nA, npool = t.npool, c0 = 1 + nA;
  const int px = pool_elems<T>(npool, KA);
  constexpr int RY = ry_elems<LMAX>();
  T* X = reinterpret_cast<T*>(smem_raw);   // X[q * KA + k]
  T* G = X + px;                           // dE/dX, same layout
  T* red = G + (px > RY ? px : RY);
  T* A = X + KA;                           // A[c * KA + k] = X[(1 + c) * KA + k]
  T* W = G + KA;                           // omega, same layout as A
  const int count = a.counts[0];
  const int ngroups = (count + KA - 1) / KA;
  double e_part = 0.0;

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    group_setup<T, KA>(a, grp, count, g);
    refine_switch<T, KA>(a, g);
    for (int c = tid; c < c0 * KA; c += kAceThreads) X[c] = (c < KA) ? T(1) : T(0);
    __syncthreads();
    densities<T, K, LMAX, KA>(a, t, g, A, G);

    // 2a. Gaunt couplings of pairs of A segments
    for (int c = tid; c < t.nC; c += kAceThreads) {
      const uint2 cp = __ldg(t.comp + c);
      const T* x1 = X + (cp.x & 0xffffu) * KA;
      const T* x2 = X + (cp.x >> 16) * KA;
      const int g0 = (int)(cp.y >> 8), g1 = g0 + (int)(cp.y & 255u);
      T acc[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) acc[k] = T(0);
#pragma unroll 4
      for (int e = g0; e < g1; ++e) {
        const Ent<T> ge = ld(t.gent + e);
        const T* u = x1 + (ge.key & 255u) * KA;
        const T* v = x2 + (ge.key >> 8) * KA;
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] += ge.v * u[k] * v[k];
      }
#pragma unroll
      for (int k = 0; k < KA; ++k) X[(c0 + c) * KA + k] = acc[k];
    }
    __syncthreads();

    // 2b. embedding channels: one dot product of two pool segments per record
    {
      Acc<T> f1[KA], f2[KA];
      for (int r = tid; r < t.nf; r += kAceThreads) {
        const Rec<T> rc = ld(t.frec + r);
        const T* u = X + (rc.key & 0xffffu) * KA;
        const T* v = X + (rc.key >> 16) * KA;
        T dot[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) dot[k] = T(0);
#pragma unroll 3
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
      atom_scalars<T, KA>(a, t, tid, p1, p2, g);
    }
    __syncthreads();

    // 3a. dE/dX: each pool value gathers the reverse row of its segment
    {
      T dfs[KA];
#pragma unroll
      for (int k = 0; k < KA; ++k) dfs[k] = g.dfs[k];
      for (int q = 1 + tid; q < npool; q += kAceThreads) {
        const int4 qr = __ldg(t.qrow + q);
        T acc[KA];
#pragma unroll
        for (int k = 0; k < KA; ++k) acc[k] = T(0);
#pragma unroll 4
        for (int e = qr.x; e < qr.y; ++e) {
          const Rec<T> rc = ld(t.arec + e);
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
      const int e1 = __ldg(t.poff + pc + 1);
#pragma unroll 4
      for (int e = __ldg(t.poff + pc); e < e1; ++e) {
        const Ent<T> b = ld(t.bent + e);
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
      W[item] = s * t.a_scale * (a.force_mix ? T(1) : g.lam[k]);
    }
    __syncthreads();
    e_part += pair_forces<T, K, LMAX, KA>(a, t, g, W);
  }
  block_energy<T, KA>(a, g, e_part);
}

template <typename T, typename K, int LMAX, int KA>
void launch_pool_lk(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  const size_t bytes = ace_pool_smem<T, LMAX, KA>(t.npool);
  cudaFuncSetAttribute(k_ace_pool<T, K, LMAX, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  launch_pdl(k_ace_pool<T, K, LMAX, KA>, blocks, kAceThreads, bytes, s, a, t);
}

// Resident blocks per SM for this pool size (0 if it does not fit).
template <typename T, typename K, int LMAX, int KA>
int occupancy_pool_lk(int npool) {
  const size_t bytes = ace_pool_smem<T, LMAX, KA>(npool);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes + (size_t)1024 > (size_t)optin) return 0;
  if (cudaFuncSetAttribute(k_ace_pool<T, K, LMAX, KA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
      cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ace_pool<T, K, LMAX, KA>, kAceThreads, bytes) !=
      cudaSuccess)
    return 0;
  return occ;
}

// launch (occ == nullptr) or occupancy query for (l_max, group)
template <typename T, typename K, int KA>
int pool_k(const Args<T>* a, const AceDev<T>& t, int blocks, cudaStream_t s, bool query) {
  switch (t.l_max) {
#define APIP_CASE(L)                                          \
  case L:                                                     \
    if (query) return occupancy_pool_lk<T, K, L, KA>(t.npool); \
    launch_pool_lk<T, K, L, KA>(*a, t, blocks, s);            \
    return 0;
    APIP_CASE(0) APIP_CASE(1) APIP_CASE(2) APIP_CASE(3)
    default: APIP_CASE(4)
#undef APIP_CASE
  }
}

template <typename T, typename K>
int pool_dispatch(const Args<T>* a, const AceDev<T>& t, int blocks, cudaStream_t s, bool query) {
  switch (t.group) {
    case 8: return pool_k<T, K, 8>(a, t, blocks, s, query);
    case 4: return pool_k<T, K, 4>(a, t, blocks, s, query);
    case 2: return pool_k<T, K, 2>(a, t, blocks, s, query);
    case 1: return pool_k<T, K, 1>(a, t, blocks, s, query);
    default: return 0;
  }
}

}  // namespace apip
