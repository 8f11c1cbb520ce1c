// ACE evaluation for body order <= 3 (the streamed kernel).  One thread block
// (8 warps) handles a group of NAT compacted atoms.  Thread t works on atom
// t % NAT and on the slice t / NAT of the basis: slice s takes the records and
// couplings s, s + NS, s + 2 NS, ... (NS = 256 / NAT slices).  Only A and dE/dA
// live in shared memory (layout [component][NAT]); each coupling
//   C_{(p1 p2) L M} = sum_{m1 m2} G(l1 m1, l2 m2, L M) A_{p1 m1} A_{p2 m2}
// is formed in registers by code unrolled for its (l1, l2, L), with the Gaunt
// values as compile-time offsets into constant memory (gaunt_layout.h), and
// contracted with its nu = 3 partners, B = C_{(p1 p2) l3} . A_{p3}:
//  2. forward: phi_c = sum_b c_cb B_b (compensated sums per slice, reduced over
//     the slices);
//  3. adjoint with k_b = c1_b + F'(phi_2) c2_b: dE/dC_M = sum_b k_b A_{p3 M},
//     dE/dA_{p3} += k_b C, and dE/dC back onto A_{p1}, A_{p2} through the same
//     unrolled Gaunt terms; contributions are added to dE/dA in shared memory
//     with atomic adds.  omega = dE/dA a_scale lam_i.
// Steps 1 and 4 are those of ace_device.cuh.
#pragma once

#include "ace_device.cuh"
#include "gaunt_layout.h"

namespace apip {

constexpr uint32_t kConstOne = 0xffffu;   // second index of a nu = 1 record: the constant 1

// dE/dA accumulation.  In float32 with l_max <= 3 every thread adds into its own
// private copy of dE/dA for its atom (plain read-modify-write, no two threads
// share an address); the copies are summed once at the end.  Otherwise (float64
// or l_max = 4, where the copies would not fit in shared memory) the
// contributions go to one shared dE/dA with atomic adds.
template <typename T, int LMAX>
__host__ __device__ constexpr bool stream_private() { return sizeof(T) == 4 && LMAX <= 3; }

template <bool PRIV, typename T>
__device__ __forceinline__ void acc_add(T* p, T v) {
  if constexpr (PRIV) *p += v;
  else atomicAdd(p, v);
}

// Words between the private copies of consecutive threads: nA * NAT, plus NAT
// when NAT < 32 so that the slices of one warp start in different banks.
template <int NAT>
__host__ __device__ constexpr int priv_stride(int nA) { return nA * NAT + (NAT < 32 ? NAT : 0); }

// Dynamic shared memory of k_ace_stream: A (then omega), the slice reduction,
// and dE/dA (shared, or the private copies of all slices), which also holds the
// per-pair R, Y rows of step 1.
template <typename T, int LMAX, int NAT>
__host__ __device__ inline size_t ace_stream_smem(int nA) {
  const size_t ry = (size_t)ry_elems<LMAX>();
  const size_t pa = (size_t)pool_elems<T>(nA, NAT);
  const size_t gs = stream_private<T, LMAX>()
                        ? (size_t)pool_elems<T>((kAceThreads / NAT) * priv_stride<NAT>(nA), 1)
                        : pa;
  return sizeof(T) * (pa + (size_t)2 * kAceWarps * NAT + (gs > ry ? gs : ry));
}

// One coupling of type (L1 <= L2, LL) for this thread's atom: forward adds its
// nu = 3 functions to (f1, f2); the adjoint adds their derivatives to G.
// Ak, Gk point at the atom's column of A and dE/dA (stride NAT).
template <typename T, typename K, int L1, int L2, int LL, int NAT, bool ADJ, bool PRIV>
__device__ __forceinline__ void coupling(const T* Ak, T* Gk, int a1, int a2, int pb, int pe, const Rec<T>* part,
                                         const Rec<T>& first, T dfs, Acc<T>& f1, Acc<T>& f2) {
  constexpr int N1 = 2 * L1 + 1, N2 = 2 * L2 + 1, NM = 2 * LL + 1;
  constexpr int G0 = gaunt_offset(L1, L2, LL);
  constexpr int PF = 1;   // the first partner's record arrives with the coupling's entry
  const Rec<T> pr[PF] = {first};
  T x1[N1], x2[N2], C[NM];
#pragma unroll
  for (int i = 0; i < N1; ++i) x1[i] = Ak[(a1 + i) * NAT];
#pragma unroll
  for (int j = 0; j < N2; ++j) x2[j] = Ak[(a2 + j) * NAT];
#pragma unroll
  for (int M = 0; M < NM; ++M) C[M] = T(0);
  {
    int e = G0;
#pragma unroll
    for (int i = 0; i < N1; ++i)
#pragma unroll
      for (int j = 0; j < N2; ++j)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const int M = gaunt_cand(i - L1, j - L2, v, LL);
          if (M != kNoM) {
            C[M + LL] += K::gaunt(e) * x1[i] * x2[j];
            ++e;
          }
        }
  }
  if constexpr (!ADJ) {
    // the few partners of one coupling are summed plainly, the coupling's total
    // enters the compensated per-slice sums
    T s1 = T(0), s2 = T(0);
#pragma unroll
    for (int q = 0; q < PF; ++q) {
      if (pb + q < pe) {
        const Rec<T> r = pr[q];
        const T* y = Ak + r.key * NAT;
        T d = T(0);
#pragma unroll
        for (int M = 0; M < NM; ++M) d += C[M] * y[M * NAT];
        s1 += r.k1 * d;
        s2 += r.k2 * d;
      }
    }
    // the remaining partners (a few per coupling): a plain loop, not unrolled, so
    // that the per-type coupling bodies stay small enough for the instruction cache
#pragma unroll 1
    for (int p = pb + PF; p < pe; ++p) {
      const Rec<T> r = ld(part + p);
      const T* y = Ak + r.key * NAT;
      T d = T(0);
#pragma unroll
      for (int M = 0; M < NM; ++M) d += C[M] * y[M * NAT];
      s1 += r.k1 * d;
      s2 += r.k2 * d;
    }
    f1.add(s1);
    f2.add(s2);
  } else {
    T gC[NM];
#pragma unroll
    for (int M = 0; M < NM; ++M) gC[M] = T(0);
    auto adj_partner = [&](const Rec<T>& r) {
      const T k = r.k1 + dfs * r.k2;
      const T* y = Ak + r.key * NAT;
      T* gy = Gk + r.key * NAT;
#pragma unroll
      for (int M = 0; M < NM; ++M) {
        gC[M] += k * y[M * NAT];
        acc_add<PRIV>(gy + M * NAT, k * C[M]);
      }
    };
    adj_partner(first);   // every coupling has at least one partner
#pragma unroll 1
    for (int p = pb + 1; p < pe; ++p) adj_partner(ld(part + p));
    T g1[N1], g2[N2];
#pragma unroll
    for (int i = 0; i < N1; ++i) g1[i] = T(0);
#pragma unroll
    for (int j = 0; j < N2; ++j) g2[j] = T(0);
    {
      int e = G0;
#pragma unroll
      for (int i = 0; i < N1; ++i)
#pragma unroll
        for (int j = 0; j < N2; ++j)
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            const int M = gaunt_cand(i - L1, j - L2, v, LL);
            if (M != kNoM) {
              const T w = K::gaunt(e) * gC[M + LL];
              g1[i] += w * x2[j];
              g2[j] += w * x1[i];
              ++e;
            }
          }
    }
#pragma unroll
    for (int i = 0; i < N1; ++i) acc_add<PRIV>(Gk + (a1 + i) * NAT, g1[i]);
#pragma unroll
    for (int j = 0; j < N2; ++j) acc_add<PRIV>(Gk + (a2 + j) * NAT, g2[j]);
  }
}

template <typename T, typename K, int LMAX, int NAT, bool ADJ, bool PRIV>
__device__ __forceinline__ void coupling_dispatch(const uint4& cp, const Rec<T>& first, const T* Ak, T* Gk,
                                                  const Rec<T>* part, T dfs, Acc<T>& f1, Acc<T>& f2) {
  const int a1 = (int)(cp.x & 255u), a2 = (int)((cp.x >> 8) & 255u), type = (int)(cp.x >> 16);
  const int pb = (int)cp.y, pe = (int)cp.z;
  switch (type) {
#define X(l1, l2, L)                                                                          \
  case gaunt_type(l1, l2, L):                                                                 \
    if constexpr (l2 <= LMAX && L <= LMAX)                                                    \
      coupling<T, K, l1, l2, L, NAT, ADJ, PRIV>(Ak, Gk, a1, a2, pb, pe, part, first, dfs, f1, f2);   \
    break;
    APIP_GAUNT_TYPES
#undef X
    default: break;
  }
}

#ifdef APIP_CHECK_BOUNDS
// Bounds-checked build: a coupling entry whose operand offsets, partner range or
// first partner key fall outside the tables is recorded and dispatched to no
// coupling type; a nu <= 2 record whose segments do not fit in A is recorded and
// skipped.
template <typename T>
__device__ __forceinline__ void check_coupling(int* status, uint4& cp, const Rec<T>& first, const AceDev<T>& t) {
  const int a1 = (int)(cp.x & 255u), a2 = (int)((cp.x >> 8) & 255u), pb = (int)cp.y, pe = (int)cp.z;
  bool ok = APIP_CHK(status, BND_ACE_TABLE, a1, t.nA) == a1;
  ok = APIP_CHK(status, BND_ACE_TABLE, a2, t.nA) == a2 && ok;
  ok = APIP_CHK(status, BND_ACE_TABLE, pb, pe) == pb && ok;
  ok = APIP_CHK(status, BND_ACE_TABLE, pe - 1, t.npart) == pe - 1 && ok;
  ok = APIP_CHK(status, BND_ACE_TABLE, (int)first.key, t.nA) == (int)first.key && ok;
  if (!ok) cp.x = 0xffff0000u;
}
template <typename T>
__device__ __forceinline__ bool record_ok(int* status, const Rec<T>& rc, int nA) {
  const int a1 = (int)(rc.key & 0xffffu), a2 = (int)(rc.key >> 16), len = (int)rc.len;
  bool ok = APIP_CHK(status, BND_ACE_TABLE, a1 + len - 1, nA) == a1 + len - 1;
  if ((uint32_t)a2 != kConstOne) ok = APIP_CHK(status, BND_ACE_TABLE, a2 + len - 1, nA) == a2 + len - 1 && ok;
  return ok;
}
#endif

template <typename T, typename K, int LMAX, int NAT>
__global__ void __launch_bounds__(kAceThreads, 2) k_ace_stream(Args<T> a, AceDev<T> t) {
  pdl_begin();
  // every list-build kernel of this call has completed: block 0 clears the
  // trigger (and, after a build, the binning counts) for the next step
  if (blockIdx.x == 0) end_list_build(a.flags, a.cell_count, a.ncell);
  static_assert(NAT <= 32 && 32 % NAT == 0, "a warp holds whole slices");
  constexpr int NS = kAceThreads / NAT;
  constexpr bool PRIV = stream_private<T, LMAX>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ AceGroup<T, NAT> g;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ka = tid % NAT, slice = tid / NAT;
  const int nA = t.nA;
  const int pa = pool_elems<T>(nA, NAT);
  const int ps = priv_stride<NAT>(nA);
  T* A = reinterpret_cast<T*>(smem_raw);   // A[c * NAT + k], then omega
  T* red = A + pa;
  T* G = red + 2 * kAceWarps * NAT;        // dE/dA (PRIV: copy of thread (s, k) at s * ps + k);
                                           // step 1 staging before that
  const T* Ak = A + ka;
  T* Gk = PRIV ? G + slice * ps + ka : G + ka;
  const int count = a.counts[0];
  const int ngroups = (count + NAT - 1) / NAT;
  double e_part = 0.0;
  if (blockIdx.x < ngroups) {
    // bring the basis tables into this SM's L1 while step 1 runs (they are read by
    // every group; 128-byte lines, one prefetch per thread and line)
    auto prefetch = [&](const void* p, size_t bytes) {
      const char* c = static_cast<const char*>(p);
      for (size_t o = (size_t)tid * 128; o < bytes; o += (size_t)kAceThreads * 128)
        asm volatile("prefetch.global.L1 [%0];" ::"l"(c + o));
    };
    prefetch(t.cpl, sizeof(uint4) * (size_t)t.ncpl);
    prefetch(t.cfirst, sizeof(Rec<T>) * (size_t)t.ncpl);
    prefetch(t.part, sizeof(Rec<T>) * (size_t)t.npart);
    prefetch(t.prec, sizeof(Rec<T>) * (size_t)t.npr);
  }

  for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    group_setup<T, NAT>(a, grp, count, g);
    refine_switch<T, NAT>(a, g);
    for (int c = tid; c < nA * NAT; c += kAceThreads) A[c] = T(0);
    __syncthreads();
    densities<T, K, LMAX, NAT>(a, t, g, A, G);

    // 2. embedding channels
    {
      Acc<T> f1, f2;
      // the next record is loaded while this one is evaluated
      Rec<T> rnext{};
      if (slice < t.npr) rnext = ld(t.prec + slice);
      for (int r = slice; r < t.npr; r += NS) {
        const Rec<T> rc = rnext;
        if (r + NS < t.npr) rnext = ld(t.prec + r + NS);
#ifdef APIP_CHECK_BOUNDS
        if (!record_ok(a.status, rc, nA)) continue;
#endif
        const int a1 = (int)(rc.key & 0xffffu);
        const uint32_t a2 = rc.key >> 16;
        T d = T(0);
        if (a2 == kConstOne) {
          d = Ak[a1 * NAT];
        } else {
          for (int m = 0; m < (int)rc.len; ++m) d += Ak[(a1 + m) * NAT] * Ak[((int)a2 + m) * NAT];
        }
        f1.add(rc.k1 * d);
        f2.add(rc.k2 * d);
      }
      // the next coupling's entry and first partner are loaded while this one is evaluated
      uint4 cn = make_uint4(0u, 0u, 0u, 0u);
      Rec<T> rn{};
      if (slice < t.ncpl) { cn = __ldg(t.cpl + slice); rn = ld(t.cfirst + slice); }
      for (int u = slice; u < t.ncpl; u += NS) {
        uint4 cp = cn;
        const Rec<T> rp = rn;
#ifdef APIP_CHECK_BOUNDS
        check_coupling(a.status, cp, rp, t);
#endif
        if (u + NS < t.ncpl) { cn = __ldg(t.cpl + u + NS); rn = ld(t.cfirst + u + NS); }
        coupling_dispatch<T, K, LMAX, NAT, false, PRIV>(cp, rp, Ak, Gk, t.part, T(0), f1, f2);
      }
      T v1 = f1.value(), v2 = f2.value();
#pragma unroll
      for (int o = NAT; o < 32; o <<= 1) {
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
      }
      if (lane < NAT) {
        red[(2 * warp) * NAT + lane] = v1;
        red[(2 * warp + 1) * NAT + lane] = v2;
      }
    }
    __syncthreads();
    if (tid < NAT) {
      T p1 = T(0), p2 = T(0);
      for (int w = 0; w < kAceWarps; ++w) {
        p1 += red[(2 * w) * NAT + tid];
        p2 += red[(2 * w + 1) * NAT + tid];
      }
      atom_scalars<T, NAT>(a, t, tid, p1, p2, g);
    }
    if (PRIV) {
      for (int c = 0; c < nA; ++c) Gk[c * NAT] = T(0);
    } else {
      for (int c = tid; c < nA * NAT; c += kAceThreads) G[c] = T(0);
    }
    __syncthreads();

    // 3. adjoint
    {
      const T dfs = g.dfs[ka];
      Acc<T> unused1, unused2;
      // the next record is loaded while this one is evaluated
      Rec<T> rnext{};
      if (slice < t.npr) rnext = ld(t.prec + slice);
      for (int r = slice; r < t.npr; r += NS) {
        const Rec<T> rc = rnext;
        if (r + NS < t.npr) rnext = ld(t.prec + r + NS);
#ifdef APIP_CHECK_BOUNDS
        if (!record_ok(a.status, rc, nA)) continue;
#endif
        const int a1 = (int)(rc.key & 0xffffu);
        const uint32_t a2 = rc.key >> 16;
        const T k = rc.k1 + dfs * rc.k2;
        if (a2 == kConstOne) {
          acc_add<PRIV>(Gk + a1 * NAT, k);
        } else {
          for (int m = 0; m < (int)rc.len; ++m) {
            acc_add<PRIV>(Gk + (a1 + m) * NAT, k * Ak[((int)a2 + m) * NAT]);
            acc_add<PRIV>(Gk + ((int)a2 + m) * NAT, k * Ak[(a1 + m) * NAT]);
          }
        }
      }
      uint4 cn = make_uint4(0u, 0u, 0u, 0u);
      Rec<T> rn{};
      if (slice < t.ncpl) { cn = __ldg(t.cpl + slice); rn = ld(t.cfirst + slice); }
      for (int u = slice; u < t.ncpl; u += NS) {
        uint4 cp = cn;
        const Rec<T> rp = rn;
#ifdef APIP_CHECK_BOUNDS
        check_coupling(a.status, cp, rp, t);
#endif
        if (u + NS < t.ncpl) { cn = __ldg(t.cpl + u + NS); rn = ld(t.cfirst + u + NS); }
        coupling_dispatch<T, K, LMAX, NAT, true, PRIV>(cp, rp, Ak, Gk, t.part, dfs, unused1, unused2);
      }
    }
    __syncthreads();
    // omega = dE/dA a_scale lam into the A region (A is not read again)
    for (int item = tid; item < nA * NAT; item += kAceThreads) {
      const int k = item % NAT;
      T v;
      if (PRIV) {
        const int c = item / NAT;
        v = T(0);
        for (int sl = 0; sl < NS; ++sl) v += G[sl * ps + c * NAT + k];
      } else {
        v = G[item];
      }
      A[item] = v * t.a_scale * (a.force_mix ? T(1) : g.lam[k]);
    }
    __syncthreads();
    e_part += pair_forces<T, K, LMAX, NAT>(a, t, g, A);
  }
  block_energy<T, NAT>(a, g, e_part);
}

template <typename T, typename K, int LMAX, int NAT>
void launch_stream_lk(const Args<T>& a, const AceDev<T>& t, int blocks, cudaStream_t s) {
  const size_t bytes = ace_stream_smem<T, LMAX, NAT>(t.nA);
  cudaFuncSetAttribute(k_ace_stream<T, K, LMAX, NAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  launch_pdl(k_ace_stream<T, K, LMAX, NAT>, blocks, kAceThreads, bytes, s, a, t);
}

template <typename T, typename K, int LMAX, int NAT>
int occupancy_stream_lk(int nA) {
  const size_t bytes = ace_stream_smem<T, LMAX, NAT>(nA);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (bytes + (size_t)1024 > (size_t)optin) return 0;
  if (cudaFuncSetAttribute(k_ace_stream<T, K, LMAX, NAT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bytes) != cudaSuccess)
    return 0;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_ace_stream<T, K, LMAX, NAT>, kAceThreads, bytes) !=
      cudaSuccess)
    return 0;
  return occ;
}

template <typename T, typename K, int NAT>
int stream_k(const Args<T>* a, const AceDev<T>& t, int blocks, cudaStream_t s, bool query) {
  switch (t.l_max) {
#define APIP_CASE(L)                                           \
  case L:                                                      \
    if (query) return occupancy_stream_lk<T, K, L, NAT>(t.nA); \
    launch_stream_lk<T, K, L, NAT>(*a, t, blocks, s);          \
    return 0;
    APIP_CASE(0) APIP_CASE(1) APIP_CASE(2) APIP_CASE(3)
    default: APIP_CASE(4)
#undef APIP_CASE
  }
}

template <typename T, typename K>
int stream_dispatch(const Args<T>* a, const AceDev<T>& t, int blocks, cudaStream_t s, bool query) {
  switch (t.group) {
    case 32: return stream_k<T, K, 32>(a, t, blocks, s, query);
    case 8: return stream_k<T, K, 8>(a, t, blocks, s, query);
    case 4: return stream_k<T, K, 4>(a, t, blocks, s, query);
    default: return 0;
  }
}

}  // namespace apip
