// All-atom passes of the adaptive-precision force pipeline: position
// preparation, the cell-binned neighbour list, the one-off CSP pair detection,
// pass 1 (EAM density and CSP^list g), pass 2 (switch, unweighted EAM force and
// stream compaction of lam > 0), the CSP part of the grad-lambda force, the
// float64 reductions and the velocity-Verlet kernels.
#include <cuda_runtime.h>

#include "kernels.h"

namespace apip {

namespace {

__device__ __forceinline__ double wrap1(double x, double L, double invL) {
  double w = x - L * floor(x * invL);
  if (w >= L) w -= L;
  if (w < 0.0) w += L;
  return w;
}

// The rare branch of wrap_near, kept out of line so that the compiler cannot
// turn it into predicated float64 instructions issued for every atom.
__device__ __noinline__ double wrap1_slow(double x, double L, double invL) { return wrap1(x, L, invL); }

// wrap1 for a position that is normally already in [0, L) (the drift of one
// step): the range test is made on the bit patterns (non-negative doubles order
// as integers), which keeps it off the float64 pipe.
__device__ __forceinline__ double wrap_near(double x, double L, double invL) {
  const long long b = __double_as_longlong(x), bl = __double_as_longlong(L);
  if (b >= 0 && b < bl) return x;
  return wrap1_slow(x, L, invL);
}

// isfinite from the exponent bits.
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000;
}

__device__ __forceinline__ int cell_of(double xw, double L, int nc) {
  int c = (int)(xw * ((double)nc / L));
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// Duties shared by k_prep and the drift of the Verlet kernels for atom i at
// position (x, y, z): finiteness and id checks, the id -> index map, the
// fixed-point coordinates (FP32 path) and the neighbour-list trigger
// (displacement since the last build > skin / 2).  In the FP32 path the
// displacement is taken from the fixed-point coordinates (integer differences),
// which keeps float64 arithmetic out of this per-atom work; ``wrapped`` says that
// (x, y, z) already lie in [0, L).
template <typename T>
__device__ __forceinline__ float prep_atom(const Args<T>& a, int i, double x, double y, double z,
                                           bool wrapped = false) {
  if (!finite_bits(x) || !finite_bits(y) || !finite_bits(z)) atomicOr(&a.status[ST_BAD_INPUT], 1);
  const int idv = a.id[i];
  if (idv < 0 || idv >= a.nmax) atomicOr(&a.status[ST_BAD_INPUT], 1);
  else a.id2idx[idv] = i;
  if (sizeof(T) == 4) {
    const double xs[3] = {x, y, z};
    unsigned int q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
      q[k] = fixed_coord(wrapped ? xs[k] : wrap1(xs[k], a.geo.L[k], a.geo.invL[k]), a.geo.unit_m[k], a.geo.unit_s[k]);
    a.posq[i] = make_uint4(q[0], q[1], q[2], 0u);
    const uint4 r = a.posq_ref[i];
    const float ex = (float)(int)(q[0] - r.x) * a.geo.unit[0], ey = (float)(int)(q[1] - r.y) * a.geo.unit[1],
                ez = (float)(int)(q[2] - r.z) * a.geo.unit[2];
    const float e2 = ex * ex + ey * ey + ez * ez;
    if (e2 > a.skin_half2_f) atomicOr(&a.flags[0], 1);
    return e2;
  }
  double dx = x - a.pos_ref[3 * i], dy = y - a.pos_ref[3 * i + 1], dz = z - a.pos_ref[3 * i + 2];
  dx -= a.geo.L[0] * rint(dx * a.geo.invL[0]);
  dy -= a.geo.L[1] * rint(dy * a.geo.invL[1]);
  dz -= a.geo.L[2] * rint(dz * a.geo.invL[2]);
  if (dx * dx + dy * dy + dz * dz > a.skin_half2) atomicOr(&a.flags[0], 1);
  return 0.f;
}

// FP32 path: the block's largest squared displacement since the list build into
// the running maximum flags[1] (float bits; non-negative floats order as
// integers), one atomic per block.  Called by every thread of the block.
template <typename T>
__device__ __forceinline__ void note_displacement(const Args<T>& a, float e2) {
  if constexpr (sizeof(T) == 4) {
    __shared__ int wmax[kBlock / 32];
    const int m = __reduce_max_sync(0xffffffffu, __float_as_int(e2));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      int b = wmax[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = max(b, wmax[w]);
      atomicMax(&a.flags[1], b);
    }
  }
}

template <typename T>
__global__ void k_prep(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) a.counts[0] = a.counts[1] = 0;
  float e2 = 0.f;
  if (i < a.n) e2 = prep_atom(a, i, a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2]);
  note_displacement(a, e2);
}

// ------------------------------------------------------------ neighbour list
// Two launches per list build (binning, fill), each returning at once when no
// build is due: cell_count is zero before a build (zeroed on allocation, and after
// each build by end_list_build, which also clears the trigger).

// The cell of atom i: FP32 path from its fixed-point coordinates (integer
// arithmetic, floor(q nc / 2^32)), FP64 path from the wrapped position.
template <typename T>
__device__ __forceinline__ void atom_cell(const Args<T>& a, int i, int c[3]) {
  if constexpr (sizeof(T) == 4) {
    const uint4 q = a.posq[i];
    const unsigned qq[3] = {q.x, q.y, q.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = (int)(((unsigned long long)qq[k] * (unsigned)a.geo.nc[k]) >> 32);
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      c[k] = cell_of(wrap1(a.pos[3 * i + k], a.geo.L[k], a.geo.invL[k]), a.geo.L[k], a.geo.nc[k]);
  }
}

// Binning: each atom takes a slot of its cell (the order of the slots follows
// the atomics, so neighbour order within a cell is not fixed and every sum over
// neighbours is order-independent up to rounding, unless the deterministic mode
// sorts the cells); FP32 path: the member's fixed-point position is copied into
// cell order for the fill.
template <typename T>
__global__ void k_bin(Args<T> a) {
  pdl_begin();
  if (!a.flags[0]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int c[3];
  atom_cell(a, i, c);
  const int cell = (c[2] * a.geo.nc[1] + c[1]) * a.geo.nc[0] + c[0];
  const int slot = atomicAdd(&a.cell_count[cell], 1);
  if (slot < a.cell_cap) {
    if constexpr (sizeof(T) == 4) {
      const uint4 q = a.posq[i];
      a.cell_q[(size_t)cell * a.cell_cap + slot] = make_uint4(q.x, q.y, q.z, (unsigned)i);
    } else {
      a.cell_atoms[cell * a.cell_cap + slot] = i;
    }
  } else {
    atomicOr(&a.status[ST_CELL_OVERFLOW], 1);
    atomicMax(&a.status[ST_MAX_CELL], slot + 1);
  }
}

// Deterministic mode, on a build: each cell's members sorted by atom index (one
// thread per cell, insertion sort: a cell holds a few atoms), so that the list's
// order, and with it every sum over neighbours, does not depend on the order of
// the binning atomics.
template <typename T>
__global__ void k_cell_sort(Args<T> a) {
  pdl_begin();
  if (!a.flags[0]) return;
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= a.ncell) return;
  const int m = min(a.cell_count[cell], a.cell_cap);
  if constexpr (sizeof(T) == 4) {
    uint4* v = a.cell_q + (size_t)cell * a.cell_cap;
    for (int k = 1; k < m; ++k) {
      const uint4 x = v[k];
      int p = k;
      for (; p > 0 && v[p - 1].w > x.w; --p) v[p] = v[p - 1];
      v[p] = x;
    }
  } else {
    int* v = a.cell_atoms + (size_t)cell * a.cell_cap;
    for (int k = 1; k < m; ++k) {
      const int x = v[k];
      int p = k;
      for (; p > 0 && v[p - 1] > x; --p) v[p] = v[p - 1];
      v[p] = x;
    }
  }
}

// One thread per atom.  Each candidate within r_list is classed by its distance:
// 0 within the EAM cutoff, 1 within the EAM cutoff + skin, 2 beyond.  Class 0
// goes straight to the list, classes 1 and 2 to the two ends of the atom's
// column of the scratch list; at the end they are copied behind class 0, so the
// list holds class 0, then 1, then 2, each in cell order.  The passes' EAM sums
// stop at nnb_e (classes 0 and 1: a pair now within the EAM cutoff was within
// cutoff + skin at the build, since each atom has moved less than skin / 2), and
// the class order keeps the lanes of a warp on the same branch of those sums.
template <typename T>
__global__ void k_nbfill(Args<T> a) {
  pdl_begin();
  if (!a.flags[0]) return;
  // the new list's reference positions are the current ones: no displacement yet
  if (blockIdx.x == 0 && threadIdx.x == 0) a.flags[1] = 0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  int c[3];
  atom_cell(a, i, c);
  const auto si = a.pv.self(i);
  const T rin2 = T(a.r_e_in2), rmid2 = T(a.r_e_mid2);
  int n0 = 0, n1 = 0, n2 = 0;   // class counts
  int w1 = 0, w2 = 0;           // class 1, 2 entries written to the scratch ends
  T min1 = T(INFINITY);         // least squared distance in class 1
  auto keep = [&](int j, T r2) {
    if (r2 < rin2) {
      if (n0 < a.max_nb) a.nbl[(size_t)n0 * a.nmax + i] = j;
      ++n0;
    } else if (r2 < rmid2) {
      if (w1 + w2 < a.max_nb) a.nbl_tmp[(size_t)(w1++) * a.nmax + i] = j;   // the ends meet only on overflow
      min1 = r2 < min1 ? r2 : min1;
      ++n1;
    } else {
      if (w1 + w2 < a.max_nb) a.nbl_tmp[(size_t)(a.max_nb - 1 - w2++) * a.nmax + i] = j;
      ++n2;
    }
  };
  // FP32 path: the squared distance from the atom to the nearest face of the
  // neighbour cell at offset -1, 0, +1 along each axis, from the atom's fraction
  // within its own cell (the low 32 bits of q * nc, exact); a cell whose nearest
  // point is beyond r_list (with a 1e-5 relative margin, far above the rounding of
  // these gaps) holds no candidate and is skipped.  Only with at least 5 cells per
  // axis, where no member of a neighbour cell is nearer through the other side of
  // the box.
  float lo2[3] = {0.f, 0.f, 0.f}, hi2[3] = {0.f, 0.f, 0.f};
  float prune2 = INFINITY;
  if constexpr (sizeof(T) == 4) {
    if (a.geo.nc[0] >= 5 && a.geo.nc[1] >= 5 && a.geo.nc[2] >= 5) {
      const unsigned qq[3] = {si.q.x, si.q.y, si.q.z};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const unsigned frac = (unsigned)((unsigned long long)qq[k] * (unsigned)a.geo.nc[k]);
        const float w = a.pv.unit[k] / (float)a.geo.nc[k];
        const float lo = (float)frac * w, hi = (4294967296.0f - (float)frac) * w;
        lo2[k] = lo * lo;
        hi2[k] = hi * hi;
      }
      prune2 = (float)(a.r_list2 * (1.0 + 1e-5));
    }
  }
  auto gap = [&](int k, int d) { return d < 0 ? lo2[k] : (d > 0 ? hi2[k] : 0.f); };
  for (int dz = -1; dz <= 1; ++dz) {
    const int cz = (c[2] + dz + a.geo.nc[2]) % a.geo.nc[2];
    for (int dy = -1; dy <= 1; ++dy) {
      const int cy = (c[1] + dy + a.geo.nc[1]) % a.geo.nc[1];
      const float gzy = gap(2, dz) + gap(1, dy);
      for (int dx = -1; dx <= 1; ++dx) {
        if (gzy + gap(0, dx) > prune2) continue;
        const int cx = (c[0] + dx + a.geo.nc[0]) % a.geo.nc[0];
        const int cell = APIP_CHK(a.status, BND_CELL, (cz * a.geo.nc[1] + cy) * a.geo.nc[0] + cx, a.ncell);
        const int m = min(a.cell_count[cell], a.cell_cap);
        if constexpr (sizeof(T) == 4) {
          // float comparison against r_list^2 rounded up: the list holds every pair
          // whose float distance is below r_list (and perhaps a few at r_list); the
          // member's index rides in .w of its fixed-point position
          const uint4* cq = a.cell_q + (size_t)cell * a.cell_cap;
          const float rl2 = __double2float_ru(a.r_list2);
#pragma unroll 2
          for (int k = 0; k < m; ++k) {
            const uint4 o = cq[k];
            const float ex = (float)(int)(o.x - si.q.x) * a.pv.unit[0];
            const float ey = (float)(int)(o.y - si.q.y) * a.pv.unit[1];
            const float ez = (float)(int)(o.z - si.q.z) * a.pv.unit[2];
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rl2 && (int)o.w != i) keep(APIP_CHK(a.status, BND_CELL, (int)o.w, a.n), r2);
          }
        } else {
          const int* v = a.cell_atoms + (size_t)cell * a.cell_cap;
          for (int k = 0; k < m; ++k) {
            const int j = APIP_CHK(a.status, BND_CELL, v[k], a.n);
            if (j == i) continue;
            const auto d = a.pv.vec(si, j);
            const T r2 = dot3(d, d);
            if ((double)r2 < a.r_list2) keep(j, r2);
          }
        }
      }
    }
  }
  const int cnt = n0 + n1 + n2;
  if (cnt > a.max_nb) {
    atomicOr(&a.status[ST_NB_OVERFLOW], 1);
    atomicMax(&a.status[ST_MAX_NNB], cnt);
  }
  // the kept entries: the first max_nb in class order
  const int k0 = min(n0, a.max_nb), k1 = min(w1, a.max_nb - k0), k2 = min(w2, a.max_nb - k0 - k1);
  for (int s = 0; s < k1; ++s) a.nbl[(size_t)(k0 + s) * a.nmax + i] = a.nbl_tmp[(size_t)s * a.nmax + i];
  for (int s = 0; s < k2; ++s)
    a.nbl[(size_t)(k0 + k1 + s) * a.nmax + i] = a.nbl_tmp[(size_t)(a.max_nb - 1 - s) * a.nmax + i];
  a.nnb[i] = k0 + k1 + k2;
  a.nnb_e[i] = k0 + k1;
  if constexpr (sizeof(T) == 4) {
    a.nnb_0[i] = k0;
    a.mind1[i] = k1 < n1 ? 0.f : min1;   // a class-1 entry dropped on overflow: never skip class 1
  }
  // the positions of this build: the FP64 path's displacement reference, and in
  // both paths what a checkpoint keeps to rebuild the same list on resume
  if (sizeof(T) == 4) a.posq_ref[i] = a.posq[i];
  a.pos_ref[3 * i] = a.pos[3 * i];
  a.pos_ref[3 * i + 1] = a.pos[3 * i + 1];
  a.pos_ref[3 * i + 2] = a.pos[3 * i + 2];
}

// -------------------------------------------------------------- CSP pairs
// Detection at t = 0 (Eq. B3): the csp_nnb nearest neighbours within
// csp_rcut (ordered by squared distance, ties by id) are paired greedily by
// ascending |r_ia + r_ib|^2 (ties by rank).  All float64 operations are
// explicitly rounded (no contraction) so the pairing is reproducible.
__device__ __forceinline__ double sq_rn(double x, double y, double z) {
  return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

__device__ __forceinline__ double minimg_rn(double d, double L) {
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

__global__ void k_csp_init(Args<double> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double r2s[kCspCap], rv[kCspCap][3];
  int ids[kCspCap];
  int m = 0;
  const int K = a.csp_nnb;
  const double xi = a.pos[3 * i], yi = a.pos[3 * i + 1], zi = a.pos[3 * i + 2];
  const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
  for (int s = 0; s < cnt; ++s) {
    const int j = APIP_CHK(a.status, BND_NEIGHBOUR, a.nbl[(size_t)s * a.nmax + i], a.n);
    const double dx = minimg_rn(__dsub_rn(a.pos[3 * j], xi), a.geo.L[0]);
    const double dy = minimg_rn(__dsub_rn(a.pos[3 * j + 1], yi), a.geo.L[1]);
    const double dz = minimg_rn(__dsub_rn(a.pos[3 * j + 2], zi), a.geo.L[2]);
    const double r2 = sq_rn(dx, dy, dz);
    if (!(r2 < a.csp_rcut2)) continue;
    const int idj = a.id[j];
    // insert into the sorted list of the K best (r2, id)
    if (m == K && !(r2 < r2s[K - 1] || (r2 == r2s[K - 1] && idj < ids[K - 1]))) continue;
    if (m < K) ++m;
    int p = m - 1;
    while (p > 0 && (r2 < r2s[p - 1] || (r2 == r2s[p - 1] && idj < ids[p - 1]))) {
      r2s[p] = r2s[p - 1]; ids[p] = ids[p - 1];
      rv[p][0] = rv[p - 1][0]; rv[p][1] = rv[p - 1][1]; rv[p][2] = rv[p - 1][2];
      --p;
    }
    r2s[p] = r2; ids[p] = idj; rv[p][0] = dx; rv[p][1] = dy; rv[p][2] = dz;
  }
  const int idv = a.id[i];   // rows are kept by atom id, so atoms may be reordered later
  if (idv < 0 || idv >= a.nmax) return;   // reported by prep (ST_BAD_INPUT)
  int* out = a.csp + (size_t)idv * kCspCap;
  for (int k = 0; k < kCspCap; ++k) out[k] = -1;
  bool used[kCspCap];
  for (int k = 0; k < kCspCap; ++k) used[k] = false;
  for (int k = 0; 2 * k < K; ++k) {
    double best = 0.0;
    int bp = -1, bq = -1;
    for (int p = 0; p < m; ++p) {
      if (used[p]) continue;
      for (int q = p + 1; q < m; ++q) {
        if (used[q]) continue;
        const double s2 = sq_rn(__dadd_rn(rv[p][0], rv[q][0]), __dadd_rn(rv[p][1], rv[q][1]),
                                __dadd_rn(rv[p][2], rv[q][2]));
        if (bp < 0 || s2 < best) { best = s2; bp = p; bq = q; }
      }
    }
    if (bp < 0) break;
    used[bp] = used[bq] = true;
    out[2 * k] = ids[bp];
    out[2 * k + 1] = ids[bq];
  }
}

// Restored partner ids: the row of atom id i (kCspCap entries) from
// src[i * nnb .. + nnb), -1 beyond.
__global__ void k_set_csp(const int32_t* src, int* dst, int n, int nnb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int k = 0; k < kCspCap; ++k) dst[(size_t)i * kCspCap + k] = k < nnb ? src[(size_t)i * nnb + k] : -1;
}

// ------------------------------------------------------------------ pass 1
// zeta_i and E_i^EAM (Eq. B1, S8), xi'(zeta_i), and g_i = CSP^list_i (Eq. B3).
// The EAM sums read only the first nnb_e list entries (the pairs that can be
// within the EAM cutoff).  FP32 path: also writes posg[i] = (posq[i], g_i) for
// pass 2.
template <typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 8 : 4) k_pass1(Args<T> a) {
  pdl_begin();
  __shared__ double sh[32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T e_out = T(0);
  if (i < a.n) {
    const auto si = a.pv.self(i);
    const T rc2 = a.k.eam_rc2, rc = a.k.eam_rc, rlo = a.k.eam_rc_lo, inv_w = a.k.eam_inv_w;
    const T A = a.k.eam_A, beta = a.k.eam_beta, re = a.k.eam_re, D = a.k.eam_D, alpha = a.k.eam_alpha,
            r0 = a.k.eam_r0;
    const bool paper_g = a.lam_mode == APIP_LAM_PAPER;
    // FP32 path: a class-1 entry (build distance r_b in [rc, rc + skin)) is now at
    // r >= r_b - d_i - d_j, where d_i is this atom's displacement since the build
    // and d_j <= the largest one (flags[1]); when the least r_b of the atom's
    // class-1 entries is at least rc + d_i + d_max (+ a rounding margin), none of
    // them is within the cutoff and the sums stop after class 0
    int end = APIP_CHK(a.status, BND_LIST_LEN, a.nnb_e[i], a.max_nb + 1);
    if constexpr (sizeof(T) == 4) {
      const float dmax2 = __int_as_float(a.flags[1]);   // NaN (-1) before the first build: no skip
      const uint4 r = a.posq_ref[i];
      const float ex = (float)(int)(si.q.x - r.x) * a.pv.unit[0], ey = (float)(int)(si.q.y - r.y) * a.pv.unit[1],
                  ez = (float)(int)(si.q.z - r.z) * a.pv.unit[2];
      const float lim = a.k.eam_rc + sqrtf(ex * ex + ey * ey + ez * ez) + sqrtf(dmax2) + 1e-3f;
      if (a.mind1[i] >= lim * lim) end = APIP_CHK(a.status, BND_LIST_LEN, a.nnb_0[i], a.max_nb + 1);
    }
    Acc<T> zeta, pair;
    walk_list(a.nbl + i, a.nmax, 0, end, a.status, a.n, [&](int j) { return a.pv.fetch(j); },
              [&](int, const auto& o) {
                const auto d = a.pv.vec_of(si, o);
                const T r2 = dot3(d, d);
                if (r2 < rc2) {
                  T r, ir;
                  len_inv(r2, &r, &ir);
                  T dfc;
                  const T fc = ftrans(r, rlo, rc, inv_w, &dfc);
                  const T x = fexp(-alpha * (r - r0));
                  zeta.add(A * fexp(-beta * (r - re)) * fc);
                  pair.add(D * (x * x - T(2) * x) * fc);
                }
              });
    const T z = zeta.value();
    const T sz = z > T(0) ? sqrt(z) : T(0);
    const T e = -sz + T(0.5) * pair.value();
    a.zeta[i] = z;
    a.xi_p[i] = z > T(0) ? T(-0.5) / sz : T(0);
    a.e_eam[i] = e;
    const double e_ind = ind_energy(a, i);   // the external indenter, if any
    if (a.e_atom) a.e_atom[i] = (double)e + e_ind;
    e_out = e + (T)e_ind;
    T g = T(0);
    if (paper_g) {
      const int idv = a.id[i], own = a.csp_owner[i];
      const int4* c4 = reinterpret_cast<const int4*>(a.csp_idx + (size_t)i * kCspCap);
      const int4 cq0 = c4[0], cq1 = c4[1];
      // g_i = sum over the partner pairs of |r_ia + r_ib|^2 (Eq. B3).  The partner
      // ids come from the row of this atom's id; their indices from the cache of
      // the last call (valid while the atom at index i keeps its id and its
      // partners keep their indices), checked against the ids, else from the
      // id -> index map, and the cache rewritten (idx = -1: no partner, -2: id
      // out of range)
      const bool idok = idv >= 0 && idv < a.nmax;   // an invalid id: reported by prep, no partners
      const int4* pr4 = reinterpret_cast<const int4*>(a.csp + (size_t)(idok ? idv : 0) * kCspCap);
      static_assert(kCspCap == 8, "two int4 rows of partner ids");
      const int4 none = make_int4(-1, -1, -1, -1);
      const int4 p0 = idok ? pr4[0] : none, p1 = idok ? pr4[1] : none;
      int pid[kCspCap] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      int idx[kCspCap] = {cq0.x, cq0.y, cq0.z, cq0.w, cq1.x, cq1.y, cq1.z, cq1.w};
#pragma unroll
      for (int k = 0; k < kCspCap; ++k)
        if (k >= a.csp_nnb) pid[k] = -1;
      // a partner entry holds: its index (checked below), -1 for no partner, -2 for
      // an id out of range
      auto holds = [&](int k) {
        if (pid[k] < 0) return idx[k] == -1;
        if (pid[k] >= a.nmax) return idx[k] == -2;
        return idx[k] >= 0 && idx[k] < a.n && a.id[idx[k]] == pid[k];
      };
      bool hit = own == idv;
#pragma unroll
      for (int k = 0; k < kCspCap; ++k) hit = hit && holds(k);
      if (!hit) {
#pragma unroll
        for (int k = 0; k < kCspCap; ++k) idx[k] = pid[k] < 0 ? -1 : (pid[k] >= a.nmax ? -2 : a.id2idx[pid[k]]);
        int4* c4 = reinterpret_cast<int4*>(a.csp_idx + (size_t)i * kCspCap);
        c4[0] = make_int4(idx[0], idx[1], idx[2], idx[3]);
        c4[1] = make_int4(idx[4], idx[5], idx[6], idx[7]);
        a.csp_owner[i] = idv;
      }
      bool bad = false;
      Acc<T> gs;
#pragma unroll
      for (int k = 0; k < kCspCap / 2; ++k) {
        if (pid[2 * k] < 0 || pid[2 * k + 1] < 0) continue;
        // the index must hold that partner now: the id -> index map keeps the
        // entries of ids that are no longer present
        const int ia = idx[2 * k], ib = idx[2 * k + 1];
        if (ia < 0 || ib < 0 || !(hit || (holds(2 * k) && holds(2 * k + 1)))) {
          bad = true;
          continue;
        }
        const V3<T> u = csp_vec(a.pv, si, ia, ib);
        gs.add(dot3(u, u));
      }
      if (bad) {
        atomicOr(&a.status[ST_BAD_PARTNER], 1);
        a.csp_owner[i] = -2;   // looked up again next call
      }
      g = gs.value();
    }
    a.g[i] = g;
    if constexpr (sizeof(T) == 4) a.posg[i] = make_uint4(si.q.x, si.q.y, si.q.z, __float_as_uint(g));
  }
  const double tot = block_sum_t(e_out, sh);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = tot;
}

// ------------------------------------------------------------------ pass 2
// Switch (Eq. 6, Eq. 2 with lam = 1 - f_trans), the EAM force with unit weights
// F_i = sum_k [(xi'_i + xi'_k) rho'(r_ik) + Phi'(r_ik)] e_ik  (S13; the lam-
// dependent part of S12 is added by the ACE kernel for the atoms with lam > 0),
// and warp-ballot compaction of {i : lam_i > 0} into ace_list.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_pass2(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < a.n;
  T lam = T(0);
  double ind_fv = 0.0;   // this atom's indenter force . centre velocity
  if (active) {
    const auto si = a.pv.self(i);
    const bool paper = a.lam_mode == APIP_LAM_PAPER || a.lam_mode == APIP_LAM_LEARNED;
    const T rw2 = a.k.sw_r_w2, rw = a.k.sw_r_w, rwlo = a.k.sw_r_w_lo, rw_inv = a.k.sw_inv_w;
    const T rc2 = a.k.eam_rc2, rc = a.k.eam_rc, rlo = a.k.eam_rc_lo, inv_w = a.k.eam_inv_w;
    const T A = a.k.eam_A, beta = a.k.eam_beta, re = a.k.eam_re, D = a.k.eam_D, alpha = a.k.eam_alpha,
            r0 = a.k.eam_r0;
    const T xi_i = a.xi_p[i];
    // the force components keep compensated sums (their rounding decides how well
    // the float32 path conserves the total momentum); w-bar and sum g w are plain:
    // they decide the compaction here, and the ACE kernel recomputes them in float64
    // for the transition atoms, where their rounding would reach the energy
    Plain<T> wbar, S;
    Acc<T> fx, fy, fz;
    wbar.add(T(1));
    if (paper) S.add(a.g[i]);
    // one neighbour: the switch sums (w-range) and, for the first nnb_e entries,
    // the EAM force
    auto term = [&](int j, const V3<T>& d, T gj, T xij, bool eam) {
      const T r2 = dot3(d, d);
      const bool in_w = paper && r2 < rw2;
      const bool in_e = eam && a.eam_force && r2 < rc2;
      if (!(in_w || in_e)) return;
      T r, ir;
      len_inv(r2, &r, &ir);
      if (in_w) {
        T dw;
        const T w = ftrans(r, rwlo, rw, rw_inv, &dw);
        wbar.add(w);
        S.add(gj * w);
      }
      if (in_e) {
        T dfc;
        const T fc = ftrans(r, rlo, rc, inv_w, &dfc);
        const T er = A * fexp(-beta * (r - re));
        const T drho = er * (dfc - beta * fc);
        const T x = fexp(-alpha * (r - r0));
        const T dphi = D * (T(2) * alpha * (x - x * x) * fc + (x * x - T(2) * x) * dfc);
        const T sc = ((xi_i + xij) * drho + dphi) * ir;
        fx.add(sc * d.x);
        fy.add(sc * d.y);
        fz.add(sc * d.z);
      }
    };
    // neighbour records, fetched one entry ahead: FP32 the posg entry (fixed-point
    // position, g in .w) and, within nnb_e, xi'_j; FP64 the position
    const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
    const int cnt_e = APIP_CHK(a.status, BND_LIST_LEN, a.nnb_e[i], cnt + 1);
    if constexpr (sizeof(T) == 4) {
      struct RecE { uint4 o; float xi; };
      walk_list(a.nbl + i, a.nmax, 0, cnt_e, a.status, a.n, [&](int j) { return RecE{a.posg[j], a.xi_p[j]}; },
                [&](int j, const RecE& e) { term(j, a.pv.vec_of(si, e.o), __uint_as_float(e.o.w), e.xi, true); });
      if (paper)
        walk_list(a.nbl + i, a.nmax, cnt_e, cnt, a.status, a.n, [&](int j) { return a.posg[j]; },
                  [&](int j, const uint4& o) { term(j, a.pv.vec_of(si, o), __uint_as_float(o.w), T(0), false); });
    } else {
      walk_list(a.nbl + i, a.nmax, 0, cnt_e, a.status, a.n, [&](int j) { return a.pv.fetch(j); },
                [&](int j, const auto& o) { term(j, a.pv.vec_of(si, o), paper ? a.g[j] : T(0), a.xi_p[j], true); });
      if (paper)
        walk_list(a.nbl + i, a.nmax, cnt_e, cnt, a.status, a.n, [&](int j) { return a.pv.fetch(j); },
                  [&](int j, const auto& o) { term(j, a.pv.vec_of(si, o), a.g[j], T(0), false); });
    }
    T dv = T(0), dl = T(0), wb = T(1);
    if (paper) {
      wb = wbar.value();
      dv = S.value() / wb - a.k.sw_d0;
      lam = ftrans_c(dv, a.k.sw_d_lo, a.k.sw_d_hi, a.k.sw_inv_d, &dl);
    } else {
      lam = a.lam_mode == APIP_LAM_CONST1 ? T(1) : T(0);
    }
    if (a.lam_fixed) {
      const double f = a.lam_fixed[i];
      if (f == f) {   // not NaN: constant lam on this atom (Appendix B)
        lam = T(f);
        dl = T(0);
      }
    }
    a.lam[i] = lam;
    a.dlam[i] = dl;
    a.wbar[i] = wb;
    a.dd[i] = dv;
    if (a.force) {
      // force mixing (Eq. 3): this atom's EAM force enters with (1 - lam_i) from the
      // fast model plus, when the precise model contains the EAM, lam_i from it
      const T wf = a.force_mix ? T(1) - lam + (a.precise_adds_eam ? lam : T(0)) : T(1);
      double gx = (double)(wf * fx.value()), gy = (double)(wf * fy.value()), gz = (double)(wf * fz.value());
      double fi[3], ei;
      if (a.ind_on && ind_term(a, i, &ei, fi)) {   // indenter: K (R - r)^2 (x_i - c) / r
        gx += fi[0];
        gy += fi[1];
        gz += fi[2];
        ind_fv = fi[0] * a.ind_v[0] + fi[1] * a.ind_v[1] + fi[2] * a.ind_v[2];
      }
      a.force[3 * i] = fix_put(gx, a.det);
      a.force[3 * i + 1] = fix_put(gy, a.det);
      a.force[3 * i + 2] = fix_put(gz, a.det);
    }
  }
  if (a.ind_on && __syncthreads_or(ind_fv != 0.0)) {
    __shared__ double shw[32];
    const double t = block_sum(ind_fv, shw);
    if (threadIdx.x == 0) scatter_add(&a.ind_acc[2], t, a.det);
  }
  const bool pred = active && lam > T(0);
  if (a.det) {   // the block's count (k_blk_scan and k_compact_det write the list in index order)
    const int cnt = __syncthreads_count(pred);
    if (threadIdx.x == 0) {
      a.blk_cnt[blockIdx.x] = cnt;
      if (cnt) atomicAdd(&a.counts[0], cnt);
    }
    return;
  }
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(&a.counts[0], __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) a.ace_list[base + __popc(mask & ((1u << lane) - 1u))] = i;
}

// Deterministic mode: pass 2's per-block counts turned into exclusive offsets, in
// place (one block; each thread a contiguous run of counts, then a scan of the
// run totals).
__global__ void __launch_bounds__(1024) k_blk_scan(int* cnt, int nb) {
  pdl_begin();
  __shared__ int sc[1024];
  const int per = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = min((int)threadIdx.x * per, nb), b1 = min(b0 + per, nb);
  int run = 0;
  for (int b = b0; b < b1; ++b) run += cnt[b];
  sc[threadIdx.x] = run;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {   // inclusive scan of the run totals
    const int v = (int)threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
    __syncthreads();
    sc[threadIdx.x] += v;
    __syncthreads();
  }
  int off = sc[threadIdx.x] - run;
  for (int b = b0; b < b1; ++b) {
    const int v = cnt[b];
    cnt[b] = off;
    off += v;
  }
}

// Deterministic mode: the compacted list {i : lam_i > 0} in index order, each
// block at the offset k_blk_scan computed for it.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_compact_det(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool pred = i < a.n && a.lam[i] > T(0);
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int wc[kBlock / 32];
  if (lane == 0) wc[warp] = __popc(mask);
  __syncthreads();
  int off = a.blk_cnt[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += wc[w];
  if (pred) a.ace_list[APIP_CHK(a.status, BND_COMPACT, off + __popc(mask & ((1u << lane) - 1u)), a.n)] = i;
}

// Deterministic mode: the force array, summed as 64-bit fixed point by pass 2 and
// the scattering kernels, back to float64.
__global__ void k_fix_finish(double* force, int n3) {
  pdl_begin();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n3) force[k] = fix_get(force + k, 1);
}

// Indenter work by the midpoint rule over one step (dt > 0), or just the shift of
// the last (sum F).v (dt = 0, a plain force evaluation).  acc[2] holds fixed point
// in deterministic mode.
__global__ void k_ind_work(double* acc, double dt, int det) {
  pdl_begin();
  const double f = fix_get(acc + 2, det);
  acc[0] += 0.5 * dt * (acc[1] + f);
  acc[1] = f;
  acc[2] = 0.0;
}

// -------------------------------------------- grad-lambda force, CSP part
// F -= grad sum_j c_j g_j (Eq. S25-S27) for the atoms with c_j != 0, where
// c_j = sum_k Et_k w(r_kj) was accumulated by the ACE kernel; resets c_j.  One
// thread per atom in index order: the few atoms with c_j != 0 lie near the
// transition region, and neighbouring threads then gather and scatter near one
// another (a list of them in the ACE kernel's first-touch order measured slower).
template <typename T>
__global__ void k_csp_force(Args<T> a) {
  pdl_begin();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.n) return;
  // c == +-0 tested on the bits (off the float64 pipe; a zero fixed-point slot has
  // the bits of +0), so that only the few atoms with c != 0 convert it
  const double raw = a.cvec[j];
  if ((__double_as_longlong(raw) << 1) == 0) return;
  const double c = a.det ? fix_get(&raw, 1) : raw;
  a.cvec[j] = 0.0;
  const auto sj = a.pv.self(j);
  // the partners' indices as pass 1 of this call checked them (cached by atom
  // index); a row pass 1 found bad is skipped (the error is reported)
  if (a.csp_owner[j] != a.id[j]) return;
  static_assert(kCspCap == 8, "two int4 rows of partner indices");
  const int4* c4 = reinterpret_cast<const int4*>(a.csp_idx + (size_t)j * kCspCap);
  const int4 q0 = c4[0], q1 = c4[1];
  const int idx[kCspCap] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
  bool ok[kCspCap / 2];
#pragma unroll
  for (int k = 0; k < kCspCap / 2; ++k) {
    const int ia = idx[2 * k], ib = idx[2 * k + 1];
    ok[k] = ia >= 0 && ib >= 0 && ia < a.n && ib < a.n;
  }
  double fj[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < kCspCap / 2; ++k) {
    if (!ok[k]) continue;
    const int ia = idx[2 * k], ib = idx[2 * k + 1];
    const V3<T> uv = csp_vec(a.pv, sj, ia, ib);
    const double u[3] = {(double)uv.x, (double)uv.y, (double)uv.z};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      scatter_add(&a.force[3 * ia + q], -2.0 * c * u[q], a.det);
      scatter_add(&a.force[3 * ib + q], -2.0 * c * u[q], a.det);
      fj[q] += 4.0 * c * u[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) scatter_add(&a.force[3 * j + q], fj[q], a.det);
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ void neumaier(double& s, double& c, double v) {
  const double t = s + v;
  c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
  s = t;
}

__global__ void k_final(const double* partials, int n_part, double* e_total, double* e_pot_slot,
                        const double* thermo_part, int n_tb, double* thermo_slot, int* flags,
                        const int* counts, int64_t* n_ace_out, int* cell_count, int ncell) {
  pdl_begin();
  end_list_build(flags, cell_count, ncell);
  __shared__ double sh[32];
  double s = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < n_part; k += blockDim.x) neumaier(s, c, partials[k]);
  const double tot = block_sum(s, sh) + block_sum(c, sh);
  if (threadIdx.x == 0) {
    if (e_total) *e_total = tot;
    if (e_pot_slot) *e_pot_slot = tot;
    if (n_ace_out) *n_ace_out = (int64_t)counts[0];
  }
  if (thermo_part) {
    for (int q = 0; q < 4; ++q) {
      double ts = 0.0, tc = 0.0;
      for (int k = threadIdx.x; k < n_tb; k += blockDim.x) neumaier(ts, tc, thermo_part[4 * k + q]);
      const double tt = block_sum(ts, sh) + block_sum(tc, sh);
      if (threadIdx.x == 0) thermo_slot[1 + q] = q == 0 ? 0.5 * tt : tt;   // partials hold 2 E_kin
    }
  }
}

__global__ void k_thermo_final(const double* thermo_part, int n_tb, double* thermo_slot) {
  pdl_begin();
  __shared__ double sh[32];
  for (int q = 0; q < 4; ++q) {
    double ts = 0.0, tc = 0.0;
    for (int k = threadIdx.x; k < n_tb; k += blockDim.x) neumaier(ts, tc, thermo_part[4 * k + q]);
    const double tt = block_sum(ts, sh) + block_sum(tc, sh);
    if (threadIdx.x == 0) thermo_slot[1 + q] = q == 0 ? 0.5 * tt : tt;   // partials hold 2 E_kin
  }
}

// ----------------------------------------------------------------- Verlet
// MODE 0: kick + drift (the first half step of a call); MODE 1: kick + kick +
// drift (the second half of step s fused with the first half of step s + 1);
// MODE 2: the final kick.  THERMO: the kinetic-energy and momentum partials of
// the step that the first kick ends (MODE 1, 2).  Both are template parameters:
// float64 arithmetic is slow on this GPU, and a run-time test would leave the
// compiler free to issue the float64 work of the other modes as predicated-off
// instructions on every atom.
template <typename T, int MODE, bool THERMO>
__global__ void __launch_bounds__(kBlock) k_verlet(Args<T> a, double* pos, double* vel, const double* force,
                                                   const double* inv_mass, double dt, double half_dt,
                                                   double* thermo_part) {
  pdl_begin();
  static_assert(!(THERMO && MODE == 0), "no thermo output before the first force");
  __shared__ double sh4[4 * 32];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (MODE != 2 && i == 0) a.counts[0] = a.counts[1] = 0;
  double ke = 0.0, p[3] = {0.0, 0.0, 0.0};   // ke: 2 E_kin of the atom (v . p; halved after the sums)
  float e2 = 0.f;                            // squared displacement since the list build (FP32 path)
  if (i < a.n) {
    const double im = inv_mass[i];
    const double h = half_dt * im;
    double f[3], v[3], x[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) f[q] = force[3 * i + q];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = vel[3 * i + q] + h * f[q];
    if constexpr (THERMO) {
      // mass = 1/inv_mass: exact in the float64 path; a float reciprocal (relative
      // error ~1e-7 on each atom's E_kin and momentum) in the float32 path, where
      // a float64 division per atom would cost more than the rest of the kernel
      const double mass = sizeof(T) == 8 ? 1.0 / im : (double)(1.0f / (float)im);
#pragma unroll
      for (int q = 0; q < 3; ++q) p[q] = v[q] * mass;
      ke = v[0] * p[0] + v[1] * p[1] + v[2] * p[2];
    }
    if constexpr (MODE == 1) {
#pragma unroll
      for (int q = 0; q < 3; ++q) v[q] += h * f[q];
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) vel[3 * i + q] = v[q];
    if constexpr (MODE != 2) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        x[q] = wrap_near(pos[3 * i + q] + dt * v[q], a.geo.L[q], a.geo.invL[q]);
        pos[3 * i + q] = x[q];
      }
      e2 = prep_atom(a, i, x[0], x[1], x[2], true);
    }
  }
  if constexpr (MODE != 2) note_displacement(a, e2);
  if constexpr (THERMO) {
    const double vals[4] = {ke, p[0], p[1], p[2]};
    double tot[4];
    block_sum4(vals, sh4, tot);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4; ++q) thermo_part[4 * blockIdx.x + q] = tot[q];
  }
}

// ------------------------------------------------------------ inspection
template <typename T>
__global__ void k_get_field(Args<T> a, int field, void* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  double* dd = (double*)dst;
  long long* di = (long long*)dst;
  switch (field) {
    case APIP_FIELD_G: dd[i] = (double)a.g[i]; break;
    case APIP_FIELD_D: dd[i] = (double)a.dd[i]; break;
    case APIP_FIELD_WBAR: dd[i] = (double)a.wbar[i]; break;
    case APIP_FIELD_LAM: dd[i] = (double)a.lam[i]; break;
    case APIP_FIELD_DLAM: dd[i] = (double)a.dlam[i]; break;
    case APIP_FIELD_E_EAM: dd[i] = (double)a.e_eam[i]; break;
    case APIP_FIELD_E_ACE: dd[i] = a.lam[i] > T(0) ? (double)a.e_ace[i] : 0.0; break;
    case APIP_FIELD_ZETA: dd[i] = (double)a.zeta[i]; break;
    case APIP_FIELD_ACE_LIST: di[i] = i < a.counts[0] ? (long long)a.ace_list[i] : -1; break;
    case APIP_FIELD_NNB: di[i] = a.nnb[i]; break;
    case APIP_FIELD_NBLIST:
      for (int s = 0; s < a.max_nb; ++s)
        di[(size_t)i * a.max_nb + s] = s < a.nnb[i] ? (long long)a.nbl[(size_t)s * a.nmax + i] : -1;
      break;
    case APIP_FIELD_CSP:
      // row i: the partners of the atom whose id is i (the rows are kept by id)
      for (int s = 0; s < a.csp_nnb; ++s) di[(size_t)i * a.csp_nnb + s] = a.csp[(size_t)i * kCspCap + s];
      break;
    case APIP_FIELD_BUILD_POS:
      for (int q = 0; q < 3; ++q) dd[3 * i + q] = a.pos_ref[3 * i + q];
      break;
    default: break;
  }
}

inline int nblocks(int n, int b = kBlock) { return (n + b - 1) / b > 0 ? (n + b - 1) / b : 1; }

}  // namespace

// ---------------------------------------------------------------- launchers
template <typename T> void launch_prep(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_prep<T>, nblocks(a.n), kBlock, 0, s, a);
}

template <typename T> void launch_neighbors(const Args<T>& a, int ncell, cudaStream_t s) {
  (void)ncell;
  launch_pdl(k_bin<T>, nblocks(a.n), kBlock, 0, s, a);
  if (a.det) launch_pdl(k_cell_sort<T>, nblocks(a.ncell), kBlock, 0, s, a);
  launch_pdl(k_nbfill<T>, nblocks(a.n), kBlock, 0, s, a);
}

void launch_set_csp(const int32_t* src, int* dst, int n, int nnb, cudaStream_t s) {
  k_set_csp<<<nblocks(n), kBlock, 0, s>>>(src, dst, n, nnb);
}

void launch_csp_init(const Args<double>& a, cudaStream_t s) {
  k_csp_init<<<nblocks(a.n, 128), 128, 0, s>>>(a);
}

template <typename T> void launch_pass1(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_pass1<T>, nblocks(a.n), kBlock, 0, s, a);
}

// Force mixing: the precise model's forces on the atoms with lam > 0 need E^prec
// of every atom within the ACE cutoff of them; those with lam = 0 are appended
// to the compacted list after pass 2.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_fm_buffer(Args<T> a) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bool pred = false;
  if (i < a.n && a.lam[i] == T(0)) {
    const auto si = a.pv.self(i);
    const T rc2 = a.ace_rc * a.ace_rc;
    const int cnt = APIP_CHK(a.status, BND_LIST_LEN, a.nnb[i], a.max_nb + 1);
    const int* nb = a.nbl + i;
    for (int s = 0; s < cnt && !pred; ++s, nb += a.nmax) {
      const int j = APIP_CHK(a.status, BND_NEIGHBOUR, *nb, a.n);
      if (a.lam[j] > T(0)) {
        const auto d = a.pv.vec(si, j);
        pred = dot3(d, d) < rc2;
      }
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == 0 && mask) base = atomicAdd(&a.counts[0], __popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pred) a.ace_list[base + __popc(mask & ((1u << lane) - 1u))] = i;
}

void launch_ind_work(double* acc, double dt, int det, cudaStream_t s) {
  launch_pdl(k_ind_work, 1, 1, 0, s, acc, dt, det);
}

void launch_fix_finish(double* force, int n, cudaStream_t s) {
  launch_pdl(k_fix_finish, nblocks(3 * n), kBlock, 0, s, force, 3 * n);
}

template <typename T> void launch_fm_buffer(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_fm_buffer<T>, nblocks(a.n), kBlock, 0, s, a);
}

template <typename T> void launch_pass2(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_pass2<T>, nblocks(a.n), kBlock, 0, s, a);
  if (a.det) {
    launch_pdl(k_blk_scan, 1, 1024, 0, s, a.blk_cnt, nblocks(a.n));
    launch_pdl(k_compact_det<T>, nblocks(a.n), kBlock, 0, s, a);
  }
}

template <typename T> void launch_csp_force(const Args<T>& a, cudaStream_t s) {
  launch_pdl(k_csp_force<T>, nblocks(a.n), kBlock, 0, s, a);
}

void launch_final(double* partials, int n_part, double* e_total, double* e_pot_slot,
                  const double* thermo_part, int n_tblocks, double* thermo_slot, int* flags,
                  const int* counts, int64_t* n_ace_out, int* cell_count, int ncell, cudaStream_t s) {
  launch_pdl(k_final, 1, 256, 0, s, partials, n_part, e_total, e_pot_slot, thermo_part, n_tblocks, thermo_slot,
                            flags, counts, n_ace_out, cell_count, ncell);
}

void launch_thermo_final(const double* thermo_part, int n_tblocks, double* thermo_slot, cudaStream_t s) {
  launch_pdl(k_thermo_final, 1, 256, 0, s, thermo_part, n_tblocks, thermo_slot);
}

template <typename T> void launch_verlet(const Args<T>& a, int mode, double* pos, double* vel,
                                         const double* force, const double* inv_mass, double dt,
                                         double* thermo_part, cudaStream_t s) {
  const bool th = mode != 0 && thermo_part != nullptr;
  auto k = mode == 0 ? k_verlet<T, 0, false>
                     : (mode == 1 ? (th ? k_verlet<T, 1, true> : k_verlet<T, 1, false>)
                                  : (th ? k_verlet<T, 2, true> : k_verlet<T, 2, false>));
  launch_pdl(k, nblocks(a.n), kBlock, 0, s, a, pos, vel, force, inv_mass, dt, 0.5 * dt, thermo_part);
}

template <typename T> void launch_get_field(const Args<T>& a, int field, void* dst, cudaStream_t s) {
  k_get_field<T><<<nblocks(a.n), kBlock, 0, s>>>(a, field, dst);
}

#define APIP_INST(T)                                                                              \
  template void launch_prep<T>(const Args<T>&, cudaStream_t);                                     \
  template void launch_neighbors<T>(const Args<T>&, int, cudaStream_t);                           \
  template void launch_pass1<T>(const Args<T>&, cudaStream_t);                                    \
  template void launch_pass2<T>(const Args<T>&, cudaStream_t);                                    \
  template void launch_fm_buffer<T>(const Args<T>&, cudaStream_t);                                \
  template void launch_csp_force<T>(const Args<T>&, cudaStream_t);                                \
  template void launch_verlet<T>(const Args<T>&, int, double*, double*, const double*,            \
                                 const double*, double, double*, cudaStream_t);                   \
  template void launch_get_field<T>(const Args<T>&, int, void*, cudaStream_t);
APIP_INST(double)
APIP_INST(float)
#undef APIP_INST

}  // namespace apip
