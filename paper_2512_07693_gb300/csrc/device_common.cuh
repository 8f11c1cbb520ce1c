// Device helpers shared by the libapip kernels: the transition function,
// minimum-image pair vectors for both precisions, compensated sums and warp
// reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "apip_internal.h"

namespace apip {

template <typename T> struct V3 { T x, y, z; };

// Programmatic dependent launch.  The kernels of the force pipeline are launched
// so that the next kernel in the stream may be scheduled while this one finishes
// (launch_pdl).  Each calls pdl_begin() before its first memory access: it waits
// until the previous kernel has completed and its writes are visible, then lets
// its own dependent launch begin.  Waits end when the previous grid ends.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T dot3(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// f_trans(x, lo, hi) of Eq. S1 and its derivative: 1 below lo, 0 above hi,
// in between the quintic 1/2 + 15/16 t - 5/8 t^3 + 3/16 t^5 of
// t = (hi + lo - 2x)/(hi - lo).  It is evaluated in the factored forms
//   f = (1 + t)^3 (8 - 9t + 3t^2) / 16,   1 - f = (1 - t)^3 (8 + 9t + 3t^2) / 16,
//   df/dt = 15/16 (1 - t^2)^2,
// which keep full relative precision near both ends (in FP32 the expanded
// polynomial loses every digit of 1 - f close to x = lo).
template <typename T>
__device__ __forceinline__ T ftrans(T x, T lo, T hi, T inv_w, T* deriv) {
  if (x <= lo) { *deriv = T(0); return T(1); }
  if (x >= hi) { *deriv = T(0); return T(0); }
  const T t = (hi + lo - T(2) * x) * inv_w;
  const T u = T(1) - t * t;
  *deriv = T(0.9375) * u * u * (T(-2) * inv_w);
  const T p = T(1) + t;
  return T(0.0625) * p * p * p * (T(8) + t * (T(-9) + T(3) * t));
}

// 1 - f_trans(x, lo, hi) and d(1 - f_trans)/dx.
template <typename T>
__device__ __forceinline__ T ftrans_c(T x, T lo, T hi, T inv_w, T* deriv) {
  if (x <= lo) { *deriv = T(0); return T(0); }
  if (x >= hi) { *deriv = T(0); return T(1); }
  const T t = (hi + lo - T(2) * x) * inv_w;
  const T u = T(1) - t * t;
  *deriv = T(0.9375) * u * u * (T(2) * inv_w);
  const T q = T(1) - t;
  return T(0.0625) * q * q * q * (T(8) + t * (T(9) + T(3) * t));
}

// exp(x) for the EAM terms: in float32 the hardware exponential (__expf;
// relative error ~1e-6 for the |x| < 10 of the EAM arguments, far below the
// float32 path's tolerances), in float64 the correctly rounded exp.
template <typename T> __device__ __forceinline__ T fexp(T x);
template <> __device__ __forceinline__ float fexp<float>(float x) { return __expf(x); }
template <> __device__ __forceinline__ double fexp<double>(double x) { return exp(x); }

// Running sum with Kahan compensation in FP32; plain in FP64.
template <typename T> struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T v) {
    const T y = v - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ T value() const { return s; }
};
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// Plain running sum (the same interface as Acc).
template <typename T> struct Plain {
  T s = T(0);
  __device__ __forceinline__ void add(T v) { s += v; }
  __device__ __forceinline__ T value() const { return s; }
};

// r = |d| and 1/r from r^2: in float32 through the reciprocal square root
// (rsqrtf, within 2 ulp), in float64 by the correctly rounded square root and a
// division.
template <typename T> __device__ __forceinline__ void len_inv(T r2, T* r, T* ir);
template <> __device__ __forceinline__ void len_inv<float>(float r2, float* r, float* ir) {
  *ir = rsqrtf(r2);
  *r = r2 * *ir;
}
template <> __device__ __forceinline__ void len_inv<double>(double r2, double* r, double* ir) {
  *r = sqrt(r2);
  *ir = 1.0 / *r;
}

// Positions.  FP64 path: the caller's float64 array, minimum image with rint.
// FP32 path: each coordinate as a 32-bit fixed-point fraction of the box,
// q = floor(x_wrapped / L * 2^32).  The unsigned difference q_j - q_i read as a
// signed integer is the minimum-image separation in units of L / 2^32
// (3.3e-8 A for L = 143 A), exact; converting it to float rounds at the scale of
// the pair distance (~1e-7 A), where plain float coordinates would carry ~1e-5 A.
template <typename T> struct PosView;

template <> struct PosView<double> {
  const double* pos;
  double L[3], invL[3];
  struct Self { double x, y, z; };
  using Rec = Self;   // what a neighbour's separation needs (fetch, then vec_of)
  __device__ __forceinline__ Self self(int i) const { return {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]}; }
  __device__ __forceinline__ Rec fetch(int j) const { return self(j); }
  __device__ __forceinline__ V3<double> vec_of(const Self& s, const Rec& o) const {
    double dx = o.x - s.x, dy = o.y - s.y, dz = o.z - s.z;
    dx -= L[0] * rint(dx * invL[0]);
    dy -= L[1] * rint(dy * invL[1]);
    dz -= L[2] * rint(dz * invL[2]);
    return {dx, dy, dz};
  }
  __device__ __forceinline__ V3<double> vec(const Self& s, int j) const { return vec_of(s, fetch(j)); }
};

template <> struct PosView<float> {
  const uint4* q;
  float unit[3];                 // L / 2^32
  struct Self { uint4 q; };
  using Rec = uint4;
  __device__ __forceinline__ Self self(int i) const { return {q[i]}; }
  __device__ __forceinline__ Rec fetch(int j) const { return q[j]; }
  // the .w word of o is not read (pass 2 passes posg records, which carry g there)
  __device__ __forceinline__ V3<float> vec_of(const Self& s, const uint4& o) const {
    return {(float)(int)(o.x - s.q.x) * unit[0], (float)(int)(o.y - s.q.y) * unit[1],
            (float)(int)(o.z - s.q.z) * unit[2]};
  }
  __device__ __forceinline__ V3<float> vec(const Self& s, int j) const { return vec_of(s, q[j]); }
};

// The CSP^list vector r_ia + r_ib of atom i's partners a and b (Eq. B3).  FP32
// path: the two fixed-point separations are added as integers (exact; partners
// lie far closer than half the box) and converted once, so the nearly cancelling
// sum keeps the relative precision of its own length.
__device__ __forceinline__ V3<double> csp_vec(const PosView<double>& pv, const PosView<double>::Self& s, int ia,
                                              int ib) {
  const V3<double> u1 = pv.vec(s, ia), u2 = pv.vec(s, ib);
  return {u1.x + u2.x, u1.y + u2.y, u1.z + u2.z};
}
__device__ __forceinline__ V3<float> csp_vec(const PosView<float>& pv, const PosView<float>::Self& s, int ia,
                                             int ib) {
  const uint4 qa = pv.q[ia], qb = pv.q[ib];
  return {(float)(int)((qa.x - s.q.x) + (qb.x - s.q.x)) * pv.unit[0],
          (float)(int)((qa.y - s.q.y) + (qb.y - s.q.y)) * pv.unit[1],
          (float)(int)((qa.z - s.q.z) + (qb.z - s.q.z)) * pv.unit[2]};
}

// Fixed-point coordinate of a wrapped position w in [0, L): floor(w 2^32 / L)
// mod 2^32 (w = L, a rounding edge, maps to 0, its periodic image), in integer
// arithmetic.  With w = m 2^(e - 1086) (m the 53-bit significand left-aligned in
// 64 bits, e the biased exponent) and 2^32 / L = M 2^s (M left-aligned, s from the
// host), the exact product is m M 2^(e - 1086 + s): its floor is the high 64 bits
// of m M shifted right by 1022 - e - s, the low 64 bits adding less than one unit.
// This keeps the per-atom conversion off the float64 pipe, slow on this GPU.
__host__ __device__ __forceinline__ unsigned int fixed_coord(double w, unsigned long long M, int s) {
  unsigned long long b;
  memcpy(&b, &w, sizeof(b));
  const int e = (int)(b >> 52);   // w >= 0: no sign bit
  const int sh = 1022 - e - s;
  if (e == 0 || sh < 0 || sh >= 64) return 0u;
  const unsigned long long m = ((b & 0xfffffffffffffull) | 0x10000000000000ull) << 11;
#ifdef __CUDA_ARCH__
  const unsigned long long hi = __umul64hi(m, M);
#else
  const unsigned long long hi = (unsigned long long)(((unsigned __int128)m * M) >> 64);
#endif
  return (unsigned int)((hi >> sh) & 0xffffffffull);
}

// Float-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2): the
// error-free sum (Knuth's TwoSum) and product (an FMA gives the rounding error of
// a product exactly), written with the _rn intrinsics, which the compiler never
// contracts or reorders.
struct FF { float hi, lo; };
__device__ __forceinline__ FF ff_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bp = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp))};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = ff_sum(a.hi, b.hi);
  return ff_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF ff_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// The separation of two fixed-point coordinates in float-float: the exact
// integer difference d (split as d_h + d_l, d_h = d with its low 8 bits cleared,
// both exact in float) times the grid unit u = u_hi + u_lo.
__device__ __forceinline__ FF ff_coord(int d, float u_hi, float u_lo) {
  const int dh = d & ~0xff;
  const float h = (float)dh, l = (float)(d - dh);
  const FF p = ff_prod(h, u_hi);
  const float small = __fmaf_rn(h, u_lo, __fmaf_rn(l, u_hi, __fmul_rn(l, u_lo)));
  return ff_sum(p.hi, __fadd_rn(p.lo, small));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide float64 sum (result valid in thread 0); blockDim.x <= 1024.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Block-wide sum of a value of the path precision, returned in float64 (valid
// in thread 0): the warp-level part in T, the rest in float64 (float64 adds are
// slow on this GPU; 32 float32 terms round at ~1e-7 of their sum).
template <typename T>
__device__ __forceinline__ double block_sum_t(T v, double* sh) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = (double)v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double d = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) d = warp_sum(d);
  __syncthreads();
  return d;
}

// Block-wide sums of four float64 values (valid in thread 0, out[0..3]).  The
// first two exchange steps halve the values a lane carries (it keeps two of the
// four partial sums, then one), so a lane does 2 + 1 + 3 = 6 float64 adds
// instead of 4 x 5.  sh holds 4 x 32 doubles; blockDim.x <= 1024.
__device__ __forceinline__ void block_sum4(const double v[4], double* sh, double out[4]) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
  double k0 = b16 ? v[2] : v[0], k1 = b16 ? v[3] : v[1];
  k0 += __shfl_xor_sync(full, b16 ? v[0] : v[2], 16);
  k1 += __shfl_xor_sync(full, b16 ? v[1] : v[3], 16);
  double k = b8 ? k1 : k0;
  k += __shfl_xor_sync(full, b8 ? k0 : k1, 8);
  k += __shfl_xor_sync(full, k, 4);
  k += __shfl_xor_sync(full, k, 2);
  k += __shfl_xor_sync(full, k, 1);
  // lane 8 q' holds the warp sum of value q = 2 (lane >> 4) + ((lane >> 3) & 1)
  if ((lane & 7) == 0) sh[((b16 ? 2 : 0) + (b8 ? 1 : 0)) * 32 + w] = k;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double d = lane < nw ? sh[q * 32 + lane] : 0.0;
      d = warp_sum(d);
      if (lane == 0) out[q] = d;
    }
  }
  __syncthreads();
}

}  // namespace apip
