// Canonical layout of the real Gaunt coefficients G(l1 m1, l2 m2, L M) used by
// the streamed ACE kernel (body order <= 3, so l1, l2, L <= 4), shared by the
// host code that fills the table and the device code that reads it at
// compile-time offsets.
//
// For real harmonics (cos(m phi) for m >= 0, sin(|m| phi) for m < 0 in the phi
// factor) the azimuthal integral of a product of three vanishes unless
// |M| = |m1| + |m2| or ||m1| - |m2||, with an even number of negative m among
// (m1, m2, M).  These candidates (a superset of the nonzero coefficients; the
// polar integral can still vanish) are enumerated in the order m1, m2, then
// |M| = |m1| + |m2| before ||m1| - |m2||; the table holds one value per
// candidate, for every coupling type (l1 <= l2, L) in the order of
// APIP_GAUNT_TYPES.
#pragma once

#include <cuda_runtime.h>

namespace apip {

constexpr int kGauntLmax = 4;
constexpr int kNoM = 1000;

__host__ __device__ constexpr int iabs_c(int x) { return x < 0 ? -x : x; }

// M of candidate v (0 or 1) of (m1, m2) for coupling degree L, or kNoM.
__host__ __device__ constexpr int gaunt_cand(int m1, int m2, int v, int L) {
  const int a = iabs_c(m1), b = iabs_c(m2);
  const bool neg = ((m1 < 0 ? 1 : 0) + (m2 < 0 ? 1 : 0)) == 1;
  const int mag = v == 0 ? a + b : iabs_c(a - b);
  if (v == 1 && mag == a + b) return kNoM;
  if (mag > L) return kNoM;
  if (neg && mag == 0) return kNoM;
  return neg ? -mag : mag;
}

__host__ __device__ constexpr bool gaunt_type_valid(int l1, int l2, int L) {
  return l1 <= l2 && L >= l2 - l1 && L <= l1 + l2 && (l1 + l2 + L) % 2 == 0;
}

__host__ __device__ constexpr int gaunt_count(int l1, int l2, int L) {
  int n = 0;
  for (int m1 = -l1; m1 <= l1; ++m1)
    for (int m2 = -l2; m2 <= l2; ++m2)
      for (int v = 0; v < 2; ++v)
        if (gaunt_cand(m1, m2, v, L) != kNoM) ++n;
  return n;
}

// Offset of type (l1, l2, L) in the table; past the last type, the table size.
__host__ __device__ constexpr int gaunt_offset(int l1, int l2, int L) {
  int off = 0;
  for (int x = 0; x <= kGauntLmax; ++x)
    for (int y = x; y <= kGauntLmax; ++y)
      for (int z = 0; z <= kGauntLmax; ++z) {
        if (x == l1 && y == l2 && z == L) return off;
        if (gaunt_type_valid(x, y, z)) off += gaunt_count(x, y, z);
      }
  return off;
}

constexpr int kGauntTotal = gaunt_offset(kGauntLmax + 1, 0, 0);

// type code of a coupling (l1 <= l2)
__host__ __device__ constexpr int gaunt_type(int l1, int l2, int L) { return (l1 * 5 + l2) * 5 + L; }

// every valid (l1 <= l2 <= 4, L <= 4)
#define APIP_GAUNT_TYPES                                                                                   \
  X(0, 0, 0) X(0, 1, 1) X(0, 2, 2) X(0, 3, 3) X(0, 4, 4) X(1, 1, 0) X(1, 1, 2) X(1, 2, 1) X(1, 2, 3)          \
  X(1, 3, 2) X(1, 3, 4) X(1, 4, 3) X(2, 2, 0) X(2, 2, 2) X(2, 2, 4) X(2, 3, 1) X(2, 3, 3) X(2, 4, 2)          \
  X(2, 4, 4) X(3, 3, 0) X(3, 3, 2) X(3, 3, 4) X(3, 4, 1) X(3, 4, 3) X(4, 4, 0) X(4, 4, 2) X(4, 4, 4)

}  // namespace apip
