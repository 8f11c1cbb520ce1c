// Host-side construction of the ACE tables: the canonical product basis, the
// real Gaunt coefficients and the coupled tables that the GPU kernel evaluates.
//
// The paper takes ACE from the literature (Appendix B; Eq. S14).  Here the
// product basis B_b is the standard rotation-invariant coupling of the atomic
// density A_nlm through real Gaunt coefficients, and the embedding channels are
// phi_c = sum_b c_cb B_b.  The kernel evaluates every B_b as one dot product of
// two segments of a per-atom pool of A and of pairwise Gaunt couplings of A
// (build_coupled below).
//
// Real Gaunt coefficients are built from complex ones (Wigner 3j by Racah's
// formula) through the unitary map from complex to real spherical harmonics:
//   Y_{l,m>0} = ((-1)^m Y_l^m + Y_l^{-m}) / sqrt2,
//   Y_{l,-m}  = ((-1)^m Y_l^m - Y_l^{-m}) / (i sqrt2),   Y_{l,0} = Y_l^0,
// which matches the real harmonics of the kernels (no Condon-Shortley phase
// in the real functions).
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <map>
#include <tuple>

#include "apip_internal.h"
#include "gaunt_layout.h"

namespace apip {
namespace {

double fact(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3) by Racah's formula.
double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  if (j3 < std::abs(j1 - j2) || j3 > j1 + j2) return 0.0;
  if (std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m3) > j3) return 0.0;
  const double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
  const double pre = std::sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                               fact(j3 + m3) * fact(j3 - m3));
  double s = 0.0;
  for (int k = 0; k <= j1 + j2 + j3; ++k) {
    const int a = j3 - j2 + k + m1, b = j3 - j1 + k - m2, c = j1 + j2 - j3 - k;
    const int d = j1 - k - m1, e = j2 - k + m2;
    if (a < 0 || b < 0 || c < 0 || d < 0 || e < 0) continue;
    const double term = 1.0 / (fact(k) * fact(a) * fact(b) * fact(c) * fact(d) * fact(e));
    s += (k % 2 ? -term : term);
  }
  const int ph = j1 - j2 - m3;
  return ((ph % 2 + 2) % 2 ? -1.0 : 1.0) * pre * s;
}

// int Y_l1^m1 Y_l2^m2 Y_l3^m3 dOmega for complex harmonics with Condon-Shortley phase.
double complex_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
  if (m1 + m2 + m3 != 0) return 0.0;
  return std::sqrt((2 * l1 + 1) * (2 * l2 + 1) * (2 * l3 + 1) / (4.0 * M_PI)) *
         wigner3j(l1, l2, l3, 0, 0, 0) * wigner3j(l1, l2, l3, m1, m2, m3);
}

// Coefficients of real Y_{l,m} on complex Y_l^{mc}: returns (count, mc[2], u[2]).
int real_to_complex(int m, int mc[2], std::complex<double> u[2]) {
  const double s2 = 1.0 / std::sqrt(2.0);
  if (m == 0) { mc[0] = 0; u[0] = 1.0; return 1; }
  const int mu = std::abs(m);
  const double sg = (mu % 2) ? -1.0 : 1.0;
  mc[0] = mu; mc[1] = -mu;
  if (m > 0) { u[0] = sg * s2; u[1] = s2; }
  else { u[0] = std::complex<double>(0.0, -sg * s2); u[1] = std::complex<double>(0.0, s2); }
  return 2;
}

struct Basis { int nu; int n[4]; int l[4]; int L; };

std::vector<Basis> enumerate(int n_max, int l_max, int nu_max) {
  std::vector<std::pair<int, int>> P;  // (n, l) ordered by p = (n-1)(l_max+1) + l
  for (int n = 1; n <= n_max; ++n)
    for (int l = 0; l <= l_max; ++l) P.push_back({n, l});
  const int np = (int)P.size();
  std::vector<Basis> out;
  if (nu_max >= 1)
    for (int n = 1; n <= n_max; ++n) out.push_back({1, {n, 0, 0, 0}, {0, 0, 0, 0}, -1});
  if (nu_max >= 2)
    for (int a = 0; a < np; ++a)
      for (int b = a; b < np; ++b)
        if (P[a].second == P[b].second)
          out.push_back({2, {P[a].first, P[b].first, 0, 0}, {P[a].second, P[b].second, 0, 0}, -1});
  if (nu_max >= 3)
    for (int a = 0; a < np; ++a)
      for (int b = a; b < np; ++b)
        for (int c = b; c < np; ++c) {
          const int l1 = P[a].second, l2 = P[b].second, l3 = P[c].second;
          if ((l1 + l2 + l3) % 2 == 0 && l3 >= std::abs(l1 - l2) && l3 <= l1 + l2)
            out.push_back({3, {P[a].first, P[b].first, P[c].first, 0}, {l1, l2, l3, 0}, -1});
        }
  if (nu_max >= 4)
    for (int a = 0; a < np; ++a)
      for (int b = a; b < np; ++b)
        for (int c = b; c < np; ++c)
          for (int d = c; d < np; ++d) {
            const int l1 = P[a].second, l2 = P[b].second, l3 = P[c].second, l4 = P[d].second;
            const int lo = std::max(std::abs(l1 - l2), std::abs(l3 - l4));
            const int hi = std::min(l1 + l2, l3 + l4);
            for (int L = lo; L <= hi; ++L)
              if ((l1 + l2 + L) % 2 == 0 && (l3 + l4 + L) % 2 == 0)
                out.push_back({4, {P[a].first, P[b].first, P[c].first, P[d].first}, {l1, l2, l3, l4}, L});
          }
  return out;
}

}  // namespace

double real_gaunt(int l1, int m1, int l2, int m2, int l3, int m3) {
  int c1[2], c2[2], c3[2];
  std::complex<double> u1[2], u2[2], u3[2];
  const int k1 = real_to_complex(m1, c1, u1), k2 = real_to_complex(m2, c2, u2),
            k3 = real_to_complex(m3, c3, u3);
  std::complex<double> s = 0.0;
  for (int a = 0; a < k1; ++a)
    for (int b = 0; b < k2; ++b)
      for (int c = 0; c < k3; ++c)
        if (c1[a] + c2[b] + c3[c] == 0)
          s += u1[a] * u2[b] * u3[c] * complex_gaunt(l1, c1[a], l2, c2[b], l3, c3[c]);
  const double v = s.real();
  return std::fabs(v) < 1e-15 ? 0.0 : v;
}

void ylm_norms(int l_max, double* out) {
  for (int l = 0; l <= l_max; ++l)
    for (int m = -l; m <= l; ++m) {
      const int am = std::abs(m);
      double nrm = std::sqrt((2 * l + 1) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
      if (m != 0) nrm *= std::sqrt(2.0);
      out[l * l + l + m] = nrm;
    }
}

int64_t basis_size(int n_max, int l_max, int nu_max) {
  if (n_max < 1 || n_max > kNmaxCap || l_max < 0 || l_max > kLmaxCap || nu_max < 1 || nu_max > 4)
    return -1;
  return (int64_t)enumerate(n_max, l_max, nu_max).size();
}

// The coupled evaluation.  Every basis function is one dot product of two
// segments of a per-atom pool X = [1 | A | C]:
//   nu = 1:  A_{n00} . 1
//   nu = 2:  A_{p1} . A_{p2}                      (l1 = l2, length 2l + 1)
//   nu = 3:  C_{(p1 p2) l3} . A_{p3}              (length 2 l3 + 1)
//   nu = 4:  C_{(p1 p2) L} . C_{(p3 p4) L}        (length 2L + 1)
// with A_p = (A_{n l m})_{m=-l..l} for p = (n, l) and the couplings
//   C_{(p1 p2) L M} = sum_{m1 m2} G(l1 m1, l2 m2, L M) A_{p1 m1} A_{p2 m2}.
// This is the same polynomial as the basis definition (the Gaunt sums are only
// grouped differently), and the reverse pass follows the same structure:
//   dE/dX_s = sum over the records touching segment s of k_b X_partner,
//   k_b = c1_b + F'(phi_2) c2_b (a record with both sides on s counts twice),
// then dE/dC is pushed back onto A through the Gaunt entries.
bool build_coupled(int n_max, int l_max, int nu_max, const double* c1, const double* c2, int64_t n_basis,
                   HostAce* out, std::string* err) {
  const int nlm = (l_max + 1) * (l_max + 1);
  const int nA = n_max * nlm;
  const auto basis = enumerate(n_max, l_max, nu_max);
  if ((int64_t)basis.size() != n_basis) {
    *err = "ace_n_basis does not match the canonical basis size " + std::to_string(basis.size());
    return false;
  }
  // pool offset of A_{n l m = -l}
  auto aoff = [&](int n, int l) { return 1 + (n - 1) * nlm + l * l; };
  struct Coupling { int n1, l1, n2, l2, L, off; };
  std::vector<Coupling> coup;
  std::map<std::tuple<int, int, int, int, int>, int> cidx;
  int next = 1 + nA;
  auto coupling = [&](int n1, int l1, int n2, int l2, int L) {
    const auto key = std::make_tuple(n1, l1, n2, l2, L);
    auto it = cidx.find(key);
    if (it != cidx.end()) return coup[it->second].off;
    cidx.emplace(key, (int)coup.size());
    coup.push_back({n1, l1, n2, l2, L, next});
    next += 2 * L + 1;
    return coup.back().off;
  };
  struct F { int o1, o2, len; double a, b; };
  std::vector<F> recs;
  recs.reserve(basis.size());
  for (size_t bi = 0; bi < basis.size(); ++bi) {
    const Basis& b = basis[bi];
    F r{0, 0, 0, c1[bi], c2[bi]};
    if (b.nu == 1) {
      r.o1 = aoff(b.n[0], 0); r.o2 = 0; r.len = 1;
    } else if (b.nu == 2) {
      r.o1 = aoff(b.n[0], b.l[0]); r.o2 = aoff(b.n[1], b.l[1]); r.len = 2 * b.l[0] + 1;
    } else if (b.nu == 3) {
      r.o1 = coupling(b.n[0], b.l[0], b.n[1], b.l[1], b.l[2]);
      r.o2 = aoff(b.n[2], b.l[2]);
      r.len = 2 * b.l[2] + 1;
    } else {
      r.o1 = coupling(b.n[0], b.l[0], b.n[1], b.l[1], b.L);
      r.o2 = coupling(b.n[2], b.l[2], b.n[3], b.l[3], b.L);
      r.len = 2 * b.L + 1;
    }
    recs.push_back(r);
  }
  const int npool = next;
  if (npool > 65535) { *err = "ACE pool of " + std::to_string(npool) + " values exceeds 65535"; return false; }
  out->nA = nA;
  out->nC = npool - 1 - nA;
  out->npool = npool;

  // Gaunt entries per (l1, l2, L, M), shared by all couplings of those degrees
  std::map<std::tuple<int, int, int, int>, std::pair<int, int>> glist;
  out->gkey.clear(); out->gval.clear(); out->comp.clear();
  auto gaunt_list = [&](int l1, int l2, int L, int M) {
    const auto key = std::make_tuple(l1, l2, L, M);
    auto it = glist.find(key);
    if (it != glist.end()) return it->second;
    const int beg = (int)out->gval.size();
    for (int m1 = -l1; m1 <= l1; ++m1)
      for (int m2 = -l2; m2 <= l2; ++m2) {
        const double g = real_gaunt(l1, m1, l2, m2, L, M);
        if (g == 0.0) continue;
        out->gkey.push_back((uint32_t)(m1 + l1) | ((uint32_t)(m2 + l2) << 8));
        out->gval.push_back(g);
      }
    const std::pair<int, int> v{beg, (int)out->gval.size() - beg};
    glist.emplace(key, v);
    return v;
  };
  // one entry per C component, in pool order
  std::vector<std::array<int, 4>> comps;   // (a1, a2, gofs, gcnt)
  for (const Coupling& u : coup)
    for (int M = -u.L; M <= u.L; ++M) {
      const auto gl = gaunt_list(u.l1, u.l2, u.L, M);
      comps.push_back({aoff(u.n1, u.l1), aoff(u.n2, u.l2), gl.first, gl.second});
      out->comp.push_back((uint32_t)aoff(u.n1, u.l1) | ((uint32_t)aoff(u.n2, u.l2) << 16));
      out->comp.push_back(((uint32_t)gl.first << 8) | (uint32_t)gl.second);
    }
  if (out->gval.size() >= (size_t(1) << 24)) { *err = "too many Gaunt entries"; return false; }

  // forward records, grouped by length so that the lanes of a warp run the same loop
  std::vector<F> fw(recs);
  std::stable_sort(fw.begin(), fw.end(), [](const F& x, const F& y) {
    return std::make_tuple(x.len, x.o1, x.o2) < std::make_tuple(y.len, y.o1, y.o2);
  });
  out->fkey.clear(); out->flen.clear(); out->f1.clear(); out->f2.clear();
  for (const F& r : fw) {
    out->fkey.push_back((uint32_t)r.o1 | ((uint32_t)r.o2 << 16));
    out->flen.push_back((uint32_t)r.len);
    out->f1.push_back(r.a);
    out->f2.push_back(r.b);
  }

  // reverse rows per segment (segment = A_p or C_u; the constant has none)
  std::vector<int> seg_of(npool, -1), seg_start(npool, 0);
  for (int n = 1; n <= n_max; ++n)
    for (int l = 0; l <= l_max; ++l)
      for (int m = 0; m < 2 * l + 1; ++m) { seg_of[aoff(n, l) + m] = aoff(n, l); seg_start[aoff(n, l) + m] = aoff(n, l); }
  for (const Coupling& u : coup)
    for (int m = 0; m < 2 * u.L + 1; ++m) { seg_of[u.off + m] = u.off; seg_start[u.off + m] = u.off; }
  std::map<int, std::vector<std::array<double, 3>>> rows;   // segment -> (partner, c1, c2)
  for (const F& r : recs) {
    if (r.o1 == r.o2) {
      rows[r.o1].push_back({(double)r.o2, 2.0 * r.a, 2.0 * r.b});
    } else {
      if (r.o1 != 0) rows[r.o1].push_back({(double)r.o2, r.a, r.b});
      if (r.o2 != 0) rows[r.o2].push_back({(double)r.o1, r.a, r.b});
    }
  }
  std::map<int, std::pair<int, int>> row_range;
  out->rkey.clear(); out->r1.clear(); out->r2.clear();
  for (const auto& kv : rows) {
    const int beg = (int)out->rkey.size();
    for (const auto& e : kv.second) {
      out->rkey.push_back((uint32_t)e[0]);
      out->r1.push_back(e[1]);
      out->r2.push_back(e[2]);
    }
    row_range[kv.first] = {beg, (int)out->rkey.size()};
  }
  out->qrow.assign((size_t)4 * npool, 0);
  for (int q = 1; q < npool; ++q) {
    const auto it = row_range.find(seg_of[q]);
    if (it != row_range.end()) {
      out->qrow[4 * q] = it->second.first;
      out->qrow[4 * q + 1] = it->second.second;
    }
    out->qrow[4 * q + 2] = q - seg_start[q];
  }

  // C -> A entries, grouped by target A component (pool index - 1), cut into
  // pieces; the partial sums of the pieces are kept in the C part of the pool,
  // so there may be at most nC pieces
  std::vector<std::vector<std::pair<uint32_t, double>>> tgt(nA);
  for (int c = 0; c < out->nC; ++c) {
    const int qc = 1 + nA + c;
    const auto& cp = comps[c];
    for (int e = cp[2]; e < cp[2] + cp[3]; ++e) {
      const int i = out->gkey[e] & 255u, j = out->gkey[e] >> 8;
      const double g = out->gval[e];
      tgt[cp[0] + i - 1].push_back({(uint32_t)qc | ((uint32_t)(cp[1] + j) << 16), g});
      tgt[cp[1] + j - 1].push_back({(uint32_t)qc | ((uint32_t)(cp[0] + i) << 16), g});
    }
  }
  out->bkey.clear(); out->bval.clear(); out->poff.clear(); out->tpiece.clear();
  for (const auto& v : tgt)
    for (const auto& e : v) { out->bkey.push_back(e.first); out->bval.push_back(e.second); }
  // piece length: a target's entries are cut into ceil(cnt / len) nearly equal
  // pieces; the length minimises the step's critical path, (rounds of
  // kAceThreads pieces) x (len + a per-piece overhead of 8 entries) plus the
  // pieces a target sums afterwards, with at most nC pieces
  auto cut = [&](int len, bool emit) {
    int np = 0, pos = 0;
    if (emit) { out->poff.assign(1, 0); out->tpiece.assign(1, 0); }
    for (int t = 0; t < nA; ++t) {
      const int cnt = (int)tgt[t].size();
      const int k = (cnt + len - 1) / len;
      for (int q = 1; q <= k; ++q)
        if (emit) out->poff.push_back(pos + (int)((int64_t)cnt * q / k));
      np += k;
      pos += cnt;
      if (emit) out->tpiece.push_back((int)out->poff.size() - 1);
    }
    return np;
  };
  int best_len = 0;
  int64_t best_cost = -1;
  for (int len = 1; len <= std::max<int>(1, (int)out->bkey.size()); len = len < 64 ? len + 1 : len + len / 8) {
    const int np = cut(len, false);
    if (np > std::max(out->nC, 0)) continue;
    const int64_t cost = (int64_t)((np + kAceThreads - 1) / kAceThreads) * (len + 8) + (np + nA - 1) / nA;
    if (best_cost < 0 || cost < best_cost) { best_cost = cost; best_len = len; }
  }
  cut(std::max(best_len, 1), true);
  return true;
}

void gaunt_fill(double* out) {
  for (int l1 = 0; l1 <= kGauntLmax; ++l1)
    for (int l2 = l1; l2 <= kGauntLmax; ++l2)
      for (int L = 0; L <= kGauntLmax; ++L) {
        if (!gaunt_type_valid(l1, l2, L)) continue;
        int e = gaunt_offset(l1, l2, L);
        for (int m1 = -l1; m1 <= l1; ++m1)
          for (int m2 = -l2; m2 <= l2; ++m2)
            for (int v = 0; v < 2; ++v) {
              const int M = gaunt_cand(m1, m2, v, L);
              if (M != kNoM) out[e++] = real_gaunt(l1, m1, l2, m2, L, M);
            }
      }
}

// Streamed tables (body order <= 3): couplings C_{(p1 p2) L} with l1 <= l2 (the
// factors swapped where needed; C is symmetric in them), sorted by type so that
// neighbouring thread slices run the same unrolled code, each with its list of
// nu = 3 partners (p3, c1, c2); nu = 1, 2 functions as dot products of A segments.
bool build_streamed(int n_max, int l_max, int nu_max, const double* c1, const double* c2, int64_t n_basis,
                    HostStream* out, std::string* err) {
  if (nu_max > 3) { *err = "the streamed ACE evaluation covers body order <= 3"; return false; }
  const int nlm = (l_max + 1) * (l_max + 1);
  const auto basis = enumerate(n_max, l_max, nu_max);
  if ((int64_t)basis.size() != n_basis) {
    *err = "ace_n_basis does not match the canonical basis size " + std::to_string(basis.size());
    return false;
  }
  auto abase = [&](int n, int l) { return (n - 1) * nlm + l * l; };   // A index of m = -l
  struct Cp { int a1, a2, l1, l2, L; std::vector<std::array<double, 3>> part; };
  std::map<std::tuple<int, int, int>, int> index;
  std::vector<Cp> cps;
  *out = HostStream{};
  for (size_t bi = 0; bi < basis.size(); ++bi) {
    const Basis& b = basis[bi];
    if (b.nu == 1) {
      out->pkey.push_back((uint32_t)abase(b.n[0], 0) | (0xffffu << 16));
      out->plen.push_back(1);
      out->p1.push_back(c1[bi]);
      out->p2.push_back(c2[bi]);
    } else if (b.nu == 2) {
      out->pkey.push_back((uint32_t)abase(b.n[0], b.l[0]) | ((uint32_t)abase(b.n[1], b.l[1]) << 16));
      out->plen.push_back((uint32_t)(2 * b.l[0] + 1));
      out->p1.push_back(c1[bi]);
      out->p2.push_back(c2[bi]);
    } else {
      int a1 = abase(b.n[0], b.l[0]), a2 = abase(b.n[1], b.l[1]), l1 = b.l[0], l2 = b.l[1];
      if (l1 > l2) { std::swap(a1, a2); std::swap(l1, l2); }
      const auto key = std::make_tuple(a1, a2, b.l[2]);
      auto it = index.find(key);
      if (it == index.end()) {
        it = index.emplace(key, (int)cps.size()).first;
        cps.push_back({a1, a2, l1, l2, b.l[2], {}});
      }
      cps[it->second].part.push_back({(double)abase(b.n[2], b.l[2]), c1[bi], c2[bi]});
    }
  }
  std::stable_sort(cps.begin(), cps.end(), [](const Cp& x, const Cp& y) {
    return std::make_tuple(gaunt_type(x.l1, x.l2, x.L), -(int)x.part.size(), x.a1, x.a2) <
           std::make_tuple(gaunt_type(y.l1, y.l2, y.L), -(int)y.part.size(), y.a1, y.a2);
  });
  for (const Cp& c : cps) {
    if (!gaunt_type_valid(c.l1, c.l2, c.L)) { *err = "internal: invalid coupling type"; return false; }
    const uint32_t beg = (uint32_t)out->tkey.size();
    for (const auto& p : c.part) {
      out->tkey.push_back((uint32_t)p[0]);
      out->t1.push_back(p[1]);
      out->t2.push_back(p[2]);
    }
    out->cpl.push_back((uint32_t)c.a1 | ((uint32_t)c.a2 << 8) | ((uint32_t)gaunt_type(c.l1, c.l2, c.L) << 16));
    out->cpl.push_back(beg);
    out->cpl.push_back((uint32_t)out->tkey.size());
    out->cpl.push_back(0u);
    out->gaunt_products += gaunt_count(c.l1, c.l2, c.L);
  }
  return true;
}

// Host check of every key and range of the tables against the arrays they
// index, run by apip_create after building them (in every build): each segment a
// record, coupling, partner, Gaunt, reverse-row or C -> A entry names lies inside
// A (or the pool) and each range inside its entry array.  The device's
// bounds-checked build tests the streamed tables again as it reads them.
bool validate_streamed(const HostStream& h, int nA, std::string* err) {
  auto bad = [&](const std::string& what) { *err = "internal: ACE table check failed: " + what; return false; };
  for (size_t r = 0; r < h.pkey.size(); ++r) {
    const int a1 = (int)(h.pkey[r] & 0xffffu), a2 = (int)(h.pkey[r] >> 16), len = (int)h.plen[r];
    if (len < 1 || a1 + len > nA) return bad("nu <= 2 record " + std::to_string(r));
    if ((uint32_t)a2 != 0xffffu && a2 + len > nA) return bad("nu = 2 record " + std::to_string(r));
  }
  if (h.cpl.size() % 4) return bad("coupling array length");
  for (size_t u = 0; u < h.cpl.size() / 4; ++u) {
    const uint32_t w = h.cpl[4 * u];
    const int a1 = (int)(w & 255u), a2 = (int)((w >> 8) & 255u), type = (int)(w >> 16);
    const int l1 = type / 25, l2 = (type / 5) % 5, L = type % 5;
    if (type >= 125 || !gaunt_type_valid(l1, l2, L)) return bad("coupling type " + std::to_string(u));
    if (a1 + 2 * l1 + 1 > nA || a2 + 2 * l2 + 1 > nA) return bad("coupling operands " + std::to_string(u));
    const uint32_t pb = h.cpl[4 * u + 1], pe = h.cpl[4 * u + 2];
    if (!(pb < pe) || pe > h.tkey.size()) return bad("coupling partner range " + std::to_string(u));
    for (uint32_t q = pb; q < pe; ++q)
      if ((int)h.tkey[q] + 2 * L + 1 > nA) return bad("partner " + std::to_string(q));
  }
  return true;
}

bool validate_coupled(const HostAce& h, std::string* err) {
  auto bad = [&](const std::string& what) { *err = "internal: ACE table check failed: " + what; return false; };
  const int nA = h.nA, npool = h.npool;
  if (npool != 1 + nA + h.nC || h.comp.size() != (size_t)2 * h.nC) return bad("pool sizes");
  for (int c = 0; c < h.nC; ++c) {
    const int a1 = (int)(h.comp[2 * c] & 0xffffu), a2 = (int)(h.comp[2 * c] >> 16);
    const int gofs = (int)(h.comp[2 * c + 1] >> 8), gcnt = (int)(h.comp[2 * c + 1] & 255u);
    if (a1 < 1 || a2 < 1 || gofs + gcnt > (int)h.gkey.size()) return bad("C component " + std::to_string(c));
    for (int e = gofs; e < gofs + gcnt; ++e)
      if (a1 + (int)(h.gkey[e] & 255u) > nA || a2 + (int)(h.gkey[e] >> 8) > nA)
        return bad("Gaunt entry " + std::to_string(e));
  }
  for (size_t r = 0; r < h.fkey.size(); ++r) {
    const int o1 = (int)(h.fkey[r] & 0xffffu), o2 = (int)(h.fkey[r] >> 16), len = (int)h.flen[r];
    if (len < 1 || o1 + len > npool || o2 + len > npool) return bad("record " + std::to_string(r));
  }
  if (h.qrow.size() != (size_t)4 * npool) return bad("reverse row table length");
  for (int q = 1; q < npool; ++q) {
    const int b = h.qrow[4 * q], e = h.qrow[4 * q + 1], m = h.qrow[4 * q + 2];
    if (b < 0 || b > e || e > (int)h.rkey.size() || m < 0 || m > q) return bad("reverse row " + std::to_string(q));
    for (int k = b; k < e; ++k)
      if ((int)h.rkey[k] + m >= npool) return bad("reverse entry " + std::to_string(k));
  }
  for (size_t k = 0; k < h.bkey.size(); ++k) {
    const int qc = (int)(h.bkey[k] & 0xffffu), qa = (int)(h.bkey[k] >> 16);
    if (qc < 1 + nA || qc >= npool || qa < 1 || qa > nA) return bad("C -> A entry " + std::to_string(k));
  }
  if (h.poff.empty() || h.poff[0] != 0 || h.poff.back() != (int)h.bkey.size()) return bad("piece offsets");
  for (size_t k = 1; k < h.poff.size(); ++k)
    if (h.poff[k] < h.poff[k - 1]) return bad("piece offsets");
  const int npc = (int)h.poff.size() - 1;
  if (npc > h.nC || h.tpiece.size() != (size_t)nA + 1) return bad("pieces per target");
  for (size_t k = 0; k < h.tpiece.size(); ++k)
    if (h.tpiece[k] < 0 || h.tpiece[k] > npc || (k && h.tpiece[k] < h.tpiece[k - 1])) return bad("pieces per target");
  return true;
}

}  // namespace apip
