// Host-side construction of the ACE tables: the canonical product basis, the
// real Gaunt coefficients and the coefficient-folded term lists that the GPU
// kernel evaluates.
//
// The paper takes ACE from the literature (Appendix B; Eq. S14).  Here the
// product basis B_b is the standard rotation-invariant coupling of the atomic
// density A_nlm through real Gaunt coefficients, and the two embedding
// channels phi_c = sum_b c_cb B_b are folded into one polynomial in A per
// channel:  phi_c = sum_t K_c[t] prod_q A[idx_q(t)],  with one term per
// distinct (sorted) index tuple.  A[nA] == 1 pads lower body orders so that
// orders 1..3 share one 3-index list and order 4 has a 4-index list.
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
#include <unordered_map>

#include "apip_internal.h"

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

struct Coef { double a = 0.0, b = 0.0; };

constexpr size_t kMaxTerms4 = size_t(1) << 22;

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

bool build_terms(int n_max, int l_max, int nu_max, const double* c1, const double* c2,
                 int64_t n_basis, HostTerms* out, std::string* err) {
  const int nlm = (l_max + 1) * (l_max + 1);
  const int nA = n_max * nlm;
  if (nA > 254) { *err = "n_max (l_max+1)^2 must be <= 254"; return false; }
  const auto basis = enumerate(n_max, l_max, nu_max);
  if ((int64_t)basis.size() != n_basis) {
    *err = "ace_n_basis does not match the canonical basis size " + std::to_string(basis.size());
    return false;
  }
  const int one = nA;
  auto aidx = [&](int n, int l, int m) { return (n - 1) * nlm + l * l + l + m; };
  // Gaunt cache for (l1, l2, l3) with m's.
  std::map<std::tuple<int, int, int, int, int, int>, double> gcache;
  auto G = [&](int l1, int m1, int l2, int m2, int l3, int m3) {
    auto key = std::make_tuple(l1, m1, l2, m2, l3, m3);
    auto it = gcache.find(key);
    if (it != gcache.end()) return it->second;
    const double v = real_gaunt(l1, m1, l2, m2, l3, m3);
    gcache.emplace(key, v);
    return v;
  };
  std::map<uint32_t, Coef> t3;
  std::unordered_map<uint32_t, Coef> t4;
  // nonzero G(l1 m1, l2 m2, L M) as (m1, m2, M, g), per (l1, l2, L)
  std::map<std::tuple<int, int, int>, std::vector<std::tuple<int, int, int, double>>> glist;
  auto GL = [&](int l1, int l2, int L) -> const std::vector<std::tuple<int, int, int, double>>& {
    auto key = std::make_tuple(l1, l2, L);
    auto it = glist.find(key);
    if (it != glist.end()) return it->second;
    std::vector<std::tuple<int, int, int, double>> v;
    for (int M = -L; M <= L; ++M)
      for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2) {
          const double g = G(l1, m1, l2, m2, L, M);
          if (g != 0.0) v.emplace_back(m1, m2, M, g);
        }
    return glist.emplace(key, std::move(v)).first->second;
  };
  auto add3 = [&](int a, int b, int c, double w, double ca, double cb) {
    int v[3] = {a, b, c};
    std::sort(v, v + 3);
    const uint32_t key = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16);
    Coef& k = t3[key];
    k.a += w * ca;
    k.b += w * cb;
  };
  auto add4 = [&](int a, int b, int c, int d, double w, double ca, double cb) {
    int v[4] = {a, b, c, d};
    std::sort(v, v + 4);
    const uint32_t key = (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16) | ((uint32_t)v[3] << 24);
    Coef& k = t4[key];
    k.a += w * ca;
    k.b += w * cb;
  };
  for (size_t bi = 0; bi < basis.size(); ++bi) {
    const Basis& b = basis[bi];
    const double ca = c1[bi], cb = c2[bi];
    if (b.nu == 1) {
      add3(aidx(b.n[0], 0, 0), one, one, 1.0, ca, cb);
    } else if (b.nu == 2) {
      const int l = b.l[0];
      for (int m = -l; m <= l; ++m) add3(aidx(b.n[0], l, m), aidx(b.n[1], l, m), one, 1.0, ca, cb);
    } else if (b.nu == 3) {
      const int l1 = b.l[0], l2 = b.l[1], l3 = b.l[2];
      for (int m1 = -l1; m1 <= l1; ++m1)
        for (int m2 = -l2; m2 <= l2; ++m2)
          for (int m3 = -l3; m3 <= l3; ++m3) {
            const double g = G(l1, m1, l2, m2, l3, m3);
            if (g != 0.0) add3(aidx(b.n[0], l1, m1), aidx(b.n[1], l2, m2), aidx(b.n[2], l3, m3), g, ca, cb);
          }
    } else {
      const int l1 = b.l[0], l2 = b.l[1], l3 = b.l[2], l4 = b.l[3], L = b.L;
      const auto& a12 = GL(l1, l2, L);
      const auto& a34 = GL(l3, l4, L);
      for (const auto& x : a12)
        for (const auto& y : a34) {
          if (std::get<2>(x) != std::get<2>(y)) continue;
          add4(aidx(b.n[0], l1, std::get<0>(x)), aidx(b.n[1], l2, std::get<1>(x)),
               aidx(b.n[2], l3, std::get<0>(y)), aidx(b.n[3], l4, std::get<1>(y)),
               std::get<3>(x) * std::get<3>(y), ca, cb);
        }
      if (t4.size() > kMaxTerms4) {
        *err = "nu_max = 4 expands to more than " + std::to_string(kMaxTerms4) +
               " product terms for this (n_max, l_max); not supported by the term-list kernel";
        return false;
      }
    }
  }
  out->key3.clear(); out->k3a.clear(); out->k3b.clear();
  out->key4.clear(); out->k4a.clear(); out->k4b.clear();
  for (const auto& kv : t3) {
    if (kv.second.a == 0.0 && kv.second.b == 0.0) continue;
    out->key3.push_back(kv.first);
    out->k3a.push_back(kv.second.a);
    out->k3b.push_back(kv.second.b);
  }
  std::vector<std::pair<uint32_t, Coef>> s4(t4.begin(), t4.end());
  std::sort(s4.begin(), s4.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  for (const auto& kv : s4) {
    if (kv.second.a == 0.0 && kv.second.b == 0.0) continue;
    out->key4.push_back(kv.first);
    out->k4a.push_back(kv.second.a);
    out->k4b.push_back(kv.second.b);
  }
  // Derivative entries: d phi_c / dA[tgt] = sum_e K_c[e] A[a] A[b] A[c] over the
  // entries e with target tgt, one per (term, position of tgt) and merged when the
  // remaining index triple coincides.  Key = tgt << 24 | a | b << 8 | c << 16 with
  // a <= b <= c (index nA = the constant 1), so the list is sorted by target.
  std::map<uint32_t, Coef> td;
  auto add_d = [&](int tgt, int a, int b, int c, const Coef& k) {
    if (tgt == one) return;
    int v[3] = {a, b, c};
    std::sort(v, v + 3);
    const uint32_t key = ((uint32_t)tgt << 24) | (uint32_t)v[0] | ((uint32_t)v[1] << 8) | ((uint32_t)v[2] << 16);
    Coef& e = td[key];
    e.a += k.a;
    e.b += k.b;
  };
  for (size_t q = 0; q < out->key3.size(); ++q) {
    const uint32_t k = out->key3[q];
    const int i0 = k & 255u, i1 = (k >> 8) & 255u, i2 = (k >> 16) & 255u;
    const Coef c{out->k3a[q], out->k3b[q]};
    add_d(i0, i1, i2, one, c);
    add_d(i1, i0, i2, one, c);
    add_d(i2, i0, i1, one, c);
  }
  for (size_t q = 0; q < out->key4.size(); ++q) {
    const uint32_t k = out->key4[q];
    const int i0 = k & 255u, i1 = (k >> 8) & 255u, i2 = (k >> 16) & 255u, i3 = k >> 24;
    const Coef c{out->k4a[q], out->k4b[q]};
    add_d(i0, i1, i2, i3, c);
    add_d(i1, i0, i2, i3, c);
    add_d(i2, i0, i1, i3, c);
    add_d(i3, i0, i1, i2, c);
  }
  // The entries, sorted by target (the map order), are cut into chunks of
  // kAceChunk that the kernel streams through shared memory.  Inside a chunk each
  // target forms one contiguous piece; pieces go to the kAceAdjWarps warps,
  // largest first to the least-loaded warp, so no two warps of a chunk write the
  // same omega component (a target split across chunks is summed chunk by chunk).
  out->keyd.clear(); out->kda.clear(); out->kdb.clear(); out->sched.clear();
  for (const auto& kv : td) {
    if (kv.second.a == 0.0 && kv.second.b == 0.0) continue;
    out->keyd.push_back(kv.first);
    out->kda.push_back(kv.second.a);
    out->kdb.push_back(kv.second.b);
  }
  const int ne = (int)out->keyd.size();
  const int nch = (ne + kAceChunk - 1) / kAceChunk;
  std::vector<int> choff(nch + 1), woff, triples;
  for (int c = 0; c <= nch; ++c) choff[c] = std::min(ne, c * kAceChunk);
  woff.push_back(0);
  for (int c = 0; c < nch; ++c) {
    std::vector<std::array<int, 3>> pieces;  // (target, rel start, rel end)
    for (int q = choff[c]; q < choff[c + 1];) {
      const int t = (int)(out->keyd[q] >> 24);
      int e = q;
      while (e < choff[c + 1] && (int)(out->keyd[e] >> 24) == t) ++e;
      pieces.push_back({t, q - choff[c], e - choff[c]});
      q = e;
    }
    std::stable_sort(pieces.begin(), pieces.end(),
                     [](const auto& x, const auto& y) { return x[2] - x[1] > y[2] - y[1]; });
    std::vector<std::vector<std::array<int, 3>>> bins(kAceAdjWarps);
    std::vector<int> load(kAceAdjWarps, 0);
    for (const auto& pc : pieces) {
      const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      bins[b].push_back(pc);
      load[b] += pc[2] - pc[1];
    }
    for (int b = 0; b < kAceAdjWarps; ++b) {
      for (const auto& pc : bins[b]) triples.insert(triples.end(), pc.begin(), pc.end());
      woff.push_back((int)(triples.size() / 3));
    }
  }
  out->sched.push_back(nch);
  out->sched.insert(out->sched.end(), choff.begin(), choff.end());
  out->sched.insert(out->sched.end(), woff.begin(), woff.end());
  out->sched.insert(out->sched.end(), triples.begin(), triples.end());
  return true;
}

}  // namespace apip
