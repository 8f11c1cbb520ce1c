// Host harness of the ACE table check (compiled and run by
// test_ace_table_check.py; no device code runs): builds the tables of a few bases,
// checks that they pass, then corrupts one entry of each kind and checks that the
// check rejects it.  Prints one line per case: "<name> ok" or "<name> FAIL".
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "apip_internal.h"

using namespace apip;

static void report(const char* name, bool pass) { std::printf("%s %s\n", name, pass ? "ok" : "FAIL"); }

int main() {
  const int streamed[][3] = {{6, 3, 3}, {4, 2, 3}, {3, 3, 2}, {2, 1, 1}, {1, 0, 1}};
  const int pooled[][3] = {{4, 3, 4}, {8, 4, 4}, {2, 4, 4}};
  std::string err;
  for (const auto& c : streamed) {
    const int64_t nb = basis_size(c[0], c[1], c[2]);
    const int nA = c[0] * (c[1] + 1) * (c[1] + 1);
    std::vector<double> c1(nb, 0.1), c2(nb, 0.2);
    HostStream h;
    const bool built = build_streamed(c[0], c[1], c[2], c1.data(), c2.data(), nb, &h, &err);
    report(("streamed_valid_" + std::to_string(c[0]) + std::to_string(c[1]) + std::to_string(c[2])).c_str(),
           built && validate_streamed(h, nA, &err));
    if (c[0] != 6) continue;
    auto bad = [&](const char* name, const std::function<void(HostStream&)>& f) {
      HostStream x = h;
      f(x);
      report(name, !validate_streamed(x, nA, &err));
    };
    bad("streamed_record_key", [&](HostStream& x) { x.pkey[0] = (uint32_t)nA | (0xffffu << 16); });
    bad("streamed_record_len", [&](HostStream& x) { x.plen.back() = (uint32_t)nA + 1; });
    bad("streamed_coupling_operand", [&](HostStream& x) { x.cpl[0] = (x.cpl[0] & ~0xff00u) | ((uint32_t)nA << 8); });
    bad("streamed_coupling_type", [&](HostStream& x) { x.cpl[0] = (x.cpl[0] & 0xffffu) | (56u << 16); });   // l1 > l2
    bad("streamed_coupling_type_range", [&](HostStream& x) { x.cpl[0] = (x.cpl[0] & 0xffffu) | (125u << 16); });
    bad("streamed_partner_range", [&](HostStream& x) { x.cpl[4 * (x.cpl.size() / 4 - 1) + 2] = (uint32_t)x.tkey.size() + 1; });
    bad("streamed_empty_range", [&](HostStream& x) { x.cpl[2] = x.cpl[1]; });
    bad("streamed_partner_key", [&](HostStream& x) { x.tkey[0] = (uint32_t)nA; });
  }
  for (const auto& c : pooled) {
    const int64_t nb = basis_size(c[0], c[1], c[2]);
    std::vector<double> c1(nb, 0.1), c2(nb, 0.2);
    HostAce h;
    const bool built = build_coupled(c[0], c[1], c[2], c1.data(), c2.data(), nb, &h, &err);
    report(("pool_valid_" + std::to_string(c[0]) + std::to_string(c[1]) + std::to_string(c[2])).c_str(),
           built && validate_coupled(h, &err));
    if (c[0] != 4) continue;
    auto bad = [&](const char* name, const std::function<void(HostAce&)>& f) {
      HostAce x = h;
      f(x);
      report(name, !validate_coupled(x, &err));
    };
    bad("pool_component", [&](HostAce& x) { x.comp[0] = (x.comp[0] & 0xffff0000u) | (uint32_t)(x.nA + 1); });
    bad("pool_gaunt_range", [&](HostAce& x) { x.comp[1] = ((uint32_t)x.gkey.size() << 8) | 1u; });
    bad("pool_record", [&](HostAce& x) { x.fkey.back() = (uint32_t)x.npool; });
    bad("pool_reverse_row", [&](HostAce& x) { x.qrow[4 * 1 + 1] = (int)x.rkey.size() + 1; });
    bad("pool_reverse_entry", [&](HostAce& x) { x.rkey[0] = (uint32_t)x.npool; });
    bad("pool_c_to_a", [&](HostAce& x) { x.bkey[0] = (x.bkey[0] & 0xffff0000u) | 1u; });
    bad("pool_pieces", [&](HostAce& x) { x.poff.back() += 1; });
    bad("pool_targets", [&](HostAce& x) { x.tpiece.back() = (int)x.poff.size(); });
  }
  return 0;
}
