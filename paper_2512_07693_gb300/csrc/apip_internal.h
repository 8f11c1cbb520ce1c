// Internal declarations of libapip shared by the host orchestration
// (apip.cu), the kernels and the ACE table builder.  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "apip.h"

namespace apip {

constexpr int kNmaxCap = 8;    // largest n_max
constexpr int kLmaxCap = 4;    // largest l_max
constexpr int kCspCap = 8;     // largest csp_nnb
constexpr int kBlock = 256;    // threads per block of the all-atom passes
constexpr int kAceAdjWarps = 8;            // warps per ACE block
constexpr int kAceChunk = 1024;            // table records per shared-memory stage
constexpr int kAceThreads = 32 * kAceAdjWarps;

// Device status words (apip_ctx::status)
enum {
  ST_NB_OVERFLOW = 0,   // some atom exceeded max_nb
  ST_CELL_OVERFLOW = 1, // some cell exceeded cell_cap
  ST_BAD_INPUT = 2,     // non-finite position / id out of range
  ST_BAD_PARTNER = 3,   // CSP partner id not present
  ST_MAX_NNB = 4,       // largest neighbour count seen (for the error text)
  ST_MAX_CELL = 5,      // largest cell occupancy seen
  ST_TIMEOUT = 6,       // a bounded device wait gave up
  ST_COUNT = 8
};

// Derived scalar parameters, passed by value to kernels.
struct Geo {
  double L[3];          // box edges
  double cs[3];         // cell edges (>= r_list)
  double invL[3];       // 1 / L
  int nc[3];            // cells per axis (>= 3)
  double inv_unit[3];   // 2^32 / L (FP32 path fixed-point coordinates)
  float unit[3];        // L / 2^32
};

struct EamP { double A, beta, re, D, alpha, r0, rc, rc_lo, inv_w; };   // inv_w = 1/(rc - rc_lo)
struct SwP { double r_w, r_w_lo, d_lo, d_hi, d0, inv_w, inv_d; };  // 1/(r_w - r_w_lo), 1/(d_hi - d_lo)

// One record of an ACE table: packed 8-bit A indices and the coefficients of the
// two embedding channels; 16-byte aligned so that chunks of records can be
// copied into shared memory by bulk asynchronous copies.
template <typename T> struct Rec;
template <> struct alignas(16) Rec<float> { uint32_t key; float k1, k2; uint32_t pad; };
template <> struct alignas(16) Rec<double> { uint32_t key, pad; double k1, k2; uint64_t pad2; };

// ACE tables on the device: terms of the folded product basis,
//   phi_c = sum_t K_c[t] prod_{q} A[idx_q(t)],  c = 1, 2,
// with A[nA] == 1 padding the lower body orders.  Keys hold 8-bit indices.
template <typename T>
struct AceDev {
  int n_max, l_max, nA;         // nA = n_max (l_max+1)^2
  T rc, rc_lo, eps, sqrt_eps, a_scale;
  const Rec<T>* rec3; int n3;   // 3-index terms
  const Rec<T>* rec4; int n4;   // 4-index terms
  const Rec<T>* recd; int nd;   // derivative entries, sorted by target
  const int* sched;             // adjoint schedule (HostTerms::sched)
  int group;                    // compacted atoms per thread block (1 or 8)
};

struct HostTerms {
  std::vector<uint32_t> key3, key4, keyd;
  std::vector<double> k3a, k3b, k4a, k4b, kda, kdb;
  // adjoint schedule: sched[0] = number of chunks nch; then nch + 1 entry offsets
  // of the chunks; then nch * kAceAdjWarps + 1 offsets (in pieces) of the pieces of
  // chunk c, warp w at index c * kAceAdjWarps + w; then the pieces as (target,
  // start, end) relative to their chunk
  std::vector<int> sched;
};

// ace_tables.cpp
int64_t basis_size(int n_max, int l_max, int nu_max);
bool build_terms(int n_max, int l_max, int nu_max, const double* c1, const double* c2,
                 int64_t n_basis, HostTerms* out, std::string* err);
// real Y_lm normalisation N_lm (times sqrt 2 for m != 0), index l^2 + l + m
void ylm_norms(int l_max, double* out);
// real Gaunt coefficient int Y_l1m1 Y_l2m2 Y_l3m3 dOmega (the library's own construction)
double real_gaunt(int l1, int m1, int l2, int m2, int l3, int m3);

}  // namespace apip

// The opaque context of the C ABI.
struct apip_ctx {
  apip_params p;
  int64_t nmax = 0;
  int dev = 0;
  double r_list = 0.0;
  apip::Geo geo{};
  bool geo_set = false;
  int ncell = 0, ncell_alloc = 0;
  bool csp_ready = false;
  std::string err;
  std::vector<double> ace_c1, ace_c2;

  // neighbour structures
  int* cell_count = nullptr;
  int* cell_atoms = nullptr;
  int* nnb = nullptr;
  int* nbl = nullptr;          // column-major [max_nb][nmax]
  double* pos_ref = nullptr;   // [nmax][3]
  uint4* posq = nullptr;       // FP32 path: fixed-point wrapped position (x, y, z, 0)
  uint4* posq_ref = nullptr;   // FP32 path: posq at the last neighbour-list build
  int* id2idx = nullptr;       // [nmax]
  int* csp = nullptr;          // [nmax][kCspCap] partner ids

  // per-atom arrays (element size = precision)
  void* zeta = nullptr; void* xi_p = nullptr; void* e_eam = nullptr; void* g = nullptr;
  void* wbar = nullptr; void* dd = nullptr; void* lam = nullptr; void* dlam = nullptr;
  void* e_ace = nullptr;
  double* cvec = nullptr;      // [nmax] grad-lambda CSP coefficients (kept zero between calls)
  int* ace_list = nullptr;     // [nmax]
  int* counts = nullptr;       // [4]: |P|, scratch
  int* flags = nullptr;        // [4]: need_rebuild
  int* status = nullptr;       // [ST_COUNT]
  double* partials = nullptr;  // energy partials: P1 blocks then ACE warps
  double* thermo_part = nullptr;  // [blocks][4] KE, px, py, pz
  double* e_scratch = nullptr;    // [2] total energy scratch
  int n_part = 0;
  int ace_blocks = 0;

  // phase timing (apip_profile)
  bool prof = false;
  struct ProfRec { int phase; int launches; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[APIP_PHASE_COUNT] = {};
  int64_t prof_n[APIP_PHASE_COUNT] = {};

  // ACE tables (element size = precision)
  void* rec3 = nullptr; int n3 = 0;   // Rec<T> arrays
  void* rec4 = nullptr; int n4 = 0;
  void* recd = nullptr; int nd = 0;
  int* sched = nullptr;

  // learned indicator
  void* mlp_w = nullptr;       // APIP_MLP_NPARAM weights (element size = precision)
  bool mlp_ready = false;
  float* mlp_ws = nullptr;     // training workspace
  size_t mlp_ws_cap = 0;       // floats
};
