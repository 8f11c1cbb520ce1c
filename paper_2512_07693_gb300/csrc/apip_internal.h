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
constexpr int kLearnedBlock = 128;   // threads per block of pass 1 with the learned switch
constexpr int kAceWarps = 8;               // warps per ACE block
constexpr int kAceThreads = 32 * kAceWarps;

// Device status words (apip_ctx::status)
enum {
  ST_NB_OVERFLOW = 0,   // some atom exceeded max_nb
  ST_CELL_OVERFLOW = 1, // some cell exceeded cell_cap
  ST_BAD_INPUT = 2,     // non-finite position / id out of range
  ST_BAD_PARTNER = 3,   // CSP partner id not present
  ST_MAX_NNB = 4,       // largest neighbour count seen (for the error text)
  ST_MAX_CELL = 5,      // largest cell occupancy seen
  ST_TIMEOUT = 6,       // a bounded device wait gave up
  ST_BOUNDS = 7,        // bounds-checked build: site of the first out-of-range index (0: none)
  ST_BOUNDS_VAL = 8,    // that index
  ST_BOUNDS_LIM = 9,    // and the limit it broke
  ST_COUNT = 10
};

// Sites of the bounds-checked build (APIP_CHECK_BOUNDS), reported by apip_sync.
enum {
  BND_NEIGHBOUR = 1,    // an atom index read from the neighbour list
  BND_LIST_LEN = 2,     // a neighbour-list length above max_nb
  BND_CELL = 3,         // a cell index or a cell member's atom index
  BND_COMPACT = 4,      // an entry of the compacted lists
  BND_ACE_TABLE = 5,    // an ACE table key or partner range
  BND_SELFTEST = 6      // apip_check_bounds_selftest
};

// Derived scalar parameters, passed by value to kernels.
struct Geo {
  double L[3];          // box edges
  double cs[3];         // cell edges (>= r_list)
  double invL[3];       // 1 / L
  int nc[3];            // cells per axis (>= 3)
  double inv_unit[3];   // 2^32 / L (FP32 path fixed-point coordinates) = unit_m 2^unit_s,
  unsigned long long unit_m[3];   // unit_m left-aligned (top bit set)
  int unit_s[3];
  float unit[3];        // L / 2^32
};

struct EamP { double A, beta, re, D, alpha, r0, rc, rc_lo, inv_w; };   // inv_w = 1/(rc - rc_lo)
struct SwP { double r_w, r_w_lo, d_lo, d_hi, d0, inv_w, inv_d; };  // 1/(r_w - r_w_lo), 1/(d_hi - d_lo)

// ACE table entries.  Rec: a forward record (key = o1 | o2 << 16, len = the
// segment length, k1/k2 = the coefficients of the two embedding channels) or a
// reverse-row entry (key = the partner segment's pool offset).  Ent: a Gaunt
// entry (key = (m1 + l1) | (m2 + l2) << 8) or a C -> A entry
// (key = C pool index | other A pool index << 16), v = the coefficient.
template <typename T> struct alignas(sizeof(T) == 4 ? 16 : 8) Rec { uint32_t key, len; T k1, k2; };
template <typename T> struct alignas(sizeof(T) == 4 ? 8 : 16) Ent { T v; uint32_t key; };

// ACE tables on the device.  Two evaluations:
//  pool (body order 4, built by build_coupled): per atom the pool
//    X = [1 | A (nA) | C (nC)] holds the atomic density and its Gaunt couplings,
//    every basis function is the dot product of two pool segments;
//  streamed (body order <= 3, built by build_streamed): the couplings are formed
//    one at a time in registers and contracted with their nu = 3 partners; nu = 1, 2
//    functions are dot products of A segments.
constexpr int kAcePool = 0, kAceStreamed = 1;

template <typename T>
struct AceDev {
  int kind;                     // kAcePool or kAceStreamed
  int n_max, l_max, nA, nC, npool;   // nA = n_max (l_max+1)^2, npool = 1 + nA + nC
  T rc, rc_lo, eps, sqrt_eps, a_scale;
  T two_over_rc, inv_width;     // 2 / rc and 1 / (rc - rc_lo) of the radial basis
  const uint2* comp;            // [nC]: (a1 | a2 << 16, gofs << 8 | gcnt) per C component
  const Ent<T>* gent;           // Gaunt entries
  const Rec<T>* frec; int nf;   // forward records, grouped by length
  const int4* qrow;             // [npool]: reverse row (begin, end) of the segment of q, m = q - segment start
  const Rec<T>* arec;           // reverse-row entries
  const Ent<T>* bent;           // C -> A entries, grouped by target
  const int* poff; int npc;     // [npc + 1] piece boundaries in bent
  const int* tpiece;            // [nA + 1] first piece of each target A component
  // streamed tables
  const Rec<T>* prec; int npr;  // nu 1, 2: key a1 | a2 << 16 (A indices; a2 = 0xffff: the constant 1), len
  const uint4* cpl; int ncpl;   // couplings: (a1 | a2 << 8 | type << 16, partner begin, partner end, 0)
  const Rec<T>* part; int npart;  // nu = 3 partners: key = A index of A_{p3, m = -l3}
  const Rec<T>* cfirst;         // the first partner record of each coupling (a copy, loaded with the coupling)
  int group;                    // compacted atoms per thread block
};

struct HostStream {
  std::vector<uint32_t> pkey, plen; std::vector<double> p1, p2;   // nu 1, 2 records
  std::vector<uint32_t> cpl;                                       // [4 per coupling]
  std::vector<uint32_t> tkey; std::vector<double> t1, t2;          // partners
  int64_t gaunt_products = 0;                                      // candidates over all couplings
};

struct HostAce {
  int nA = 0, nC = 0, npool = 0;
  std::vector<uint32_t> comp;                 // [2 nC]
  std::vector<uint32_t> gkey; std::vector<double> gval;
  std::vector<uint32_t> fkey, flen; std::vector<double> f1, f2;
  std::vector<int> qrow;                      // [4 npool]
  std::vector<uint32_t> rkey; std::vector<double> r1, r2;
  std::vector<uint32_t> bkey; std::vector<double> bval;
  std::vector<int> poff, tpiece;
};

// ace_tables.cpp
int64_t basis_size(int n_max, int l_max, int nu_max);
bool build_coupled(int n_max, int l_max, int nu_max, const double* c1, const double* c2, int64_t n_basis,
                   HostAce* out, std::string* err);
bool build_streamed(int n_max, int l_max, int nu_max, const double* c1, const double* c2, int64_t n_basis,
                    HostStream* out, std::string* err);
bool validate_streamed(const HostStream& h, int nA, std::string* err);
bool validate_coupled(const HostAce& h, std::string* err);
// real Gaunt values in the canonical layout of gaunt_layout.h (kGauntTotal entries)
void gaunt_fill(double* out);
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
  int64_t built_n = -1;        // atom count of the last neighbour-list build (or the last call)
  int ncell = 0, ncell_alloc = 0;
  bool csp_ready = false;
  const double* lam_fixed = nullptr;  // caller's per-atom constant lam (NaN = switch)
  bool ind_on = false;                 // spherical indenter
  double ind_c[3] = {}, ind_v[3] = {}, ind_R = 0.0, ind_K = 0.0;
  double* ind_acc = nullptr;           // [3] device: W, (sum F).v old, new
  int64_t lam_fixed_n = 0;
  std::string err;
  std::vector<double> ace_c1, ace_c2;

  // neighbour structures
  int* cell_count = nullptr;   // binning counters, zero outside a list build (read by the fill)
  uint4* cell_q = nullptr;     // FP32 path: posq of the cell members in cell order
  int* cell_atoms = nullptr;
  int* nnb = nullptr;
  int* nnb_e = nullptr;        // entries within eam_rc + skin at build time (they come first)
  int* nnb_0 = nullptr;        // FP32 path: entries within eam_rc at build time (they come first)
  float* mind1 = nullptr;      // FP32 path: least squared build distance of the entries in [eam_rc, eam_rc + skin)
  uint4* posg = nullptr;       // FP32 path: posq with g in .w (pass 1 -> pass 2)
  int* nbl = nullptr;          // column-major [max_nb][nmax]
  int* nbl_tmp = nullptr;      // list build scratch, same layout
  double* pos_ref = nullptr;   // [nmax][3]
  uint4* posq = nullptr;       // FP32 path: fixed-point wrapped position (x, y, z, 0)
  uint4* posq_ref = nullptr;   // FP32 path: posq at the last neighbour-list build
  int* id2idx = nullptr;       // [nmax]
  int* csp = nullptr;          // [nmax][kCspCap] partner ids
  int* csp_idx = nullptr;      // [nmax][kCspCap] partner indices of the atom at each index (cache)
  int* csp_owner = nullptr;    // [nmax] id of the atom each csp_idx row was built for (-1: none)

  // per-atom arrays (element size = precision)
  void* zeta = nullptr; void* xi_p = nullptr; void* e_eam = nullptr; void* g = nullptr;
  void* wbar = nullptr; void* dd = nullptr; void* lam = nullptr; void* dlam = nullptr;
  void* e_ace = nullptr;
  double* cvec = nullptr;      // [nmax] grad-lambda CSP coefficients (kept zero between calls)
  int* ace_list = nullptr;     // [nmax]
  int* clist = nullptr;        // [nmax] learned switch: atoms with a grad-lambda coefficient
  int* counts = nullptr;       // [4]: |P|, learned c-vector count, scratch
  int* blk_cnt = nullptr;      // deterministic mode: pass 2's per-block counts of lam > 0, then their offsets
  bool det = false;            // apip_params.deterministic
  int* flags = nullptr;        // [4]: need_rebuild, largest squared displacement since the build (float bits)
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

  // ACE tables (element size = precision): one device buffer, sub-arrays at
  // the byte offsets ace_off (order of AceDev's pointers)
  void* ace_tab = nullptr;
  size_t ace_off[8] = {};
  int ace_nf = 0, ace_npc = 0, ace_nC = 0, ace_npool = 0;
  int ace_group = 1;
  int ace_kind = 0, ace_npr = 0, ace_ncpl = 0, ace_npart = 0;
  int64_t ace_info[APIP_ACE_INFO_COUNT] = {};

  // learned indicator
  void* mlp_w = nullptr;       // APIP_MLP_NPARAM weights (element size = precision)
  void* mlp_img = nullptr;     // FP32: the weights as split bfloat16 tensor-core operand images
  int learned_slots = 0;       // FP32: resident CTAs of the tensor-core learned force kernel
  int learned_slots1 = 0;      // FP32: resident CTAs of the tensor-core network of pass 1
  float* mlp_x0 = nullptr;     // FP32 learned switch: network inputs [nmax][32]
  bool mlp_ready = false;
  float* mlp_ws = nullptr;     // training workspace
  size_t mlp_ws_cap = 0;       // floats
};
