// C ABI of libapip: context management and the host-side orchestration of the
// adaptive-precision force pipeline (one stream, no host synchronisation):
//
//   prep -> [neighbour rebuild, skipped on the device unless an atom moved more
//   than skin/2] -> pass 1 (EAM density, g) -> pass 2 (switch, EAM force,
//   compaction of lam > 0) -> ACE on the compacted atoms -> CSP part of
//   grad-lambda -> float64 energy reduction.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "gaunt_layout.h"
#include "kernels.h"

using namespace apip;

namespace {

// An NVTX range: a named span of host time that a profiler attached to the
// process shows on its timeline and by which ncu's --nvtx filters select the
// kernels launched inside it.  Each call is one range ("apip_energy_forces", ...)
// with one nested range per phase ("apip.pass2", ...).  Without an attached
// tool a push or pop costs a few nanoseconds.
struct NvtxRange {
  bool open = true;
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  void end() {
    if (open) nvtxRangePop();
    open = false;
  }
  ~NvtxRange() { end(); }
};

apip_status fail(apip_ctx* c, apip_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define APIP_CK(expr)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(ctx, APIP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int nblk(int64_t n) { return (int)std::max<int64_t>(1, (n + kBlock - 1) / kBlock); }

size_t esize(const apip_ctx* c) { return c->p.precision == APIP_FP32 ? sizeof(float) : sizeof(double); }

template <typename T> T* as(void* p) { return reinterpret_cast<T*>(p); }

cudaEvent_t take_event(apip_ctx* c) {
  if (!c->prof_pool.empty()) {
    cudaEvent_t e = c->prof_pool.back();
    c->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records CUDA events around one phase of a call when profiling is enabled.
struct Phase {
  apip_ctx* c;
  int phase, launches;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  Phase(apip_ctx* c_, int ph, int nl, cudaStream_t s_) : c(c_), phase(ph), launches(nl), s(s_) {
    if (c->prof) {
      a = take_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~Phase() {
    if (!c->prof) return;
    cudaEvent_t b = take_event(c);
    cudaEventRecord(b, s);
    c->prof_pending.push_back({phase, launches, a, b});
  }
};

void free_all(apip_ctx* c) {
  for (auto& r : c->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
  c->prof_pending.clear();
  c->prof_pool.clear();
  void* ptrs[] = {c->cell_count, c->cell_atoms, c->cell_q, c->nnb, c->nnb_e, c->nnb_0, c->mind1, c->posg, c->nbl, c->nbl_tmp, c->pos_ref, c->posq, c->posq_ref, c->id2idx,
                  c->csp, c->csp_idx, c->csp_owner, c->zeta, c->xi_p, c->e_eam, c->g, c->wbar, c->dd, c->lam, c->dlam, c->e_ace,
                  c->cvec, c->ace_list, c->clist, c->counts, c->flags, c->status, c->partials, c->thermo_part,
                  c->e_scratch, c->ind_acc, c->blk_cnt, c->ace_tab, c->mlp_w, c->mlp_img, c->mlp_x0, c->mlp_ws};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

apip_status check_params(const apip_params* p, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return APIP_ERR_ARG; };
  if (p->precision != APIP_FP64 && p->precision != APIP_FP32) return bad("precision must be APIP_FP64 or APIP_FP32");
  if (p->lam_mode < APIP_LAM_PAPER || p->lam_mode > APIP_LAM_LEARNED) return bad("unknown lam_mode");
  if (p->ace_n_max < 1 || p->ace_n_max > kNmaxCap) return bad("ace_n_max must be in [1, 8]");
  if (p->ace_l_max < 0 || p->ace_l_max > kLmaxCap) return bad("ace_l_max must be in [0, 4]");
  if (p->ace_nu_max < 1 || p->ace_nu_max > 4) return bad("ace_nu_max must be in [1, 4]");
  if (p->ace_n_max * (p->ace_l_max + 1) * (p->ace_l_max + 1) > 254) return bad("n_max (l_max+1)^2 must be <= 254");
  if (p->ace_group != 0 && p->ace_group != 1 && p->ace_group != 2 && p->ace_group != 4 && p->ace_group != 8 &&
      p->ace_group != 32)
    return bad("ace_group must be 0, 1, 2, 4, 8 or 32");
  if (!p->ace_c1 || !p->ace_c2) return bad("ace_c1 / ace_c2 must not be NULL");
  if (p->mixing != APIP_MIX_ENERGY && p->mixing != APIP_MIX_FORCE) return bad("unknown mixing");
  if (p->deterministic != 0 && p->deterministic != 1) return bad("deterministic must be 0 or 1");
  if (p->deterministic && p->mixing == APIP_MIX_FORCE) return bad("the deterministic mode does not support force mixing");
  // the float64 path and the evaluations with l_max = 4 or body order 4 sum dE/dA
  // with shared-memory atomics, whose order is not fixed
  if (p->deterministic && !(p->precision == APIP_FP32 && p->ace_nu_max <= 3 && p->ace_l_max <= 3))
    return bad("the deterministic mode needs the float32 path with ACE body order <= 3 and l_max <= 3");
  if (!(p->ace_rc > 0 && p->ace_rc_width > 0 && p->ace_rc_width <= p->ace_rc)) return bad("bad ACE cutoff");
  if (!(p->ace_eps > 0)) return bad("ace_eps must be > 0");
  if (!std::isfinite(p->prec_shift)) return bad("prec_shift must be finite");
  if (!(p->eam_rc > 0 && p->eam_rc_width > 0 && p->eam_rc_width <= p->eam_rc)) return bad("bad EAM cutoff");
  if (!(p->sw_r_w > 0 && p->sw_r_w_width > 0 && p->sw_r_w_width <= p->sw_r_w)) return bad("bad switch cutoff");
  if (!(p->sw_d_hi > p->sw_d_lo)) return bad("sw_d_hi must exceed sw_d_lo");
  if (p->csp_nnb < 2 || p->csp_nnb > kCspCap || p->csp_nnb % 2) return bad("csp_nnb must be even, 2..8");
  if (!(p->csp_rcut > 0)) return bad("csp_rcut must be > 0");
  if (!(p->skin >= 0)) return bad("skin must be >= 0");
  if (p->max_nb < 1 || p->max_nb > 1024) return bad("max_nb must be in [1, 1024]");
  if (p->cell_cap < 1 || p->cell_cap > 1024) return bad("cell_cap must be in [1, 1024]");
  const double cut = std::max(std::max(p->eam_rc, p->ace_rc), p->sw_r_w);
  if (p->csp_rcut > cut + p->skin) return bad("csp_rcut must not exceed the neighbour cutoff + skin");
  return APIP_OK;
}

// Cell grid for a new box; marks the neighbour list for rebuild.
apip_status set_geometry(apip_ctx* ctx, const double* box, cudaStream_t s) {
  if (!box) return fail(ctx, APIP_ERR_ARG, "box must not be NULL");
  for (int k = 0; k < 3; ++k)
    if (!(std::isfinite(box[k]) && box[k] > 0)) return fail(ctx, APIP_ERR_ARG, "box edges must be finite and > 0");
  if (ctx->geo_set && box[0] == ctx->geo.L[0] && box[1] == ctx->geo.L[1] && box[2] == ctx->geo.L[2]) return APIP_OK;
  Geo g{};
  int ncell = 1;
  for (int k = 0; k < 3; ++k) {
    g.L[k] = box[k];
    g.nc[k] = (int)std::floor(box[k] / ctx->r_list);
    if (g.nc[k] < 3)
      return fail(ctx, APIP_ERR_ARG, "each box edge must be >= 3 * (cutoff + skin) = " + std::to_string(3 * ctx->r_list));
    g.cs[k] = box[k] / g.nc[k];
    g.invL[k] = 1.0 / box[k];
    g.inv_unit[k] = 4294967296.0 / box[k];
    int x = 0;
    const double f = std::frexp(g.inv_unit[k], &x);   // f in [0.5, 1): f 2^64 is an exact integer
    g.unit_m[k] = (unsigned long long)std::ldexp(f, 64);
    g.unit_s[k] = x - 64;
    g.unit[k] = (float)(box[k] / 4294967296.0);
    ncell *= g.nc[k];
  }
  if (ncell > ctx->ncell_alloc) {
    if (ctx->cell_count) cudaFree(ctx->cell_count);
    if (ctx->cell_atoms) cudaFree(ctx->cell_atoms);
    if (ctx->cell_q) cudaFree(ctx->cell_q);
    ctx->cell_count = nullptr;
    ctx->cell_atoms = nullptr;
    ctx->cell_q = nullptr;
    APIP_CK(cudaMalloc(&ctx->cell_count, sizeof(int) * ncell));
    APIP_CK(cudaMemsetAsync(ctx->cell_count, 0, sizeof(int) * ncell, s));
    // members: FP64 path their indices, FP32 path their fixed-point positions with
    // the index in .w
    if (ctx->p.precision == APIP_FP32)
      APIP_CK(cudaMalloc(&ctx->cell_q, sizeof(uint4) * (size_t)ncell * ctx->p.cell_cap));
    else
      APIP_CK(cudaMalloc(&ctx->cell_atoms, sizeof(int) * (size_t)ncell * ctx->p.cell_cap));
    ctx->ncell_alloc = ncell;
  }
  ctx->ncell = ncell;
  ctx->geo = g;
  ctx->geo_set = true;
  APIP_CK(cudaMemsetAsync(ctx->flags, 0xff, sizeof(int), s));
  return APIP_OK;
}

// A call with another atom count than the last list build needs a new list: the
// old one holds indices of atoms that may be gone (n shrank) or misses the new
// atoms (n grew).  Marks the list for rebuild on the stream.
void mark_atom_count(apip_ctx* c, int n, cudaStream_t s) {
  if (n == c->built_n) return;
  cudaMemsetAsync(c->flags, 0xff, sizeof(int), s);
  c->built_n = n;
}

}  // namespace

namespace apip {

// The indenter centre for the kernels: as given (FP64 path) and as wrapped
// fixed-point coordinates (FP32 path).
template <typename T>
void set_ind_center(Args<T>& a, const Geo& g, const double c[3]) {
  unsigned q[3];
  for (int k = 0; k < 3; ++k) {
    a.ind_c[k] = c[k];
    double w = c[k] - g.L[k] * std::floor(c[k] * g.invL[k]);
    if (w >= g.L[k]) w -= g.L[k];
    q[k] = fixed_coord(w, g.unit_m[k], g.unit_s[k]);
  }
  a.ind_q = make_uint4(q[0], q[1], q[2], 0u);
}

template <typename T>
Args<T> make_args(apip_ctx* c, const double* pos, const int* id, int n, double* force, double* e_atom) {
  Args<T> a{};
  const apip_params& p = c->p;
  a.n = n;
  a.nmax = (int)c->nmax;
  a.max_nb = p.max_nb;
  a.cell_cap = p.cell_cap;
  a.csp_nnb = p.csp_nnb;
  a.lam_mode = p.lam_mode;
  a.precise_adds_eam = p.precise_adds_eam;
  a.force_mix = p.mixing == APIP_MIX_FORCE;
  a.grad_lambda = a.force_mix ? 0 : p.grad_lambda;
  a.eam_force = 1;
  a.lam_fixed = c->lam_fixed;
  a.ind_on = c->ind_on ? 1 : 0;
  a.ind_acc = c->ind_acc;
  a.ind_R2 = T(c->ind_R * c->ind_R);
  a.ind_Rd = c->ind_R;
  a.ind_Kd = c->ind_K;
  for (int k = 0; k < 3; ++k) a.ind_v[k] = c->ind_v[k];
  set_ind_center(a, c->geo, c->ind_c);
  a.geo = c->geo;
  a.eam = {p.eam_A, p.eam_beta, p.eam_re, p.eam_D, p.eam_alpha, p.eam_r0, p.eam_rc, p.eam_rc - p.eam_rc_width,
           1.0 / p.eam_rc_width};
  a.sw = {p.sw_r_w, p.sw_r_w - p.sw_r_w_width, p.sw_d_lo, p.sw_d_hi, p.sw_d0, 1.0 / p.sw_r_w_width,
          1.0 / (p.sw_d_hi - p.sw_d_lo)};
  a.k = {T(p.eam_A), T(p.eam_beta), T(p.eam_re), T(p.eam_D), T(p.eam_alpha), T(p.eam_r0), T(p.eam_rc),
         T(p.eam_rc * p.eam_rc), T(p.eam_rc - p.eam_rc_width), T(1.0 / p.eam_rc_width),
         T(p.sw_r_w), T(p.sw_r_w * p.sw_r_w), T(p.sw_r_w - p.sw_r_w_width), T(1.0 / p.sw_r_w_width),
         T(p.sw_d_lo), T(p.sw_d_hi), T(1.0 / (p.sw_d_hi - p.sw_d_lo)), T(p.sw_d0), T(p.prec_shift)};
  for (int k = 0; k < 3; ++k) {
    const double u = c->geo.L[k] / 4294967296.0;
    a.swff.u_hi[k] = (float)u;
    a.swff.u_lo[k] = (float)(u - (double)a.swff.u_hi[k]);
  }
  {
    const double cc = p.sw_r_w + (p.sw_r_w - p.sw_r_w_width);
    a.swff.c_hi = (float)cc;
    a.swff.c_lo = (float)(cc - (double)a.swff.c_hi);
    a.swff.inv_w = (float)(1.0 / p.sw_r_w_width);
    // the float-float r^2 is compared on its high part: bounds rounded outwards, so
    // that every pair of the taper is evaluated (beyond r_w, w = 0 exactly)
    a.swff.rw2 = std::nextafter((float)(p.sw_r_w * p.sw_r_w), INFINITY);
    a.swff.rw_lo2 = std::nextafter((float)((p.sw_r_w - p.sw_r_w_width) * (p.sw_r_w - p.sw_r_w_width)), 0.0f);
  }
  a.r_list2 = c->r_list * c->r_list;
  a.skin_half2 = 0.25 * p.skin * p.skin;
  a.skin_half2_f = (float)a.skin_half2;
  if ((double)a.skin_half2_f > a.skin_half2) a.skin_half2_f = std::nextafter(a.skin_half2_f, 0.0f);
  // a pair now within eam_rc was within eam_rc + skin at the last build (each atom
  // moved less than skin / 2); the margin covers the rounding of the trigger
  a.r_e_in2 = p.eam_rc * p.eam_rc;
  a.r_e_mid2 = (p.eam_rc + p.skin + 1e-3) * (p.eam_rc + p.skin + 1e-3);
  a.csp_rcut2 = p.csp_rcut * p.csp_rcut;
  a.pos = pos;
  a.id = id;
  a.nnb_e = c->nnb_e; a.nnb_0 = c->nnb_0; a.mind1 = c->mind1; a.posg = c->posg;
  a.nnb = c->nnb; a.nbl = c->nbl; a.nbl_tmp = c->nbl_tmp; a.pos_ref = c->pos_ref; a.posq = c->posq; a.posq_ref = c->posq_ref;
  a.id2idx = c->id2idx; a.csp = c->csp; a.csp_idx = c->csp_idx; a.csp_owner = c->csp_owner; a.cell_count = c->cell_count; a.cell_atoms = c->cell_atoms;
  a.ncell = c->ncell;
  a.cell_q = c->cell_q;
  a.zeta = as<T>(c->zeta); a.xi_p = as<T>(c->xi_p); a.e_eam = as<T>(c->e_eam); a.g = as<T>(c->g);
  a.wbar = as<T>(c->wbar); a.dd = as<T>(c->dd); a.lam = as<T>(c->lam); a.dlam = as<T>(c->dlam);
  a.e_ace = as<T>(c->e_ace);
  a.cvec = c->cvec; a.ace_list = c->ace_list; a.clist = c->clist; a.counts = c->counts;
  a.flags = c->flags; a.status = c->status;
  a.det = c->det ? 1 : 0; a.blk_cnt = c->blk_cnt;
  a.partials = c->partials;
  // one energy partial per pass-1 block, ahead of the ACE blocks' partials
  if (p.lam_mode != APIP_LAM_LEARNED) a.n_part_p1 = nblk(n);
  else if (sizeof(T) == 4) a.n_part_p1 = nblk(n);   // the descriptor kernel's blocks
  else a.n_part_p1 = (int)std::max<int64_t>(1, (n + kLearnedBlock - 1) / kLearnedBlock);
  a.force = force;
  a.e_atom = e_atom;
  a.mlp_w = as<T>(c->mlp_w);
  a.mlp_img = static_cast<const uint4*>(c->mlp_img);
  a.mlp_x0 = c->mlp_x0;
  a.learned_grid = c->learned_slots;
  a.learned_grid1 = c->learned_slots1;
  a.ace_rc = T(p.ace_rc);
  a.ace_rc_lo = T(p.ace_rc - p.ace_rc_width);
  return a;
}

}  // namespace apip

namespace {

template <typename T> void set_view(Args<T>& a, apip_ctx* c);
template <> void set_view<double>(Args<double>& a, apip_ctx* c) {
  a.pv.pos = a.pos;
  for (int k = 0; k < 3; ++k) { a.pv.L[k] = c->geo.L[k]; a.pv.invL[k] = 1.0 / c->geo.L[k]; }
}
template <> void set_view<float>(Args<float>& a, apip_ctx* c) {
  a.pv.q = c->posq;
  for (int k = 0; k < 3; ++k) a.pv.unit[k] = c->geo.unit[k];
}

template <typename T>
AceDev<T> ace_dev(apip_ctx* c) {
  AceDev<T> t{};
  const apip_params& p = c->p;
  t.n_max = p.ace_n_max;
  t.l_max = p.ace_l_max;
  t.nA = p.ace_n_max * (p.ace_l_max + 1) * (p.ace_l_max + 1);
  t.rc = T(p.ace_rc);
  t.rc_lo = T(p.ace_rc - p.ace_rc_width);
  t.eps = T(p.ace_eps);
  t.sqrt_eps = T(std::sqrt(p.ace_eps));
  t.a_scale = T(p.ace_a_scale);
  t.two_over_rc = T(2.0 / p.ace_rc);
  t.inv_width = T(1.0 / p.ace_rc_width);
  t.kind = c->ace_kind;
  t.nC = c->ace_nC;
  t.npool = c->ace_npool;
  unsigned char* b = static_cast<unsigned char*>(c->ace_tab);
  if (t.kind == kAceStreamed) {
    t.prec = reinterpret_cast<const Rec<T>*>(b + c->ace_off[0]);
    t.npr = c->ace_npr;
    t.cpl = reinterpret_cast<const uint4*>(b + c->ace_off[1]);
    t.ncpl = c->ace_ncpl;
    t.part = reinterpret_cast<const Rec<T>*>(b + c->ace_off[2]);
    t.npart = c->ace_npart;
    t.cfirst = reinterpret_cast<const Rec<T>*>(b + c->ace_off[3]);
    t.group = c->ace_group;
    return t;
  }
  t.comp = reinterpret_cast<const uint2*>(b + c->ace_off[0]);
  t.gent = reinterpret_cast<const Ent<T>*>(b + c->ace_off[1]);
  t.frec = reinterpret_cast<const Rec<T>*>(b + c->ace_off[2]);
  t.nf = c->ace_nf;
  t.qrow = reinterpret_cast<const int4*>(b + c->ace_off[3]);
  t.arec = reinterpret_cast<const Rec<T>*>(b + c->ace_off[4]);
  t.bent = reinterpret_cast<const Ent<T>*>(b + c->ace_off[5]);
  t.poff = reinterpret_cast<const int*>(b + c->ace_off[6]);
  t.npc = c->ace_npc;
  t.tpiece = reinterpret_cast<const int*>(b + c->ace_off[7]);
  t.group = c->ace_group;
  return t;
}

apip_status check_call(apip_ctx* ctx, const double* pos, const int32_t* id, int64_t n) {
  if (!ctx) return APIP_ERR_ARG;
  if (n < 0 || n > ctx->nmax) return fail(ctx, APIP_ERR_ARG, "n must be in [0, n_atoms_max]");
  if (ctx->lam_fixed && n > ctx->lam_fixed_n)
    return fail(ctx, APIP_ERR_ARG, "lam_fixed holds fewer than n entries");
  if (n > 0 && (!pos || !id)) return fail(ctx, APIP_ERR_ARG, "pos and id must not be NULL");
  return APIP_OK;
}

// Call-order state: the switch needs its inputs set up first.
apip_status ready(apip_ctx* ctx) {
  if (ctx->p.lam_mode == APIP_LAM_PAPER && !ctx->csp_ready)
    return fail(ctx, APIP_ERR_STATE, "apip_init_csp_pairs must be called before the paper's switch is used");
  if (ctx->p.lam_mode == APIP_LAM_LEARNED && !ctx->mlp_ready)
    return fail(ctx, APIP_ERR_STATE, "apip_set_mlp must be called before the learned switch is used");
  return APIP_OK;
}

apip_status launch_status(apip_ctx* ctx) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, APIP_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return APIP_OK;
}

// Pass 1 for the switch in use: CSP^list g, or the learned g = MLP(G).
template <typename T>
void pass1(const Args<T>& a, cudaStream_t s) {
  if (a.lam_mode == APIP_LAM_LEARNED) launch_pass1_learned<T>(a, s);
  else launch_pass1<T>(a, s);
}

// The force pipeline after prep (or after the drift of a Verlet step).
template <typename T>
void force_pipeline(apip_ctx* c, Args<T>& a, cudaStream_t s) {
  { NvtxRange nv("apip.neighbor"); Phase ph(c, APIP_PHASE_NEIGHBOR, a.det ? 3 : 2, s); launch_neighbors<T>(a, c->ncell, s); }
  { NvtxRange nv("apip.pass1"); Phase ph(c, APIP_PHASE_PASS1, 1, s); pass1<T>(a, s); }
  { NvtxRange nv("apip.pass2"); Phase ph(c, APIP_PHASE_PASS2, a.det ? 3 : 1, s); launch_pass2<T>(a, s);
    if (a.force_mix) launch_fm_buffer<T>(a, s); }
  { NvtxRange nv("apip.ace"); Phase ph(c, APIP_PHASE_ACE, 1, s); const AceDev<T> t = ace_dev<T>(c);
    if (t.kind == kAceStreamed) launch_ace_stream<T>(a, t, c->ace_blocks, s);
    else launch_ace_pool<T>(a, t, c->ace_blocks, s); }
  if (a.lam_mode == APIP_LAM_PAPER && a.grad_lambda) {
    NvtxRange nv("apip.csp");
    Phase ph(c, APIP_PHASE_CSP, 1, s);
    launch_csp_force<T>(a, s);
  } else if (a.lam_mode == APIP_LAM_LEARNED && a.grad_lambda) {
    NvtxRange nv("apip.csp");
    Phase ph(c, APIP_PHASE_CSP, 1, s);
    launch_mlp_force<T>(a, s);
  }
  if (a.det && a.force) {   // the fixed-point force sums back to float64
    NvtxRange nv("apip.csp");
    Phase ph(c, APIP_PHASE_CSP, 1, s);
    launch_fix_finish(a.force, a.n, s);
  }
}

template <typename T>
apip_status energy_forces_t(apip_ctx* c, const double* pos, const int32_t* id, int n, double* force,
                            double* e_atom, double* e_total, cudaStream_t s) {
  NvtxRange nv_call("apip_energy_forces");
  Args<T> a = make_args<T>(c, pos, id, n, force, e_atom);
  set_view<T>(a, c);
  mark_atom_count(c, n, s);
  { NvtxRange nv("apip.prep"); Phase ph(c, APIP_PHASE_PREP, 1, s); launch_prep<T>(a, s); }
  force_pipeline<T>(c, a, s);
  if (e_total) {
    Phase ph(c, APIP_PHASE_REDUCE, 1, s);
    launch_final(c->partials, a.n_part_p1 + c->ace_blocks, e_total, nullptr, nullptr, 0, nullptr,
                 c->flags, c->counts, nullptr, c->cell_count, c->ncell, s);
  }
  if (a.ind_on) launch_ind_work(c->ind_acc, 0.0, a.det, s);
  return launch_status(c);
}

template <typename T>
apip_status switch_t(apip_ctx* c, const double* pos, const int32_t* id, int n, double* lam_out,
                     double* dlam_out, int64_t* n_ace_out, cudaStream_t s) {
  NvtxRange nv_call("apip_switch");
  Args<T> a = make_args<T>(c, pos, id, n, nullptr, nullptr);
  set_view<T>(a, c);
  a.eam_force = 0;
  mark_atom_count(c, n, s);
  launch_prep<T>(a, s);
  launch_neighbors<T>(a, c->ncell, s);
  pass1<T>(a, s);
  launch_pass2<T>(a, s);
  if (lam_out) launch_get_field<T>(a, APIP_FIELD_LAM, lam_out, s);
  if (dlam_out) launch_get_field<T>(a, APIP_FIELD_DLAM, dlam_out, s);
  launch_final(c->partials, 0, nullptr, nullptr, nullptr, 0, nullptr, c->flags, c->counts, n_ace_out, c->cell_count,
               c->ncell, s);
  return launch_status(c);
}

template <typename T>
apip_status neighbors_t(apip_ctx* c, const double* pos, const int32_t* id, int n, cudaStream_t s) {
  NvtxRange nv_call("apip_build_neighbors");
  Args<T> a = make_args<T>(c, pos, id, n, nullptr, nullptr);
  set_view<T>(a, c);
  launch_prep<T>(a, s);
  cudaMemsetAsync(c->flags, 0xff, sizeof(int), s);
  c->built_n = n;
  launch_neighbors<T>(a, c->ncell, s);
  cudaMemsetAsync(c->cell_count, 0, sizeof(int) * c->ncell, s);
  cudaMemsetAsync(c->flags, 0, sizeof(int), s);
  return launch_status(c);
}

template <typename T>
apip_status verlet_t(apip_ctx* c, double* pos, double* vel, double* force, const double* inv_mass,
                     const int32_t* id, int n, double dt, int steps, double* thermo, cudaStream_t s) {
  NvtxRange nv_call("apip_verlet_step");
  Args<T> a = make_args<T>(c, pos, id, n, force, nullptr);
  set_view<T>(a, c);
  mark_atom_count(c, n, s);
  const int ntb = nblk(n);
  const int n_part = a.n_part_p1 + c->ace_blocks;
  // without thermo output the step needs no reduction at all: the energy partials
  // are left unread and the ACE kernel clears the rebuild flag
  double* tp = thermo ? c->thermo_part : nullptr;
  for (int k = 0; k < steps; ++k) {
    { NvtxRange nv("apip.prep"); Phase ph(c, APIP_PHASE_PREP, 1, s); launch_verlet<T>(a, k == 0 ? 0 : 1, pos, vel, force, inv_mass, dt, k > 0 ? tp : nullptr, s); }
    if (a.ind_on) {   // the indenter centre moves with the drift
      for (int q = 0; q < 3; ++q) c->ind_c[q] += dt * c->ind_v[q];
      set_ind_center(a, c->geo, c->ind_c);
    }
    force_pipeline<T>(c, a, s);
    if (a.ind_on) launch_ind_work(c->ind_acc, dt, a.det, s);
    if (thermo) {
      Phase ph(c, APIP_PHASE_REDUCE, 1, s);
      launch_final(c->partials, n_part, nullptr, thermo + 5 * k, k > 0 ? tp : nullptr, ntb,
                   k > 0 ? thermo + 5 * (k - 1) : nullptr, c->flags, c->counts, nullptr, c->cell_count, c->ncell, s);
    }
  }
  { NvtxRange nv("apip.prep"); Phase ph(c, APIP_PHASE_PREP, 1, s); launch_verlet<T>(a, 2, pos, vel, force, inv_mass, dt, tp, s); }
  if (thermo) {
    Phase ph(c, APIP_PHASE_REDUCE, 1, s);
    launch_thermo_final(c->thermo_part, ntb, thermo + 5 * (steps - 1), s);
  }
  return launch_status(c);
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

int64_t apip_ace_basis_size(int32_t n_max, int32_t l_max, int32_t nu_max) {
  return basis_size(n_max, l_max, nu_max);
}

apip_status apip_create(const apip_params* p, int64_t n_atoms_max, apip_ctx** out) {
  if (!p || !out) return APIP_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (check_params(p, &why) != APIP_OK) return APIP_ERR_ARG;
  if (n_atoms_max < 1 || n_atoms_max > (int64_t)1 << 30 || n_atoms_max * (int64_t)p->max_nb > ((int64_t)1 << 40))
    return APIP_ERR_ARG;
  const int64_t nb = basis_size(p->ace_n_max, p->ace_l_max, p->ace_nu_max);
  if (nb != p->ace_n_basis) return APIP_ERR_ARG;
  apip_ctx* ctx = new (std::nothrow) apip_ctx();
  if (!ctx) return APIP_ERR_ARG;
  ctx->p = *p;
  ctx->ace_c1.assign(p->ace_c1, p->ace_c1 + nb);
  ctx->ace_c2.assign(p->ace_c2, p->ace_c2 + nb);
  ctx->p.ace_c1 = nullptr;
  ctx->p.ace_c2 = nullptr;
  ctx->nmax = n_atoms_max;
  ctx->r_list = std::max(std::max(p->eam_rc, p->ace_rc), p->sw_r_w) + p->skin;
  // body order <= 3: streamed couplings; body order 4: the coupling pool
  const bool streamed = p->ace_nu_max <= 3;
  HostAce tab;
  HostStream st;
  if (streamed ? !build_streamed(p->ace_n_max, p->ace_l_max, p->ace_nu_max, ctx->ace_c1.data(), ctx->ace_c2.data(),
                                 nb, &st, &why)
               : !build_coupled(p->ace_n_max, p->ace_l_max, p->ace_nu_max, ctx->ace_c1.data(), ctx->ace_c2.data(),
                                nb, &tab, &why)) {
    delete ctx;
    return APIP_ERR_ARG;
  }
  if (streamed ? !validate_streamed(st, p->ace_n_max * (p->ace_l_max + 1) * (p->ace_l_max + 1), &why)
               : !validate_coupled(tab, &why)) {
    delete ctx;
    return APIP_ERR_ARG;
  }
  ctx->ace_kind = streamed ? kAceStreamed : kAcePool;
  const int nA = p->ace_n_max * (p->ace_l_max + 1) * (p->ace_l_max + 1);
  auto fail_create = [&](cudaError_t e) {
    free_all(ctx);
    delete ctx;
    (void)e;
    return APIP_ERR_CUDA;
  };
#define APIP_ALLOC(ptr, bytes)                                 \
  do {                                                         \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));      \
    if (e_ != cudaSuccess) return fail_create(e_);             \
  } while (0)
  cudaGetDevice(&ctx->dev);
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->dev);
  // atoms per ACE block.  Pool kernel: the largest group whose pools leave room
  // for two resident blocks per SM, else the largest that fits.  Streamed
  // kernel: 8 atoms per block for the adaptive switches (a few thousand
  // compacted atoms fill the resident blocks in one round; 4 per block took two
  // rounds and 28 % longer on the 249 k-atom void crystal), 32 for constant lam
  // (every atom compacted).
  {
    const bool f32 = p->precision == APIP_FP32;
    auto occ_of = [&](int g) {
      if (f32) {
        AceDev<float> t{};
        t.kind = ctx->ace_kind; t.l_max = p->ace_l_max; t.nA = nA; t.npool = tab.npool; t.group = g;
        return streamed ? ace_stream_occupancy<float>(t) : ace_pool_occupancy<float>(t);
      }
      AceDev<double> t{};
      t.kind = ctx->ace_kind; t.l_max = p->ace_l_max; t.nA = nA; t.npool = tab.npool; t.group = g;
      return streamed ? ace_stream_occupancy<double>(t) : ace_pool_occupancy<double>(t);
    };
    int group = p->ace_group, occ = 0;
    if (group != 0) {
      occ = occ_of(group);   // 0 for a group the kernel does not provide
    } else if (streamed) {
      const bool adaptive = p->lam_mode == APIP_LAM_PAPER || p->lam_mode == APIP_LAM_LEARNED;
      const int order_a[3] = {8, 4, 32}, order_c[3] = {32, 8, 4};
      for (int q = 0; q < 3 && occ == 0; ++q) {
        group = adaptive ? order_a[q] : order_c[q];
        occ = occ_of(group);
      }
    } else {
      for (int g : {8, 4, 2, 1}) {
        const int o = occ_of(g);
        if (o >= 2 || (o >= 1 && g == 1)) { group = g; occ = o; break; }
      }
      if (occ == 0)
        for (int g : {8, 4, 2, 1})
          if ((occ = occ_of(g)) >= 1) { group = g; break; }
    }
    cudaGetLastError();
    if (occ < 1) {
      delete ctx;
      return APIP_ERR_ARG;
    }
    ctx->ace_group = group;
    ctx->ace_blocks = std::max(1, sms) * occ;
  }
  const size_t N = (size_t)n_atoms_max;
  const size_t es = esize(ctx);
  APIP_ALLOC(ctx->nnb, sizeof(int) * N);
  APIP_ALLOC(ctx->nnb_e, sizeof(int) * N);
  APIP_ALLOC(ctx->nbl, sizeof(int) * N * p->max_nb);
  APIP_ALLOC(ctx->nbl_tmp, sizeof(int) * N * p->max_nb);
  APIP_ALLOC(ctx->pos_ref, sizeof(double) * 3 * N);
  if (p->precision == APIP_FP32) {
    APIP_ALLOC(ctx->nnb_0, sizeof(int) * N);
    APIP_ALLOC(ctx->mind1, sizeof(float) * N);
    APIP_ALLOC(ctx->posq, sizeof(uint4) * N);
    APIP_ALLOC(ctx->posq_ref, sizeof(uint4) * N);
    APIP_ALLOC(ctx->posg, sizeof(uint4) * N);
  }
  APIP_ALLOC(ctx->id2idx, sizeof(int) * N);
  APIP_ALLOC(ctx->csp, sizeof(int) * N * kCspCap);
  APIP_ALLOC(ctx->csp_idx, sizeof(int) * N * kCspCap);
  APIP_ALLOC(ctx->csp_owner, sizeof(int) * N);
  void** per_atom[] = {&ctx->zeta, &ctx->xi_p, &ctx->e_eam, &ctx->g, &ctx->wbar, &ctx->dd, &ctx->lam, &ctx->dlam, &ctx->e_ace};
  for (void** q : per_atom) APIP_ALLOC(*q, es * N);
  APIP_ALLOC(ctx->cvec, sizeof(double) * N);
  APIP_ALLOC(ctx->ace_list, sizeof(int) * N);
  if (p->lam_mode == APIP_LAM_LEARNED) APIP_ALLOC(ctx->clist, sizeof(int) * N);
  APIP_ALLOC(ctx->counts, sizeof(int) * 4);
  ctx->det = p->deterministic != 0;
  if (ctx->det) APIP_ALLOC(ctx->blk_cnt, sizeof(int) * nblk(N));
  APIP_ALLOC(ctx->flags, sizeof(int) * 4);
  APIP_ALLOC(ctx->status, sizeof(int) * ST_COUNT);
  // pass-1 partials: the most blocks either pass 1 launches (the learned one has
  // smaller blocks)
  const int p1 = (int)std::max<int64_t>(nblk(n_atoms_max), (n_atoms_max + kLearnedBlock - 1) / kLearnedBlock);
  APIP_ALLOC(ctx->partials, sizeof(double) * (p1 + ctx->ace_blocks));
  APIP_ALLOC(ctx->thermo_part, sizeof(double) * 4 * p1);
  APIP_ALLOC(ctx->e_scratch, sizeof(double) * 2);
  APIP_ALLOC(ctx->ind_acc, sizeof(double) * 3);
  APIP_ALLOC(ctx->mlp_w, es * APIP_MLP_NPARAM);
  if (p->precision == APIP_FP32) {
    APIP_ALLOC(ctx->mlp_img, mlp_img_bytes());
    ctx->learned_slots = learned_tc_slots(&ctx->learned_slots1);
    if (p->lam_mode == APIP_LAM_LEARNED) APIP_ALLOC(ctx->mlp_x0, sizeof(float) * N * APIP_MLP_IN);
    cudaGetLastError();
    if ((ctx->learned_slots < 1 || ctx->learned_slots1 < 1) && p->lam_mode == APIP_LAM_LEARNED)
      return fail_create(cudaErrorInvalidConfiguration);
  }
  // ACE tables: one buffer, sub-arrays 256-byte aligned
  const bool f32 = p->precision == APIP_FP32;
  std::vector<unsigned char> host;
  auto put = [&](int slot, const void* src, size_t bytes) {
    const size_t off = (host.size() + 255) / 256 * 256;
    host.resize(off + std::max<size_t>(bytes, 16));
    if (bytes) std::memcpy(host.data() + off, src, bytes);
    ctx->ace_off[slot] = off;
  };
  auto put_ent = [&](int slot, const std::vector<uint32_t>& key, const std::vector<double>& v) {
    if (f32) {
      std::vector<Ent<float>> r(key.size());
      for (size_t q = 0; q < key.size(); ++q) r[q] = Ent<float>{(float)v[q], key[q]};
      put(slot, r.data(), sizeof(Ent<float>) * r.size());
    } else {
      std::vector<Ent<double>> r(key.size());
      for (size_t q = 0; q < key.size(); ++q) r[q] = Ent<double>{v[q], key[q]};
      put(slot, r.data(), sizeof(Ent<double>) * r.size());
    }
  };
  auto put_rec = [&](int slot, const std::vector<uint32_t>& key, const std::vector<uint32_t>* len,
                     const std::vector<double>& k1, const std::vector<double>& k2) {
    if (f32) {
      std::vector<Rec<float>> r(key.size());
      for (size_t q = 0; q < key.size(); ++q) r[q] = Rec<float>{key[q], len ? (*len)[q] : 0u, (float)k1[q], (float)k2[q]};
      put(slot, r.data(), sizeof(Rec<float>) * r.size());
    } else {
      std::vector<Rec<double>> r(key.size());
      for (size_t q = 0; q < key.size(); ++q) r[q] = Rec<double>{key[q], len ? (*len)[q] : 0u, k1[q], k2[q]};
      put(slot, r.data(), sizeof(Rec<double>) * r.size());
    }
  };
  if (streamed) {
    put_rec(0, st.pkey, &st.plen, st.p1, st.p2);
    put(1, st.cpl.data(), sizeof(uint32_t) * st.cpl.size());
    put_rec(2, st.tkey, nullptr, st.t1, st.t2);
    {
      // the first partner record of every coupling again, indexed by the coupling,
      // so that it can be loaded together with the coupling's entry
      std::vector<uint32_t> fk;
      std::vector<double> f1, f2;
      for (size_t u = 0; u < st.cpl.size() / 4; ++u) {
        const uint32_t q = st.cpl[4 * u + 1];
        fk.push_back(st.tkey[q]);
        f1.push_back(st.t1[q]);
        f2.push_back(st.t2[q]);
      }
      put_rec(3, fk, nullptr, f1, f2);
    }
    ctx->ace_npr = (int)st.pkey.size();
    ctx->ace_ncpl = (int)(st.cpl.size() / 4);
    ctx->ace_npart = (int)st.tkey.size();
    ctx->ace_npool = 1 + nA;
    int64_t* info = ctx->ace_info;
    info[0] = 1 + nA;
    info[1] = ctx->ace_ncpl;
    info[2] = st.gaunt_products;
    info[3] = (int64_t)(st.pkey.size() + st.tkey.size());
    int64_t part_len = 0, pair_len = 0;
    for (size_t u = 0; u < st.cpl.size() / 4; ++u) {
      const int L = (int)((st.cpl[4 * u] >> 16) % 5);
      part_len += (int64_t)(st.cpl[4 * u + 2] - st.cpl[4 * u + 1]) * (2 * L + 1);
    }
    for (uint32_t l : st.plen) pair_len += l;
    info[4] = part_len + pair_len;
    // forward: 3 per Gaunt product (C), 2 per partner element + 4 per partner (two
    // channels), 2 per pair element + 4 per pair record; adjoint: 3 per product (C
    // again) + 5 per product (back onto A), 4 per partner element + 2 per partner,
    // 4 per pair element + 2 per pair record
    info[10] = 11 * st.gaunt_products + 6 * part_len + 6 * (int64_t)st.tkey.size() + 6 * pair_len +
               6 * (int64_t)st.pkey.size();
  } else {
    put(0, tab.comp.data(), sizeof(uint32_t) * tab.comp.size());
    put_ent(1, tab.gkey, tab.gval);
    put_rec(2, tab.fkey, &tab.flen, tab.f1, tab.f2);
    put(3, tab.qrow.data(), sizeof(int) * tab.qrow.size());
    put_rec(4, tab.rkey, nullptr, tab.r1, tab.r2);
    put_ent(5, tab.bkey, tab.bval);
    put(6, tab.poff.data(), sizeof(int) * tab.poff.size());
    put(7, tab.tpiece.data(), sizeof(int) * tab.tpiece.size());
    ctx->ace_nC = tab.nC;
    ctx->ace_npool = tab.npool;
    ctx->ace_nf = (int)tab.fkey.size();
    ctx->ace_npc = (int)tab.poff.size() - 1;
    int64_t* info = ctx->ace_info;
    info[0] = tab.npool;
    info[1] = tab.nC;
    for (int c = 0; c < tab.nC; ++c) info[2] += tab.comp[2 * c + 1] & 255u;
    info[3] = (int64_t)tab.fkey.size();
    for (uint32_t l : tab.flen) info[4] += l;
    for (int q = 1; q < tab.npool; ++q) info[5] += tab.qrow[4 * q + 1] - tab.qrow[4 * q];
    info[6] = (int64_t)tab.bkey.size();
    // couplings 3 per Gaunt product, basis records 2 per element + 4 each, reverse
    // rows 4 per element, C -> A entries 3 each
    info[10] = 3 * info[2] + 2 * info[4] + 4 * info[3] + 4 * info[5] + 3 * info[6];
  }
  ctx->ace_info[7] = ctx->ace_group;
  ctx->ace_info[8] = ctx->ace_blocks;
  ctx->ace_info[9] = ctx->ace_kind;
  APIP_ALLOC(ctx->ace_tab, host.size());
#undef APIP_ALLOC
  cudaError_t e = cudaMemcpy(ctx->ace_tab, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ctx->id2idx, 0xff, sizeof(int) * N);
  if (e == cudaSuccess) e = cudaMemset(ctx->csp, 0xff, sizeof(int) * N * kCspCap);
  if (e == cudaSuccess) e = cudaMemset(ctx->csp_owner, 0xff, sizeof(int) * N);
  if (e == cudaSuccess) e = cudaMemset(ctx->cvec, 0, sizeof(double) * N);
  if (e == cudaSuccess) e = cudaMemset(ctx->ind_acc, 0, sizeof(double) * 3);
  if (e == cudaSuccess) e = cudaMemset(ctx->counts, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->flags, 0xff, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(int) * ST_COUNT);
  if (e == cudaSuccess) e = cudaMemset(ctx->pos_ref, 0, sizeof(double) * 3 * N);
  if (e == cudaSuccess && ctx->posq_ref) e = cudaMemset(ctx->posq_ref, 0, sizeof(uint4) * N);
  if (e == cudaSuccess) e = cudaMemset(ctx->nnb, 0, sizeof(int) * N);
  if (e == cudaSuccess) e = cudaMemset(ctx->nnb_e, 0, sizeof(int) * N);
  if (e != cudaSuccess) return fail_create(e);
  double norms[(kLmaxCap + 1) * (kLmaxCap + 1)];
  ylm_norms(kLmaxCap, norms);
  const int nn = (kLmaxCap + 1) * (kLmaxCap + 1);
  // the harmonic norms and Gaunt values are the same for every context: constant
  // memory of the current device, (re)filled by each apip_create
  if (streamed) {
    std::vector<double> gv(kGauntTotal);
    gaunt_fill(gv.data());
    e = p->precision == APIP_FP64 ? ace_stream_set_consts<double>(norms, nn, gv.data())
                                  : ace_stream_set_consts<float>(norms, nn, gv.data());
  } else {
    e = p->precision == APIP_FP64 ? ace_pool_set_norms<double>(norms, nn) : ace_pool_set_norms<float>(norms, nn);
  }
  if (e != cudaSuccess) return fail_create(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_create(e);
  *out = ctx;
  return APIP_OK;
}

apip_status apip_destroy(apip_ctx* ctx) {
  if (!ctx) return APIP_OK;
  cudaDeviceSynchronize();
  free_all(ctx);
  delete ctx;
  return APIP_OK;
}

const char* apip_last_error(apip_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

apip_status apip_build_neighbors(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* id,
                                 int64_t n, void* stream) {
  apip_status st = check_call(ctx, pos, id, n);
  if (st != APIP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_geometry(ctx, box, s)) != APIP_OK) return st;
  if (n == 0) return APIP_OK;
  return ctx->p.precision == APIP_FP32 ? neighbors_t<float>(ctx, pos, id, (int)n, s)
                                       : neighbors_t<double>(ctx, pos, id, (int)n, s);
}

apip_status apip_init_csp_pairs(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* id,
                                int64_t n, void* stream) {
  apip_status st = apip_build_neighbors(ctx, pos, box, id, n, stream);
  if (st != APIP_OK) return st;
  if (n == 0) { ctx->csp_ready = true; return APIP_OK; }
  Args<double> a = make_args<double>(ctx, pos, id, (int)n, nullptr, nullptr);
  launch_csp_init(a, (cudaStream_t)stream);
  // new partner rows: the cached partner indices are looked up again
  cudaMemsetAsync(ctx->csp_owner, 0xff, sizeof(int) * ctx->nmax, (cudaStream_t)stream);
  st = launch_status(ctx);
  if (st == APIP_OK) ctx->csp_ready = true;
  return st;
}

apip_status apip_set_csp_pairs(apip_ctx* ctx, const int32_t* partner_ids, int64_t n, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  if (n < 0 || n > ctx->nmax) return fail(ctx, APIP_ERR_ARG, "n must be in [0, n_atoms_max]");
  if (n > 0 && !partner_ids) return fail(ctx, APIP_ERR_ARG, "partner_ids must not be NULL");
  if (n > 0) launch_set_csp(partner_ids, ctx->csp, (int)n, ctx->p.csp_nnb, (cudaStream_t)stream);
  cudaMemsetAsync(ctx->csp_owner, 0xff, sizeof(int) * ctx->nmax, (cudaStream_t)stream);
  const apip_status st = launch_status(ctx);
  if (st == APIP_OK) ctx->csp_ready = true;
  return st;
}

apip_status apip_switch(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* type,
                        const int32_t* id, int64_t n, double* lam_out, double* dlam_out, int64_t* n_ace_out,
                        void* stream) {
  (void)type;
  apip_status st = check_call(ctx, pos, id, n);
  if (st != APIP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_geometry(ctx, box, s)) != APIP_OK) return st;
  if ((st = ready(ctx)) != APIP_OK) return st;
  if (n == 0) {
    if (n_ace_out) cudaMemsetAsync(n_ace_out, 0, sizeof(int64_t), s);
    return launch_status(ctx);
  }
  return ctx->p.precision == APIP_FP32 ? switch_t<float>(ctx, pos, id, (int)n, lam_out, dlam_out, n_ace_out, s)
                                       : switch_t<double>(ctx, pos, id, (int)n, lam_out, dlam_out, n_ace_out, s);
}

apip_status apip_energy_forces(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* type,
                               const int32_t* id, int64_t n, double* force_out, double* e_atom_out,
                               double* e_total_out, void* stream) {
  (void)type;
  apip_status st = check_call(ctx, pos, id, n);
  if (st != APIP_OK) return st;
  if (n > 0 && !force_out) return fail(ctx, APIP_ERR_ARG, "force_out must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_geometry(ctx, box, s)) != APIP_OK) return st;
  if ((st = ready(ctx)) != APIP_OK) return st;
  if (n == 0) {
    if (e_total_out) cudaMemsetAsync(e_total_out, 0, sizeof(double), s);
    return launch_status(ctx);
  }
  return ctx->p.precision == APIP_FP32
             ? energy_forces_t<float>(ctx, pos, id, (int)n, force_out, e_atom_out, e_total_out, s)
             : energy_forces_t<double>(ctx, pos, id, (int)n, force_out, e_atom_out, e_total_out, s);
}

apip_status apip_verlet_step(apip_ctx* ctx, double* pos, double* vel, double* force, const double* inv_mass,
                             const double box[3], const int32_t* type, const int32_t* id, int64_t n, double dt,
                             int32_t n_steps, double* thermo_out, void* stream) {
  (void)type;
  apip_status st = check_call(ctx, pos, id, n);
  if (st != APIP_OK) return st;
  if (n > 0 && (!vel || !force || !inv_mass)) return fail(ctx, APIP_ERR_ARG, "vel, force, inv_mass must not be NULL");
  if (n_steps < 0 || !std::isfinite(dt)) return fail(ctx, APIP_ERR_ARG, "n_steps must be >= 0 and dt finite");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_geometry(ctx, box, s)) != APIP_OK) return st;
  if ((st = ready(ctx)) != APIP_OK) return st;
  if (n == 0 || n_steps == 0) return launch_status(ctx);
  return ctx->p.precision == APIP_FP32
             ? verlet_t<float>(ctx, pos, vel, force, inv_mass, id, (int)n, dt, n_steps, thermo_out, s)
             : verlet_t<double>(ctx, pos, vel, force, inv_mass, id, (int)n, dt, n_steps, thermo_out, s);
}

apip_status apip_sync(apip_ctx* ctx, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  APIP_CK(cudaStreamSynchronize((cudaStream_t)stream));
  int st[ST_COUNT];
  APIP_CK(cudaMemcpy(st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost));
  APIP_CK(cudaMemset(ctx->status, 0, sizeof(st)));
  if (st[ST_BOUNDS]) {
    static const char* const site[] = {"?", "neighbour-list entry", "neighbour-list length", "cell index or member",
                                       "compacted-list entry", "ACE table key or range", "self-test"};
    const int k = st[ST_BOUNDS] >= 1 && st[ST_BOUNDS] <= BND_SELFTEST ? st[ST_BOUNDS] : 0;
    return fail(ctx, APIP_ERR_BOUNDS, std::string("bounds check: ") + site[k] + " " + std::to_string(st[ST_BOUNDS_VAL]) +
                                          " outside [0, " + std::to_string(st[ST_BOUNDS_LIM]) + ")");
  }
  if (st[ST_NB_OVERFLOW])
    return fail(ctx, APIP_ERR_NB_OVERFLOW, "neighbour list overflow: an atom has " + std::to_string(st[ST_MAX_NNB]) +
                                              " neighbours, max_nb = " + std::to_string(ctx->p.max_nb));
  if (st[ST_CELL_OVERFLOW])
    return fail(ctx, APIP_ERR_NB_OVERFLOW, "cell overflow: a cell holds " + std::to_string(st[ST_MAX_CELL]) +
                                              " atoms, cell_cap = " + std::to_string(ctx->p.cell_cap));
  if (st[ST_TIMEOUT])
    return fail(ctx, APIP_ERR_TIMEOUT,
                "a bounded device wait gave up (a tensor-core kernel's wait for its matrix products: training or the "
                "learned switch)");
  if (st[ST_BAD_INPUT]) return fail(ctx, APIP_ERR_BAD_INPUT, "non-finite position or atom id out of range");
  if (st[ST_BAD_PARTNER]) return fail(ctx, APIP_ERR_BAD_INPUT, "a CSP partner id is not present");
  return APIP_OK;
}

apip_status apip_set_mlp(apip_ctx* ctx, const float* params, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  if (!params) return fail(ctx, APIP_ERR_ARG, "params must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (ctx->p.precision == APIP_FP32) {
    launch_cast_params<float>(params, as<float>(ctx->mlp_w), s);
    launch_mlp_images(as<float>(ctx->mlp_w), ctx->mlp_img, s);
  }
  else launch_cast_params<double>(params, as<double>(ctx->mlp_w), s);
  const apip_status st = launch_status(ctx);
  if (st == APIP_OK) ctx->mlp_ready = true;
  return st;
}

apip_status apip_descriptors(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* id,
                             int64_t n, uint16_t* desc_bf16, void* stream) {
  apip_status st = check_call(ctx, pos, id, n);
  if (st != APIP_OK) return st;
  if (n > 0 && !desc_bf16) return fail(ctx, APIP_ERR_ARG, "desc_bf16 must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_geometry(ctx, box, s)) != APIP_OK) return st;
  if (n == 0) return APIP_OK;
  if (ctx->p.precision == APIP_FP32) {
    Args<float> a = make_args<float>(ctx, pos, id, (int)n, nullptr, nullptr);
    set_view<float>(a, ctx);
    mark_atom_count(ctx, (int)n, s);
    launch_prep<float>(a, s);
    launch_neighbors<float>(a, ctx->ncell, s);
    launch_descriptors<float>(a, desc_bf16, s);
  } else {
    Args<double> a = make_args<double>(ctx, pos, id, (int)n, nullptr, nullptr);
    set_view<double>(a, ctx);
    mark_atom_count(ctx, (int)n, s);
    launch_prep<double>(a, s);
    launch_neighbors<double>(a, ctx->ncell, s);
    launch_descriptors<double>(a, desc_bf16, s);
  }
  APIP_CK(cudaMemsetAsync(ctx->cell_count, 0, sizeof(int) * ctx->ncell, s));
  APIP_CK(cudaMemsetAsync(ctx->flags, 0, sizeof(int), s));
  return launch_status(ctx);
}

apip_status apip_mlp_loss_grad(apip_ctx* ctx, const uint16_t* desc_bf16, const float* y, int64_t batch,
                               const float* params, float* grad_out, float* loss_out, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  if (batch < 1 || batch > (1 << 26) || !desc_bf16 || !y || !params || !grad_out || !loss_out)
    return fail(ctx, APIP_ERR_ARG, "bad batch or NULL pointer");
  const size_t need = mlp_workspace_floats((int)batch);
  if (need > ctx->mlp_ws_cap) {
    if (ctx->mlp_ws) cudaFree(ctx->mlp_ws);
    ctx->mlp_ws = nullptr;
    ctx->mlp_ws_cap = 0;
    APIP_CK(cudaMalloc(&ctx->mlp_ws, sizeof(float) * need));
    ctx->mlp_ws_cap = need;
  }
  if (!launch_mlp_loss_grad(desc_bf16, y, (int)batch, params, grad_out, loss_out, ctx->mlp_ws, ctx->status,
                            (cudaStream_t)stream))
    return fail(ctx, APIP_ERR_ARG, "desc_bf16 not 16-byte aligned, or no TMA descriptor for it");
  return launch_status(ctx);
}

apip_status apip_mlp_adam(apip_ctx* ctx, float* params, const float* grad, float* m, float* v, int32_t t,
                          float lr, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  if (!params || !grad || !m || !v || t < 1) return fail(ctx, APIP_ERR_ARG, "NULL pointer or t < 1");
  launch_mlp_adam(params, grad, m, v, t, lr, (cudaStream_t)stream);
  return launch_status(ctx);
}

apip_status apip_profile(apip_ctx* ctx, int32_t enable) {
  if (!ctx) return APIP_ERR_ARG;
  ctx->prof = enable != 0;
  return APIP_OK;
}

apip_status apip_profile_read(apip_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx || !ms || !launches) return APIP_ERR_ARG;
  for (auto& r : ctx->prof_pending) {
    APIP_CK(cudaEventSynchronize(r.b));
    float t = 0.f;
    APIP_CK(cudaEventElapsedTime(&t, r.a, r.b));
    ctx->prof_ms[r.phase] += t;
    ctx->prof_n[r.phase] += r.launches;
    ctx->prof_pool.push_back(r.a);
    ctx->prof_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
  for (int k = 0; k < APIP_PHASE_COUNT; ++k) {
    ms[k] = ctx->prof_ms[k];
    launches[k] = ctx->prof_n[k];
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  return APIP_OK;
}

apip_status apip_set_indenter(apip_ctx* ctx, const double center[3], const double velocity[3], double radius,
                              double k) {
  if (!ctx) return APIP_ERR_ARG;
  if (radius > 0.0) {
    if (!center || !velocity) return fail(ctx, APIP_ERR_ARG, "center and velocity must not be NULL");
    if (!(k > 0.0)) return fail(ctx, APIP_ERR_ARG, "the indenter stiffness must be > 0");
    for (int q = 0; q < 3; ++q) {
      if (!std::isfinite(center[q]) || !std::isfinite(velocity[q]))
        return fail(ctx, APIP_ERR_ARG, "non-finite indenter centre or velocity");
      ctx->ind_c[q] = center[q];
      ctx->ind_v[q] = velocity[q];
    }
  }
  ctx->ind_on = radius > 0.0;
  ctx->ind_R = radius > 0.0 ? radius : 0.0;
  ctx->ind_K = k;
  APIP_CK(cudaMemset(ctx->ind_acc, 0, sizeof(double) * 3));
  return APIP_OK;
}

apip_status apip_indenter_state(apip_ctx* ctx, double center[3], double* work) {
  if (!ctx || !center || !work) return APIP_ERR_ARG;
  APIP_CK(cudaDeviceSynchronize());
  double acc[3];
  APIP_CK(cudaMemcpy(acc, ctx->ind_acc, sizeof(acc), cudaMemcpyDeviceToHost));
  for (int q = 0; q < 3; ++q) center[q] = ctx->ind_c[q];
  *work = acc[0];
  return APIP_OK;
}

apip_status apip_set_lam_fixed(apip_ctx* ctx, const double* lam_fixed, int64_t n) {
  if (!ctx) return APIP_ERR_ARG;
  if (lam_fixed && (n < 0 || n > ctx->nmax)) return fail(ctx, APIP_ERR_ARG, "n must be in [0, n_atoms_max]");
  ctx->lam_fixed = lam_fixed;
  ctx->lam_fixed_n = lam_fixed ? n : 0;
  return APIP_OK;
}

apip_status apip_ace_info(apip_ctx* ctx, int64_t* out) {
  if (!ctx || !out) return APIP_ERR_ARG;
  for (int k = 0; k < APIP_ACE_INFO_COUNT; ++k) out[k] = ctx->ace_info[k];
  return APIP_OK;
}

apip_status apip_get_field(apip_ctx* ctx, int32_t field, void* dst, int64_t n, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  if (!dst || n < 0 || n > ctx->nmax) return fail(ctx, APIP_ERR_ARG, "bad dst or n");
  if (field < APIP_FIELD_G || field > APIP_FIELD_BUILD_POS) return fail(ctx, APIP_ERR_ARG, "unknown field");
  if (n == 0) return APIP_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (ctx->p.precision == APIP_FP32) {
    Args<float> a = make_args<float>(ctx, nullptr, nullptr, (int)n, nullptr, nullptr);
    launch_get_field<float>(a, field, dst, s);
  } else {
    Args<double> a = make_args<double>(ctx, nullptr, nullptr, (int)n, nullptr, nullptr);
    launch_get_field<double>(a, field, dst, s);
  }
  return launch_status(ctx);
}

#ifdef APIP_CHECK_BOUNDS
namespace {
__global__ void k_bounds_selftest(int* status) {
  // an out-of-range index that touches no memory: 7 against the limit 5
  if (threadIdx.x == 0) (void)APIP_CHK(status, BND_SELFTEST, 7, 5);
}
}  // namespace

// Exported only by the bounds-checked build: records a violation through the
// device check (no memory is accessed with the bad index), so that the next
// apip_sync reports APIP_ERR_BOUNDS.
apip_status apip_check_bounds_selftest(apip_ctx* ctx, void* stream) {
  if (!ctx) return APIP_ERR_ARG;
  k_bounds_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->status);
  return launch_status(ctx);
}
#endif

}  // extern "C"
