// Kernel argument block and launch wrappers of libapip (internal).
#pragma once

#include <cuda_runtime.h>

#include "apip_internal.h"
#include "device_common.cuh"

namespace apip {

// The model parameters the per-atom passes use, converted (and squared) once on
// the host in the path precision: float64 arithmetic is slow on this GPU, so no
// kernel converts parameters per thread.
template <typename T>
struct PassK {
  T eam_A, eam_beta, eam_re, eam_D, eam_alpha, eam_r0, eam_rc, eam_rc2, eam_rc_lo, eam_inv_w;
  T sw_r_w, sw_r_w2, sw_r_w_lo, sw_inv_w, sw_d_lo, sw_d_hi, sw_inv_d, sw_d0;
  T prec_shift;   // energy zero of the precise model (subtracted from E^prec per atom)
};

// Float-float constants of the float32 switch refinement: the grid unit L / 2^32
// per axis, r_w + r_w_lo, and the float bounds of the taper.
struct SwFF {
  float u_hi[3], u_lo[3];
  float c_hi, c_lo, inv_w, rw2, rw_lo2;
};

// Everything a kernel of the force pipeline may need, passed by value.
template <typename T>
struct Args {
  int n, nmax, max_nb, cell_cap, csp_nnb;
  int lam_mode, precise_adds_eam, grad_lambda;
  int eam_force;          // pass 2 computes the (unweighted) EAM force
  int force_mix;          // force mixing (Eq. 3) instead of the AP force (Eq. 5)
  const double* lam_fixed;  // per-atom constant lam (NaN = switch) or null
  // spherical indenter (external potential), ind_on = 0 when absent
  int ind_on;
  double ind_c[3];        // centre (FP64 path)
  uint4 ind_q;            // centre as fixed-point coordinates (FP32 path)
  T ind_R2;               // R^2 in the path precision (the float32 path's contact test)
  double ind_Rd, ind_Kd;  // radius and stiffness
  double ind_v[3];        // centre velocity
  double* ind_acc;        // [3] device: work W, (sum F).v of the previous and of this evaluation
  PosView<T> pv;
  Geo geo;
  EamP eam;
  SwP sw;
  SwFF swff;
  PassK<T> k;
  double r_list2, skin_half2, csp_rcut2;
  float skin_half2_f;     // skin_half2 rounded down to float (the FP32 path's rebuild trigger)
  double r_e_in2, r_e_mid2;   // list-order bounds: eam_rc^2, (eam_rc + skin + margin)^2

  const double* pos;      // caller positions [n][3]
  const int* id;          // caller ids [n]
  int* nnb; int* nbl; int* nbl_tmp; double* pos_ref; uint4* posq; uint4* posq_ref; int* id2idx; int* csp;
  int* csp_idx; int* csp_owner;   // CSP^list partner indices by atom index (cache), the id each row is for
  int* nnb_e;             // entries of the list whose build-time distance is below eam_rc + skin
  int* nnb_0;             // FP32 path: entries whose build-time distance is below eam_rc
  float* mind1;           // FP32 path: least squared build-time distance of the entries in [eam_rc, eam_rc + skin)
  uint4* posg;            // FP32 path: (posq.x, posq.y, posq.z, bits of g), written by pass 1
  int* cell_count; int* cell_atoms;   // binning counts (zero outside a build) and members
  int ncell;
  uint4* cell_q;          // FP32 path: fixed-point positions of the cell members, cell order
  T* zeta; T* xi_p; T* e_eam; T* g; T* wbar; T* dd; T* lam; T* dlam; T* e_ace;
  double* cvec; int* ace_list; int* counts; int* flags; int* status;
  int det;                // deterministic mode: fixed-point scatter sums, index-ordered compaction
  int* blk_cnt;           // deterministic mode: pass 2's per-block counts, then offsets
  int* clist;             // learned switch: the atoms with cvec != 0 (counts[1] of them)
  double* partials; int n_part_p1;
  double* force;          // caller force [n][3]
  double* e_atom;         // caller per-atom energy [n] or null
  const T* mlp_w;         // learned indicator weights (APIP_MLP_NPARAM, layout of apip.h)
  const uint4* mlp_img;   // FP32 path: the weights as split bfloat16 tensor-core operand images
  float* mlp_x0;          // FP32 path: the network inputs x0 = G / 4 of every atom [nmax][32]
  int learned_grid;       // FP32 path: persistent CTAs of the tensor-core learned force kernel
  int learned_grid1;      // FP32 path: persistent CTAs of the tensor-core network of pass 1
  T ace_rc, ace_rc_lo;    // cutoff of the radial descriptors (the ACE cutoff)
};

// Scattered sums (forces, the grad-lambda c-vector, the indenter work).  In
// deterministic mode a contribution v is rounded to a multiple of 2^-40 and added
// as a 64-bit integer into the same 8 bytes: integer addition is associative, so
// the sum does not depend on the order in which the atomics arrive.  fix_get
// reads such a slot back as float64, fix_put gives the bits of a plain value in
// that form.  Otherwise the slot holds a float64 and takes float64 atomic adds.
constexpr double kFixOne = 1099511627776.0;          // 2^40
constexpr double kFixUnit = 1.0 / 1099511627776.0;   // 2^-40
__device__ __forceinline__ void scatter_add(double* p, double v, int det) {
  if (det) atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double2ll_rn(v * kFixOne));
  else atomicAdd(p, v);
}
__device__ __forceinline__ double fix_get(const double* p, int det) {
  const double v = *p;
  return det ? (double)__double_as_longlong(v) * kFixUnit : v;
}
__device__ __forceinline__ double fix_put(double v, int det) {
  return det ? __longlong_as_double(__double2ll_rn(v * kFixOne)) : v;
}

// Bounds-checked build (APIP_CHECK_BOUNDS): an index v outside [0, lim) is
// recorded (the first violation's site, index and limit go to the status words,
// reported by apip_sync as APIP_ERR_BOUNDS) and replaced by 0, so that no access
// leaves its array.  In the normal build the check is the index itself.
#ifdef APIP_CHECK_BOUNDS
static __device__ __noinline__ void bounds_violation(int* status, int site, int v, int lim) {
  if (atomicCAS(&status[ST_BOUNDS], 0, site) == 0) {
    status[ST_BOUNDS_VAL] = v;
    status[ST_BOUNDS_LIM] = lim;
  }
}
__device__ __forceinline__ int bounds_check(int* status, int site, int v, int lim) {
  if ((unsigned)v < (unsigned)lim) return v;
  bounds_violation(status, site, v, lim);
  return 0;
}
#define APIP_CHK(status, site, v, lim) ::apip::bounds_check((status), (site), (v), (lim))
#else
#define APIP_CHK(status, site, v, lim) (v)
#endif

// Ends a call's use of the list-build trigger, by one whole block, after every
// kernel that reads the trigger or the binning counts has completed: after a
// build (trigger set) the counts are cleared for the next build, then the
// trigger.
__device__ __forceinline__ void end_list_build(int* flags, int* cell_count, int ncell) {
  const int built = flags[0];
  __syncthreads();
  if (built)
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) cell_count[c] = 0;
  if (threadIdx.x == 0) flags[0] = 0;
}

// Entries [s0, s1) of atom i's neighbour list (column-major, stride nmax) with
// the index fetched two entries and the neighbour's record (load(j)) one entry
// ahead of the arithmetic f(j, record), so that the gathers of the next entries
// are in flight while the current one is evaluated.
// (status, n: the bounds-checked build's check of each index against [0, n).)
template <typename L, typename F>
__device__ __forceinline__ void walk_list(const int* nb, int nmax, int s0, int s1, int* status, int n, L&& load,
                                          F&& f) {
  (void)status;
  (void)n;
  if (s0 >= s1) return;
  int j = APIP_CHK(status, BND_NEIGHBOUR, nb[(size_t)s0 * nmax], n);
  auto r = load(j);
  int jn = s0 + 1 < s1 ? APIP_CHK(status, BND_NEIGHBOUR, nb[(size_t)(s0 + 1) * nmax], n) : j;
  for (int s = s0; s < s1; ++s) {
    const int jc = j;
    const auto rc = r;
    j = jn;
    r = load(j);
    jn = s + 2 < s1 ? APIP_CHK(status, BND_NEIGHBOUR, nb[(size_t)(s + 2) * nmax], n) : j;
    f(jc, rc);
  }
}

// EAM density and pair terms of one neighbour at distance r < rc (Eq. B1, S7-S8):
// rho(r) = A exp(-beta (r - r_e)) fc(r), Phi(r) = D [x^2 - 2x] fc(r), x = exp(-alpha (r - r_0)).
template <typename T>
__device__ __forceinline__ void eam_terms(const PassK<T>& k, T r, T* rho, T* phi) {
  T dfc;
  const T fc = ftrans(r, k.eam_rc_lo, k.eam_rc, k.eam_inv_w, &dfc);
  const T x = fexp(-k.eam_alpha * (r - k.eam_r0));
  *rho = k.eam_A * fexp(-k.eam_beta * (r - k.eam_re)) * fc;
  *phi = k.eam_D * (x * x - T(2) * x) * fc;
}

// The spherical indenter's term for atom i: for r = |x_i - c| < R, the energy
// K/3 (R - r)^3 and the force K (R - r)^2 (x_i - c)/r; returns false (and leaves
// the outputs) outside the sphere.  In float64 in both paths: the gap R - r is a
// small difference of numbers near R (40 A), which float32 would carry to ~1e-5 A.
// The float32 path tests the sphere on float distances first, so that only the
// few atoms in contact reach the float64 arithmetic; it takes the separation from
// the exact fixed-point difference.
template <typename T>
__device__ __forceinline__ bool ind_term(const Args<T>& a, int i, double* e, double f[3]) {
  double d[3];
  if constexpr (sizeof(T) == 4) {
    const uint4 q = a.posq[i];
    const int di[3] = {(int)(q.x - a.ind_q.x), (int)(q.y - a.ind_q.y), (int)(q.z - a.ind_q.z)};
    const float fx = (float)di[0] * a.pv.unit[0], fy = (float)di[1] * a.pv.unit[1], fz = (float)di[2] * a.pv.unit[2];
    if (!(fx * fx + fy * fy + fz * fz < a.ind_R2 * 1.0001f)) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = (double)di[k] * (a.geo.L[k] * 0x1p-32);
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      d[k] = a.pos[3 * i + k] - a.ind_c[k];
      d[k] -= a.geo.L[k] * rint(d[k] * a.geo.invL[k]);
    }
  }
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  if (!(r2 < a.ind_Rd * a.ind_Rd) || !(r2 > 0.0)) return false;
  const double r = sqrt(r2), gap = a.ind_Rd - r;
  *e = a.ind_Kd / 3.0 * gap * gap * gap;
  const double sc = a.ind_Kd * gap * gap / r;
#pragma unroll
  for (int k = 0; k < 3; ++k) f[k] = sc * d[k];
  return true;
}

// Indenter energy K/3 (R - r)^3 of atom i (zero outside the sphere or without one).
template <typename T>
__device__ __forceinline__ double ind_energy(const Args<T>& a, int i) {
  if (!a.ind_on) return 0.0;
  double e, f[3];
  return ind_term(a, i, &e, f) ? e : 0.0;
}

// Launch with programmatic stream serialization (the kernel must start with
// pdl_begin()).
template <typename... KArgs, typename... Act>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Act&&>(args)...);
}

template <typename T> Args<T> make_args(apip_ctx* c, const double* pos, const int* id, int n,
                                        double* force, double* e_atom);

// all-atom passes (kernels_atoms.cu)
template <typename T> void launch_prep(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_neighbors(const Args<T>& a, int ncell, cudaStream_t s);
void launch_csp_init(const Args<double>& a, cudaStream_t s);
void launch_set_csp(const int32_t* src, int* dst, int n, int nnb, cudaStream_t s);
template <typename T> void launch_pass1(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_pass2(const Args<T>& a, cudaStream_t s);
// force mixing: append to the compacted list every atom with lam = 0 that has a
// neighbour within the ACE cutoff with lam > 0 (the precise model's buffer)
template <typename T> void launch_fm_buffer(const Args<T>& a, cudaStream_t s);
// indenter work: W += dt/2 ((sum F).v old + new) when dt > 0; then old = new, new = 0
void launch_ind_work(double* acc, double dt, int det, cudaStream_t s);
void launch_fix_finish(double* force, int n, cudaStream_t s);
template <typename T> void launch_csp_force(const Args<T>& a, cudaStream_t s);
void launch_final(double* partials, int n_part, double* e_total, double* e_pot_slot,
                  const double* thermo_part, int n_tblocks, double* thermo_slot, int* flags,
                  const int* counts, int64_t* n_ace_out, int* cell_count, int ncell, cudaStream_t s);
template <typename T> void launch_get_field(const Args<T>& a, int field, void* dst, cudaStream_t s);
void launch_fill_const_list(int* list, int* counts, int n, cudaStream_t s);

// velocity Verlet (kernels_atoms.cu); mode 0 = first (kick, drift), 1 = mid
// (kick, thermo partials, kick, drift), 2 = last (kick, thermo partials)
template <typename T> void launch_verlet(const Args<T>& a, int mode, double* pos, double* vel,
                                         const double* force, const double* inv_mass, double dt,
                                         double* thermo_part, cudaStream_t s);
void launch_thermo_final(const double* thermo_part, int n_tblocks, double* thermo_slot, cudaStream_t s);

// learned indicator (kernels_mlp.cu)
template <typename T> void launch_pass1_learned(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_mlp_force(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_descriptors(const Args<T>& a, uint16_t* out, cudaStream_t s);
template <typename T> void launch_cast_params(const float* src, T* dst, cudaStream_t s);
// FP32 learned pass 1 on the tensor cores: resident blocks on the device, blocks
// for n atoms, the weight fragments (from the float32 weights) and their size
int learned_tc_slots(int* grid_pass1);
void launch_mlp_images(const float* w, void* img, cudaStream_t s);
size_t mlp_img_bytes();
// training on the tensor cores (kernels_train_tc.cu); a bounded wait that gives up
// sets status[ST_TIMEOUT].  False (nothing launched) when desc is not 16-byte
// aligned or its TMA descriptor cannot be made.
bool launch_mlp_loss_grad(const uint16_t* desc, const float* y, int batch, const float* params, float* grad,
                          float* loss, float* ws, int* status, cudaStream_t s);
size_t mlp_workspace_floats(int batch);
void launch_mlp_adam(float* p, const float* g, float* m, float* v, int t, float lr, cudaStream_t s);

// ACE: body order 4 (kernels_ace_f32.cu, kernels_ace_f64.cu) and body order
// <= 3 (kernels_ace3_f32.cu, kernels_ace3_f64.cu).  The occupancy queries return
// resident blocks per SM for ace.group atoms per block (0 if it does not fit).
template <typename T> cudaError_t ace_pool_set_norms(const double* norms, int count);
template <typename T> void launch_ace_pool(const Args<T>& a, const AceDev<T>& ace, int blocks, cudaStream_t s);
template <typename T> int ace_pool_occupancy(const AceDev<T>& ace);
template <typename T> cudaError_t ace_stream_set_consts(const double* norms, int count, const double* gaunt);
template <typename T> void launch_ace_stream(const Args<T>& a, const AceDev<T>& ace, int blocks, cudaStream_t s);
template <typename T> int ace_stream_occupancy(const AceDev<T>& ace);

}  // namespace apip
