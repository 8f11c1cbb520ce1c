/*
 * apip.h -- C ABI of libapip, the GB300 (sm_103a) force evaluation of the
 * conservative adaptive-precision (AP) EAM+ACE potential of arxiv 2512.07693
 * ("Conservative adaptive-precision interatomic potentials").
 *
 *   E   = sum_i [ lam_i E_i^prec + (1 - lam_i) E_i^EAM ]           (Eq. 4)
 *   F_i = -grad_i E, including the (E^prec - E^EAM) grad lam terms  (Eq. 5)
 *
 * lam is the weight of the PRECISE model (lam = 1: precise, lam = 0: fast EAM);
 * the paper's lambda (Eq. 2) is the weight of the fast model, lambda = 1 - lam.
 * The precise model is ACE, optionally on top of the EAM
 * (apip_params.precise_adds_eam: E^prec = E^ACE + E^EAM).
 *
 * Conventions for every call:
 *  - Units: Angstrom, eV, ps; inv_mass in (A/ps^2)/(eV/A), i.e. 1/(m[amu] * 1.0364269e-4).
 *  - Vectors are AoS [n][3] float64, row-major, contiguous.  Every array
 *    argument is a DEVICE pointer owned by the caller, except where a comment
 *    says "host".  The library never frees caller memory.
 *  - box: host array of the three edge lengths of an orthorhombic periodic
 *    cell.  Each edge must be >= 3 * (cutoff + skin).  Positions may lie
 *    outside [0, L); they are treated periodically.
 *  - id: int32 atom identifiers, unique, in [0, n_atoms_max).  The CSP pair
 *    list stores partner IDs, so atoms may be reordered between calls.
 *  - type: int32, single species; must be 0.
 *  - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls are asynchronous: the returned status covers argument checks and
 *    launch errors.  Errors detected on the device (neighbour overflow,
 *    non-finite input) are latched in the context and returned by the next
 *    apip_sync() (which synchronises the stream).
 *  - Not thread-safe for one context; distinct contexts are independent.
 */
#ifndef APIP_H
#define APIP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apip_ctx apip_ctx;

typedef enum {
  APIP_OK = 0,
  APIP_ERR_ARG = 1,          /* invalid argument: NULL pointer, size, parameter, box too small */
  APIP_ERR_CUDA = 2,         /* a CUDA runtime call failed (apip_last_error has the text) */
  APIP_ERR_NB_OVERFLOW = 3,  /* an atom had more neighbours than max_nb, or a cell more atoms
                                than cell_cap; apip_last_error reports the size needed */
  APIP_ERR_BAD_INPUT = 4,    /* non-finite position, id out of range, or a CSP partner ID
                                that is not present */
  APIP_ERR_STATE = 5,        /* call order: apip_init_csp_pairs must precede calls that use
                                the paper's switch */
  APIP_ERR_SIZE = 6,         /* input larger than a fixed-capacity entry point can hold */
  APIP_ERR_TIMEOUT = 7,      /* a bounded device wait gave up: the tensor-core kernels of
                                training and of the learned switch wait for their matrix
                                products with a 2 s limit; no kernel waits on another */
  APIP_ERR_BOUNDS = 8        /* only in a library compiled with APIP_CHECK_BOUNDS: an index
                                read from a device list or table fell outside its array;
                                the access went to index 0 instead and the call's results
                                are invalid.  apip_last_error names the first site, the
                                index and the limit */
} apip_status;

enum { APIP_FP64 = 0, APIP_FP32 = 1 };

/* How lam is obtained.
 * APIP_LAM_PAPER : lam_i = 1 - f_trans(d_i, d_lo, d_hi), d_i the locally averaged
 *                  CSP^list descriptor (Eq. 2, Eq. 6, Eq. B3).
 * APIP_LAM_CONST0: lam = 0 for all atoms (pure fast model).
 * APIP_LAM_CONST1: lam = 1 for all atoms (pure precise model).
 * APIP_LAM_LEARNED: the paper's switch (Eq. 2, Eq. 6) with the atomic quantity g_k
 *                  given by a small MLP on radial descriptors instead of CSP^list
 *                  (any differentiable, distance-only g_k is allowed by the paper,
 *                  main text after Eq. 5); weights from apip_set_mlp. */
enum { APIP_LAM_PAPER = 0, APIP_LAM_CONST0 = 1, APIP_LAM_CONST1 = 2, APIP_LAM_LEARNED = 3 };

/* How the two models are combined.
 * APIP_MIX_ENERGY: the conservative AP potential, E = sum_i [lam_i E_i^prec +
 *   (1 - lam_i) E_i^EAM] (Eq. 4) and F = -grad E (Eq. 5).
 * APIP_MIX_FORCE: force mixing (Eq. 3), the non-conservative comparison:
 *   F_i = (1 - lam_i) F_i^EAM + lam_i F_i^prec with F^m = -grad sum_k E_k^m; the
 *   precise model is evaluated on the atoms with lam > 0 and on every atom within
 *   the ACE cutoff of one; grad_lambda is ignored.  The energy output is Eq. 4. */
enum { APIP_MIX_ENERGY = 0, APIP_MIX_FORCE = 1 };

/* Learned indicator network: radial descriptors
 *   G_im = sum_{j, r_ij < ace_rc} exp(-eta (r_ij - mu_m)^2) fc(r_ij),  m = 0..31,
 *   mu_m = 1.5 + m (5.0 - 1.5)/31 A, eta = 1/(2 * 0.15^2) A^-2, fc the ACE cutoff function,
 * then g = w4 . h3 + b4 with h_k = silu(W_k h_{k-1} + b_k), h_0 = 0.25 G, widths
 * 32 -> 64 -> 64 -> 64 -> 1, silu(x) = x / (1 + exp(-x)).  Parameters are one flat
 * float32 array of APIP_MLP_NPARAM values in the order W1 [64][32], b1 [64],
 * W2 [64][64], b2 [64], W3 [64][64], b3 [64], w4 [64], b4 [1] (row-major). */
#define APIP_MLP_IN 32
#define APIP_MLP_WIDTH 64
#define APIP_MLP_NPARAM 10497

/* Model and run parameters; copied by apip_create.  Field order is ABI. */
typedef struct apip_params {
  int32_t precision;         /* APIP_FP64 (all arithmetic in float64) or APIP_FP32 (pair
                                arithmetic in float32 with compensated sums; positions,
                                velocities, force output and energy reductions float64) */
  int32_t lam_mode;          /* APIP_LAM_* */
  int32_t grad_lambda;       /* 1: include F^(grad lambda) (conservative, Eq. S15-S27);
                                0: drop it (the non-conservative ablation of Fig. 3b) */
  int32_t precise_adds_eam;  /* 1: E^prec = E^ACE + E^EAM; 0: E^prec = E^ACE */
  /* fast model, Eq. B1: rho(r) = A exp(-beta (r - re)) fc(r),
     Phi(r) = D [exp(-2 alpha (r - r0)) - 2 exp(-alpha (r - r0))] fc(r),
     xi(z) = -sqrt(z), fc(r) = f_trans(r, rc - rc_width, rc) */
  double eam_A, eam_beta, eam_re, eam_D, eam_alpha, eam_r0, eam_rc, eam_rc_width;
  /* precise model: ACE with Chebyshev radial basis R_n = T_{n-1}(1 - 2r/rc) fc(r),
     real Y_lm, A_nlm = a_scale sum_j R_n Y_lm, canonical product basis of body
     order <= nu_max, E = c1.B + (( c2.B )^2 + eps^2)^(1/4) - sqrt(eps).
     n_max in [1, 8], l_max in [0, 4], nu_max in [1, 4], n_max (l_max+1)^2 <= 254. */
  int32_t ace_n_max, ace_l_max, ace_nu_max;
  int32_t ace_group;         /* compacted atoms per ACE thread block, or 0 = automatic.
                                Body order <= 3 (streamed): 4, 8 or 32 (automatic: 8 for the
                                paper and learned switches, 32 for constant lam).  Body
                                order 4 (pool): 1, 2, 4 or 8 (automatic: the largest whose
                                two per-atom pools leave room for two resident blocks per
                                SM).  A group the evaluation does not provide, or whose
                                shared memory does not fit, is rejected by apip_create
                                (APIP_ERR_ARG). */
  double ace_rc, ace_rc_width, ace_eps, ace_a_scale;
  const double* ace_c1;      /* host, ace_n_basis entries (copied) */
  const double* ace_c2;      /* host, ace_n_basis entries (copied) */
  int64_t ace_n_basis;       /* must equal apip_ace_basis_size(n_max, l_max, nu_max) */
  /* switch (Eq. 2, Eq. 6, Appendix B): w(r) = f_trans(r, r_w - r_w_width, r_w) */
  double sw_r_w, sw_r_w_width, sw_d_lo, sw_d_hi, sw_d0;
  /* CSP^list pair detection (Eq. B3): csp_nnb nearest neighbours within csp_rcut */
  double csp_rcut;
  int32_t csp_nnb;           /* even, <= 8 */
  int32_t nb_pad;
  /* neighbour list: cutoff = max(eam_rc, ace_rc, sw_r_w) + skin */
  double skin;
  int32_t max_nb;            /* neighbour capacity per atom (1 .. 1024) */
  int32_t cell_cap;          /* atom capacity per cell (1 .. 1024) */
  int32_t mixing;            /* APIP_MIX_ENERGY or APIP_MIX_FORCE */
  int32_t deterministic;     /* 1: results that do not depend on the order in which the
                                device's threads run.  Each cell's members are sorted by
                                index after binning, the compacted list is written in index
                                order, and every scattered force, c-vector and indenter-work
                                contribution is rounded to a multiple of 2^-40 and summed as a
                                64-bit integer (each sum must stay below 2^23 = 8.4e6 in
                                magnitude: eV/A for forces).  Repeated runs from the same state then give
                                the same bits, and a run resumed from a checkpoint that holds
                                APIP_FIELD_BUILD_POS continues the trajectory bit for bit.
                                Costs three small kernels per call and one per list build.
                                Requires APIP_FP32 with ace_nu_max <= 3 and ace_l_max <= 3
                                (elsewhere dE/dA is summed with shared-memory atomics) and
                                APIP_MIX_ENERGY; otherwise APIP_ERR_ARG.  0: float64 atomics,
                                results reproducible to rounding */
  double prec_shift;         /* energy zero of the precise model: E^prec_i is lowered by this
                                constant (eV per atom).  0 keeps E^prec as defined above.  Set
                                to the models' difference per atom in the perfect lattice, it
                                makes E^prec - E^EAM vanish in the bulk, as for two potentials
                                fitted to the same reference energies (a constant per-atom
                                shift moves no force of either model, but it enters the
                                grad-lambda force of Eq. 5 through E^prec - E^EAM) */
} apip_params;

/* Number of product-basis functions of the canonical ACE basis (the length of
 * ace_c1 / ace_c2), or -1 for out-of-range arguments.  Enumeration order: nu = 1
 * (n, 0); nu = 2 pairs p1 <= p2 with equal l; nu = 3 triples p1 <= p2 <= p3 with
 * even l-sum and the triangle rule; nu = 4 quadruples p1 <= ... <= p4 with an
 * intermediate L coupling (12)(34); p = (n-1)(l_max+1) + l. */
int64_t apip_ace_basis_size(int32_t n_max, int32_t l_max, int32_t nu_max);

/* Create a context for up to n_atoms_max atoms.  Allocates all scratch (cells,
 * neighbour list, per-atom switch arrays, ACE tables) on the current device.
 * Errors: APIP_ERR_ARG (bad parameters, or an ACE group that does not fit in
 * shared memory), APIP_ERR_CUDA (allocation). */
apip_status apip_create(const apip_params* p, int64_t n_atoms_max, apip_ctx** out);

/* Free a context and its device memory (synchronises the device). NULL is ok. */
apip_status apip_destroy(apip_ctx* ctx);

/* Build the cell-binned neighbour list (cutoff + skin) for the n atoms at pos.
 * Normally not needed: the force calls rebuild on their own when an atom has
 * moved more than skin/2 since the last build, when the box changes, and when n
 * differs from the n of the last build (any n in [0, n_atoms_max] may be passed to
 * each call).  Paper: distances only (main text
 * after Eq. 5); the list itself is an implementation device. */
apip_status apip_build_neighbors(apip_ctx* ctx, const double* pos, const double box[3],
                                 const int32_t* id, int64_t n, void* stream);

/* Detect the CSP^list opposite-neighbour pairs once (t = 0, Appendix B, Eq. B3):
 * for each atom the csp_nnb nearest neighbours within csp_rcut (ties by ID) are
 * paired greedily by ascending |r_ia + r_ib|^2.  Partner IDs are kept for the
 * rest of the context's life, by atom ID, so the atoms may be reordered in later
 * calls. */
apip_status apip_init_csp_pairs(apip_ctx* ctx, const double* pos, const double box[3],
                                const int32_t* id, int64_t n, void* stream);

/* Restore the CSP^list partner ids of a run (Appendix B: detected once, then fixed
 * by ID), for a context that resumes it from a checkpoint instead of detecting
 * them again at the resumed configuration.  partner_ids (device, int32
 * [n][csp_nnb], caller-owned, -1 for no partner): row k holds the partners of the
 * atom whose id is k, for ids 0 .. n-1, as apip_get_field (APIP_FIELD_CSP)
 * returns them.  Copied on the stream; the paper's
 * switch may be used afterwards.  Partner ids that are not present are reported
 * by apip_sync (APIP_ERR_BAD_INPUT).  Errors: APIP_ERR_ARG (n outside
 * [0, n_atoms_max], NULL pointer), APIP_ERR_CUDA. */
apip_status apip_set_csp_pairs(apip_ctx* ctx, const int32_t* partner_ids, int64_t n, void* stream);

/* Switch only (Eq. 2, Eq. 6): writes lam (ACE weight) and dlam = d lam/d d_i for
 * every atom (float64, optional, may be NULL) and the number of atoms with lam > 0
 * (the compacted precise + transition set) to *n_ace_out (device int64, may be NULL). */
apip_status apip_switch(apip_ctx* ctx, const double* pos, const double box[3],
                        const int32_t* type, const int32_t* id, int64_t n,
                        double* lam_out, double* dlam_out, int64_t* n_ace_out, void* stream);

/* Energy and forces (Eq. 4, Eq. 5).  force_out [n][3] is overwritten with F = -grad E.
 * e_atom_out [n] (optional) receives lam_i E_i^prec + (1 - lam_i) E_i^EAM.
 * e_total_out (device scalar, optional) receives E, reduced in float64. */
apip_status apip_energy_forces(apip_ctx* ctx, const double* pos, const double box[3],
                               const int32_t* type, const int32_t* id, int64_t n,
                               double* force_out, double* e_atom_out, double* e_total_out,
                               void* stream);

/* A spherical repulsive indenter (an external potential of the indentation
 * workload, not part of the AP Hamiltonian): for r = |x_i - c| < radius,
 * E_i = k/3 (radius - r)^3 and F_i = k (radius - r)^2 (x_i - c)/r, added to E,
 * e_atom and F.  The centre (host, Angstrom) moves at velocity (host, A/ps) during
 * apip_verlet_step (by velocity * dt per step, with the drift); the work
 * W = int (sum_i F_i) . velocity dt done on the atoms accumulates on the device
 * (midpoint rule), so that H - W is conserved.  radius <= 0 removes it; every
 * call resets W to 0.  Errors: APIP_ERR_ARG. */
apip_status apip_set_indenter(apip_ctx* ctx, const double center[3], const double velocity[3], double radius,
                              double k);

/* The indenter's current centre and accumulated work W (host outputs;
 * synchronises the device).  Errors: APIP_ERR_ARG (NULL argument), APIP_ERR_CUDA. */
apip_status apip_indenter_state(apip_ctx* ctx, double center[3], double* work);

/* Constant lam on a subset of atoms (Appendix B): lam_fixed (device, float64,
 * n entries, caller-owned and kept alive while set) holds NaN for atoms whose lam
 * follows the switch and the constant value (in [0, 1]) for the others; those
 * have dlam = 0 and so no grad-lambda force of their own.  Applies to every later
 * call; NULL clears it.  Errors: APIP_ERR_ARG (n outside [0, n_atoms_max]). */
apip_status apip_set_lam_fixed(apip_ctx* ctx, const double* lam_fixed, int64_t n);

/* n_steps velocity-Verlet NVE steps (float64 state).  On entry force holds F(pos)
 * (from apip_energy_forces); on exit pos, vel, force are advanced and wrapped into
 * the box.  thermo_out (device, optional) receives per step s = 0..n_steps-1 five
 * float64 values: E_pot, E_kin = sum v^2 / (2 inv_mass), and the total momentum
 * sum v / inv_mass (x, y, z), all after the step. */
apip_status apip_verlet_step(apip_ctx* ctx, double* pos, double* vel, double* force,
                             const double* inv_mass, const double box[3],
                             const int32_t* type, const int32_t* id, int64_t n, double dt,
                             int32_t n_steps, double* thermo_out, void* stream);

/* Synchronise the stream and return the first device-side error latched since
 * the last apip_sync (APIP_OK if none); clears the latch. */
apip_status apip_sync(apip_ctx* ctx, void* stream);

/* Text of the last error of this context ("" if none). Never NULL. */
const char* apip_last_error(apip_ctx* ctx);

/* Internal per-atom arrays of the last force/switch call, for inspection and
 * testing.  Copies n entries as float64 into dst (device) unless stated:
 *   APIP_FIELD_G, _D, _WBAR, _LAM, _DLAM, _E_EAM, _E_ACE (0 unless lam > 0), _ZETA
 *   APIP_FIELD_ACE_LIST : int64 dst, the compacted atom indices with lam > 0
 *                         (unordered, in index order in the deterministic mode; only the
 *                         first count entries are defined)
 *   APIP_FIELD_NNB      : int64 dst, neighbours per atom (within cutoff + skin)
 *   APIP_FIELD_NBLIST   : int64 dst [n][max_nb], neighbour indices (-1 padded)
 *   APIP_FIELD_CSP      : int64 dst [n][csp_nnb], partner IDs (-1 = none); row k holds
 *                         the partners of the atom whose id is k
 *   APIP_FIELD_BUILD_POS: float64 dst [n][3], the positions (as the caller passed them)
 *                         from which the current neighbour list was built.  A checkpoint
 *                         that stores them rebuilds the same list with
 *                         apip_build_neighbors on resume */
enum {
  APIP_FIELD_G = 0, APIP_FIELD_D = 1, APIP_FIELD_WBAR = 2, APIP_FIELD_LAM = 3,
  APIP_FIELD_DLAM = 4, APIP_FIELD_E_EAM = 5, APIP_FIELD_E_ACE = 6, APIP_FIELD_ZETA = 7,
  APIP_FIELD_ACE_LIST = 8, APIP_FIELD_NNB = 9, APIP_FIELD_NBLIST = 10, APIP_FIELD_CSP = 11,
  APIP_FIELD_BUILD_POS = 12
};
apip_status apip_get_field(apip_ctx* ctx, int32_t field, void* dst, int64_t n, void* stream);

/* Per-phase device timing (tracing).  While enabled, every call records CUDA
 * events around its phases on the call's stream; apip_profile_read synchronises,
 * writes the accumulated device milliseconds and launch counts per phase since
 * the last read into the host arrays ms[APIP_PHASE_COUNT] and
 * launches[APIP_PHASE_COUNT], and resets them.  Phases: PREP (position
 * preparation or Verlet kernels), NEIGHBOR (the two conditional neighbour-list
 * kernels; three in the deterministic mode), PASS1, PASS2 (with the deterministic
 * mode's ordered compaction), ACE, CSP (CSP or learned part of grad-lambda, and
 * the deterministic mode's fixed-point to float64 conversion), REDUCE.
 * Independently of apip_profile, every call is an NVTX range named after it
 * ("apip_energy_forces", "apip_verlet_step", "apip_switch",
 * "apip_build_neighbors") holding one range per phase ("apip.prep",
 * "apip.neighbor", "apip.pass1", "apip.pass2", "apip.ace", "apip.csp"), which a
 * profiler attached to the process shows and by which ncu --nvtx selects
 * kernels; without an attached tool they cost a few nanoseconds per call. */
enum {
  APIP_PHASE_PREP = 0, APIP_PHASE_NEIGHBOR = 1, APIP_PHASE_PASS1 = 2, APIP_PHASE_PASS2 = 3,
  APIP_PHASE_ACE = 4, APIP_PHASE_CSP = 5, APIP_PHASE_REDUCE = 6, APIP_PHASE_COUNT = 7
};
apip_status apip_profile(apip_ctx* ctx, int32_t enable);
apip_status apip_profile_read(apip_ctx* ctx, double* ms, int64_t* launches);

/* Bounds-checked build.  Compiled with -DAPIP_CHECK_BOUNDS (the package's build
 * with checked=True writes libapip_checked.so), every index the kernels read from
 * a device list or table (neighbour entries and list lengths, cell indices and
 * members, compacted-list entries, the streamed ACE tables' keys and ranges) is
 * tested against its array before use; the first index out of range is
 * recorded, the access goes to index 0 instead, and apip_sync returns
 * APIP_ERR_BOUNDS naming the site, the index and the limit.  CSP partner indices
 * are checked against the ids in every build.  Every build checks all ACE tables
 * (streamed and pool) on the host when apip_create builds them.
 * apip_check_bounds_selftest records one violation through the device check
 * without touching memory, so that the next apip_sync reports it (a test of the
 * reporting path).  Errors: APIP_ERR_ARG (NULL ctx). */
#ifdef APIP_CHECK_BOUNDS
apip_status apip_check_bounds_selftest(apip_ctx* ctx, void* stream);
#endif

/* Sizes of the ACE evaluation that apip_create built, for work accounting
 * (host call, no device work).  Body order <= 3 uses the streamed evaluation
 * (couplings C_{(p1 p2) L M} = sum G A_{p1} A_{p2} formed in registers and
 * contracted with their nu = 3 partners), body order 4 the coupling pool (all C
 * of an atom stored, every basis function a dot product of two pool segments).
 * out (host, APIP_ACE_INFO_COUNT entries):
 *   [0] values per atom in shared memory: 1 + n_max (l_max+1)^2 (+ pool couplings)
 *   [1] couplings (streamed) or coupling components (pool)
 *   [2] Gaunt products per atom (one multiply and one multiply-add each)
 *   [3] basis records (nu = 1, 2 records and nu = 3 partners, or pool records)
 *   [4] sum over the records of their segment length
 *   [5] pool: sum over the pool values of the length of their reverse row
 *   [6] pool: C -> A back-propagation entries
 *   [7] compacted atoms per ACE thread block
 *   [8] ACE thread blocks per launch
 *   [9] evaluation: 0 = pool, 1 = streamed
 *   [10] floating-point operations per compacted atom of the table work (forward
 *        and adjoint; a multiply-add counts 2); the per-neighbour work is not
 *        included
 * Errors: APIP_ERR_ARG (NULL argument). */
#define APIP_ACE_INFO_COUNT 11
apip_status apip_ace_info(apip_ctx* ctx, int64_t* out);

/* Learned indicator (workload row: MLP on radial descriptors trained on per-atom
 * |E^prec - E^EAM|; no counterpart in the paper beyond its allowance of any
 * differentiable distance-only g_k).
 *
 * apip_set_mlp: copy the network parameters (device, float32, APIP_MLP_NPARAM)
 *   into the context; required before APIP_LAM_LEARNED calls (APIP_ERR_STATE otherwise).
 * apip_descriptors: the 32 radial descriptors of every atom as bfloat16 (round to
 *   nearest even), desc_bf16 device [n][32] (training inputs).
 * apip_mlp_loss_grad: for a batch of descriptors (bfloat16 [batch][32], rows
 *   contiguous, the start 16-byte aligned: it is read by TMA; APIP_ERR_ARG
 *   otherwise) and labels y (float32 [batch]): *loss_out = mean (g - y)^2 and
 *   grad_out[APIP_MLP_NPARAM]
 *   its gradient with respect to params (all device; bfloat16 GEMM operands,
 *   float32 accumulation).  The gradient is the same bit for bit on every call with
 *   the same inputs (no atomics: per-CTA sums added in a fixed order).  The context
 *   keeps a workspace of about 42 KiB per SM of the device, allocated on the first
 *   call.
 * apip_mlp_adam: one Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias
 *   corrected, step t >= 1) of params with grad; m and v are the moment arrays. */
apip_status apip_set_mlp(apip_ctx* ctx, const float* params, void* stream);
apip_status apip_descriptors(apip_ctx* ctx, const double* pos, const double box[3], const int32_t* id,
                             int64_t n, uint16_t* desc_bf16, void* stream);
apip_status apip_mlp_loss_grad(apip_ctx* ctx, const uint16_t* desc_bf16, const float* y, int64_t batch,
                               const float* params, float* grad_out, float* loss_out, void* stream);
apip_status apip_mlp_adam(apip_ctx* ctx, float* params, const float* grad, float* m, float* v, int32_t t,
                          float lr, void* stream);

/* Allocation-free total energy.  The paper has no counterpart: this is a service
 * for callers that cannot call cudaMalloc, such as a host program whose device
 * memory is entirely owned by its own pool allocator, or a latency-critical loop
 * that must never enter the allocator.  It needs no context.
 *
 * Sums the caller's per-atom energies e_atom[0..n) (device, float64) into
 * *e_total (device scalar) with the same compensated two-stage float64 reduction
 * that apip_energy_forces uses for e_total_out.  Its block partials are kept in
 * one fixed file-scope device array of APIP_STATIC_MAX_BLOCKS doubles (32 KiB),
 * which every GPU that loads the library holds until the process exits, so n is
 * limited to APIP_STATIC_MAX_ATOMS; larger n returns APIP_ERR_SIZE without any
 * GPU work.  The call allocates nothing: no cudaMalloc, cudaFree or allocating
 * library routine.
 *  - The first call on each device looks up the array's device address (with that
 *    device current) and caches it; make that first call before any stream capture.
 *    The cached address belongs to the device's primary context: after
 *    cudaDeviceReset (or anything else that destroys that context) it is stale,
 *    so do not call this entry point again in a process that has reset the device.
 *  - All calls share the one array.  Each call writes every partial it reads, so
 *    nothing needs clearing between calls, but calls that overlap on the GPU (on
 *    different streams, or from different host threads) race on the partials and
 *    may return wrong sums: serialise them.
 * Errors: APIP_ERR_ARG (NULL pointer, n < 0), APIP_ERR_SIZE, APIP_ERR_CUDA. */
#define APIP_STATIC_ATOMS_PER_BLOCK 4096
#define APIP_STATIC_MAX_BLOCKS 4096
#define APIP_STATIC_MAX_ATOMS ((int64_t)APIP_STATIC_ATOMS_PER_BLOCK * APIP_STATIC_MAX_BLOCKS)
apip_status apip_reduce_energy_static(const double* e_atom, int64_t n, double* e_total, void* stream);

/* Measured multiply-add peaks of the current device, the denominators of the
 * roofline of the ACE kernels (float32 pipe) and of the float64 path.  The paper
 * has no counterpart: it is a measurement aid.  A register-resident loop of
 * independent multiply-adds runs on every SM; the best of three launches, timed
 * with CUDA events on the stream, is written to the host outputs in TFLOP/s (a
 * multiply-add counts 2).  Synchronises the stream; changes no clock or power
 * setting; takes well under a second.  Errors: APIP_ERR_ARG (NULL output),
 * APIP_ERR_CUDA. */
apip_status apip_measure_peaks(double* fp32_tflops, double* fp64_tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* APIP_H */
