// Kernel argument block and launch wrappers of libapip (internal).
#pragma once

#include <cuda_runtime.h>

#include "apip_internal.h"
#include "device_common.cuh"

namespace apip {

// Everything a kernel of the force pipeline may need, passed by value.
template <typename T>
struct Args {
  int n, nmax, max_nb, cell_cap, csp_nnb;
  int lam_mode, precise_adds_eam, grad_lambda;
  int eam_force;          // pass 2 computes the (unweighted) EAM force
  PosView<T> pv;
  Geo geo;
  EamP eam;
  SwP sw;
  double r_list2, skin_half2, csp_rcut2;

  const double* pos;      // caller positions [n][3]
  const int* id;          // caller ids [n]
  int* nnb; int* nbl; double* pos_ref; float4* posh; float4* posl; int* id2idx; int* csp;
  int* cell_count; int* cell_atoms;
  T* zeta; T* xi_p; T* e_eam; T* g; T* wbar; T* dd; T* lam; T* dlam; T* e_ace;
  double* cvec; int* ace_list; int* counts; int* flags; int* status;
  double* partials; int n_part_p1;
  double* force;          // caller force [n][3]
  double* e_atom;         // caller per-atom energy [n] or null
};

template <typename T> Args<T> make_args(apip_ctx* c, const double* pos, const int* id, int n,
                                        double* force, double* e_atom);

// all-atom passes (kernels_atoms.cu)
template <typename T> void launch_prep(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_neighbors(const Args<T>& a, int ncell, cudaStream_t s);
void launch_csp_init(const Args<double>& a, cudaStream_t s);
template <typename T> void launch_pass1(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_pass2(const Args<T>& a, cudaStream_t s);
template <typename T> void launch_csp_force(const Args<T>& a, cudaStream_t s);
void launch_final(double* partials, int n_part, double* e_total, double* e_pot_slot,
                  const double* thermo_part, int n_tblocks, double* thermo_slot, int* flags,
                  const int* counts, int64_t* n_ace_out, cudaStream_t s);
template <typename T> void launch_get_field(const Args<T>& a, int field, void* dst, cudaStream_t s);
void launch_fill_const_list(int* list, int* counts, int n, cudaStream_t s);

// velocity Verlet (kernels_atoms.cu); mode 0 = first (kick, drift), 1 = mid
// (kick, thermo partials, kick, drift), 2 = last (kick, thermo partials)
template <typename T> void launch_verlet(const Args<T>& a, int mode, double* pos, double* vel,
                                         const double* force, const double* inv_mass, double dt,
                                         double* thermo_part, cudaStream_t s);
void launch_thermo_final(const double* thermo_part, int n_tblocks, double* thermo_slot, cudaStream_t s);

// ACE (kernels_ace.cu)
template <typename T> void ace_set_norms(const double* norms, int count);
template <typename T> void launch_ace(const Args<T>& a, const AceDev<T>& ace, int blocks, cudaStream_t s);

}  // namespace apip
