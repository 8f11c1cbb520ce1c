"""Python binding of libapip (ctypes over the C ABI of include/apip.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Functions carry the C names; tensors are torch CUDA tensors
(float64 for positions/velocities/forces/energies, int32 for ids and types)
and are passed by device pointer.  ``stream`` defaults to torch's current
stream.  Importing this module fails loudly if the library has not been built.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# APIP_LIBRARY may name another build of the same ABI (the bounds-checked
# libapip_checked.so); the default is the in-tree libapip.so
LIB_PATH = os.environ.get("APIP_LIBRARY") or os.path.join(_PKG, "libapip.so")

(APIP_OK, APIP_ERR_ARG, APIP_ERR_CUDA, APIP_ERR_NB_OVERFLOW, APIP_ERR_BAD_INPUT, APIP_ERR_STATE, APIP_ERR_SIZE,
 APIP_ERR_TIMEOUT, APIP_ERR_BOUNDS) = range(9)
STATUS_NAMES = {0: "APIP_OK", 1: "APIP_ERR_ARG", 2: "APIP_ERR_CUDA", 3: "APIP_ERR_NB_OVERFLOW",
                4: "APIP_ERR_BAD_INPUT", 5: "APIP_ERR_STATE", 6: "APIP_ERR_SIZE", 7: "APIP_ERR_TIMEOUT",
                8: "APIP_ERR_BOUNDS"}
APIP_STATIC_MAX_ATOMS = 4096 * 4096
APIP_FP64, APIP_FP32 = 0, 1
APIP_LAM_PAPER, APIP_LAM_CONST0, APIP_LAM_CONST1, APIP_LAM_LEARNED = 0, 1, 2, 3
APIP_MIX_ENERGY, APIP_MIX_FORCE = 0, 1
MIXING = {"energy": APIP_MIX_ENERGY, "force": APIP_MIX_FORCE}
LAM_MODES = {"paper": APIP_LAM_PAPER, "const0": APIP_LAM_CONST0, "const1": APIP_LAM_CONST1,
             "learned": APIP_LAM_LEARNED}
APIP_MLP_NPARAM = 10497
MLP_LAYOUT = (("W1", (64, 32)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64, 64)), ("b3", (64,)),
              ("w4", (64,)), ("b4", ()))
PHASES = ("prep", "neighbor", "pass1", "pass2", "ace", "csp", "reduce")
FIELDS = dict(g=0, d=1, wbar=2, lam=3, dlam=4, e_eam=5, e_ace=6, zeta=7, ace_list=8, nnb=9, nblist=10, csp=11,
              build_pos=12)
MVV2E = 1.0364269e-4   # amu A^2 / ps^2 -> eV

_c_int32, _c_int64, _c_double, _vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class ApipParams(ctypes.Structure):
    """Mirror of struct apip_params (field order is ABI)."""
    _fields_ = [
        ("precision", _c_int32), ("lam_mode", _c_int32), ("grad_lambda", _c_int32), ("precise_adds_eam", _c_int32),
        ("eam_A", _c_double), ("eam_beta", _c_double), ("eam_re", _c_double), ("eam_D", _c_double),
        ("eam_alpha", _c_double), ("eam_r0", _c_double), ("eam_rc", _c_double), ("eam_rc_width", _c_double),
        ("ace_n_max", _c_int32), ("ace_l_max", _c_int32), ("ace_nu_max", _c_int32), ("ace_group", _c_int32),
        ("ace_rc", _c_double), ("ace_rc_width", _c_double), ("ace_eps", _c_double), ("ace_a_scale", _c_double),
        ("ace_c1", ctypes.POINTER(_c_double)), ("ace_c2", ctypes.POINTER(_c_double)), ("ace_n_basis", _c_int64),
        ("sw_r_w", _c_double), ("sw_r_w_width", _c_double), ("sw_d_lo", _c_double), ("sw_d_hi", _c_double),
        ("sw_d0", _c_double),
        ("csp_rcut", _c_double), ("csp_nnb", _c_int32), ("nb_pad", _c_int32),
        ("skin", _c_double), ("max_nb", _c_int32), ("cell_cap", _c_int32), ("mixing", _c_int32),
        ("deterministic", _c_int32), ("prec_shift", _c_double),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2512_07693_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "apip_ace_basis_size": (_c_int64, [_c_int32, _c_int32, _c_int32]),
        "apip_create": (ctypes.c_int, [P(ApipParams), _c_int64, P(_vp)]),
        "apip_destroy": (ctypes.c_int, [_vp]),
        "apip_build_neighbors": (ctypes.c_int, [_vp, _vp, P(_c_double), _vp, _c_int64, _vp]),
        "apip_init_csp_pairs": (ctypes.c_int, [_vp, _vp, P(_c_double), _vp, _c_int64, _vp]),
        "apip_set_csp_pairs": (ctypes.c_int, [_vp, _vp, _c_int64, _vp]),
        "apip_switch": (ctypes.c_int, [_vp, _vp, P(_c_double), _vp, _vp, _c_int64, _vp, _vp, _vp, _vp]),
        "apip_energy_forces": (ctypes.c_int, [_vp, _vp, P(_c_double), _vp, _vp, _c_int64, _vp, _vp, _vp, _vp]),
        "apip_verlet_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, P(_c_double), _vp, _vp, _c_int64, _c_double,
                                            _c_int32, _vp, _vp]),
        "apip_sync": (ctypes.c_int, [_vp, _vp]),
        "apip_last_error": (ctypes.c_char_p, [_vp]),
        "apip_get_field": (ctypes.c_int, [_vp, _c_int32, _vp, _c_int64, _vp]),
        "apip_profile": (ctypes.c_int, [_vp, _c_int32]),
        "apip_profile_read": (ctypes.c_int, [_vp, P(_c_double), P(_c_int64)]),
        "apip_ace_info": (ctypes.c_int, [_vp, P(_c_int64)]),
        "apip_reduce_energy_static": (ctypes.c_int, [_vp, _c_int64, _vp, _vp]),
        "apip_measure_peaks": (ctypes.c_int, [P(_c_double), P(_c_double), _vp]),
        "apip_set_mlp": (ctypes.c_int, [_vp, _vp, _vp]),
        "apip_set_lam_fixed": (ctypes.c_int, [_vp, _vp, _c_int64]),
        "apip_set_indenter": (ctypes.c_int, [_vp, P(_c_double), P(_c_double), _c_double, _c_double]),
        "apip_indenter_state": (ctypes.c_int, [_vp, P(_c_double), P(_c_double)]),
        "apip_descriptors": (ctypes.c_int, [_vp, _vp, P(_c_double), _vp, _c_int64, _vp, _vp]),
        "apip_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _c_int64, _vp, _vp, _vp, _vp]),
        "apip_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _c_int32, ctypes.c_float, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if hasattr(lib, "apip_check_bounds_selftest"):   # the bounds-checked build only
        lib.apip_check_bounds_selftest.restype = ctypes.c_int
        lib.apip_check_bounds_selftest.argtypes = [_vp, _vp]
    return lib


lib = _load()


class ApipError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _box(box):
    return (_c_double * 3)(*[float(x) for x in box])


def _check(ctx, st):
    if st != APIP_OK:
        raise ApipError(st, lib.apip_last_error(ctx).decode() if ctx else "")


# ------------------------------------------------------------ C-named calls
def apip_ace_basis_size(n_max, l_max, nu_max):
    return int(lib.apip_ace_basis_size(n_max, l_max, nu_max))


def apip_create(params, n_atoms_max):
    ctx = _vp()
    st = lib.apip_create(ctypes.byref(params), int(n_atoms_max), ctypes.byref(ctx))
    if st != APIP_OK:
        raise ApipError(st, "apip_create rejected the parameters or could not allocate")
    return ctx


def apip_destroy(ctx):
    return lib.apip_destroy(ctx)


def apip_build_neighbors(ctx, pos, box, id, n, stream=None):
    _check(ctx, lib.apip_build_neighbors(ctx, _ptr(pos), _box(box), _ptr(id), int(n), _stream(stream)))


def apip_init_csp_pairs(ctx, pos, box, id, n, stream=None):
    _check(ctx, lib.apip_init_csp_pairs(ctx, _ptr(pos), _box(box), _ptr(id), int(n), _stream(stream)))


def apip_set_csp_pairs(ctx, partner_ids, n, stream=None):
    _check(ctx, lib.apip_set_csp_pairs(ctx, _ptr(partner_ids), int(n), _stream(stream)))


def apip_switch(ctx, pos, box, type, id, n, lam_out=None, dlam_out=None, n_ace_out=None, stream=None):
    _check(ctx, lib.apip_switch(ctx, _ptr(pos), _box(box), _ptr(type), _ptr(id), int(n), _ptr(lam_out),
                                _ptr(dlam_out), _ptr(n_ace_out), _stream(stream)))


def apip_energy_forces(ctx, pos, box, type, id, n, force_out, e_atom_out=None, e_total_out=None, stream=None):
    _check(ctx, lib.apip_energy_forces(ctx, _ptr(pos), _box(box), _ptr(type), _ptr(id), int(n), _ptr(force_out),
                                       _ptr(e_atom_out), _ptr(e_total_out), _stream(stream)))


def apip_verlet_step(ctx, pos, vel, force, inv_mass, box, type, id, n, dt, n_steps, thermo_out=None, stream=None):
    _check(ctx, lib.apip_verlet_step(ctx, _ptr(pos), _ptr(vel), _ptr(force), _ptr(inv_mass), _box(box), _ptr(type),
                                     _ptr(id), int(n), float(dt), int(n_steps), _ptr(thermo_out), _stream(stream)))


def apip_sync(ctx, stream=None):
    _check(ctx, lib.apip_sync(ctx, _stream(stream)))


def apip_last_error(ctx):
    return lib.apip_last_error(ctx).decode()


def apip_get_field(ctx, field, dst, n, stream=None):
    f = FIELDS[field] if isinstance(field, str) else int(field)
    _check(ctx, lib.apip_get_field(ctx, f, _ptr(dst), int(n), _stream(stream)))


def apip_profile(ctx, enable):
    _check(ctx, lib.apip_profile(ctx, int(bool(enable))))


def apip_profile_read(ctx):
    """{phase: (milliseconds, launches)} accumulated since the last read."""
    ms = (_c_double * len(PHASES))()
    nl = (_c_int64 * len(PHASES))()
    _check(ctx, lib.apip_profile_read(ctx, ms, nl))
    return {name: (ms[k], nl[k]) for k, name in enumerate(PHASES)}


ACE_INFO = ("values_per_atom", "couplings", "gaunt_products", "records", "record_len_sum", "row_len_sum",
            "c_to_a_entries", "group", "blocks", "kind", "table_flops")


def apip_ace_info(ctx):
    """Sizes of the ACE evaluation built at creation, as a dict (see ACE_INFO)."""
    out = (_c_int64 * len(ACE_INFO))()
    _check(ctx, lib.apip_ace_info(ctx, out))
    return {k: int(out[q]) for q, k in enumerate(ACE_INFO)}


def apip_reduce_energy_static(e_atom, n, e_total, stream=None):
    """Total of e_atom[0..n) into e_total[0] without any device allocation (for
    callers that cannot call cudaMalloc); n <= APIP_STATIC_MAX_ATOMS.  Calls that
    overlap on the GPU share one scratch array and race; serialise them."""
    st = lib.apip_reduce_energy_static(_ptr(e_atom), int(n), _ptr(e_total), _stream(stream))
    if st != APIP_OK:
        why = {APIP_ERR_SIZE: f"n = {n} exceeds APIP_STATIC_MAX_ATOMS = {APIP_STATIC_MAX_ATOMS}",
               APIP_ERR_ARG: "NULL pointer or negative n"}.get(st, "CUDA error")
        raise ApipError(st, why)


def apip_measure_peaks(stream=None):
    """Measured float32 and float64 multiply-add peaks (TFLOP/s) of the current device."""
    f32, f64 = _c_double(0.0), _c_double(0.0)
    _check(None, lib.apip_measure_peaks(ctypes.byref(f32), ctypes.byref(f64), _stream(stream)))
    return f32.value, f64.value


def apip_set_mlp(ctx, params, stream=None):
    _check(ctx, lib.apip_set_mlp(ctx, _ptr(params), _stream(stream)))


def apip_set_lam_fixed(ctx, lam_fixed, n):
    """Constant lam on a subset (float64 device tensor, NaN = follow the switch),
    or None to clear."""
    _check(ctx, lib.apip_set_lam_fixed(ctx, _ptr(lam_fixed), int(n)))


def apip_set_indenter(ctx, center, velocity, radius, k):
    """Spherical indenter (host centre and velocity); radius <= 0 removes it."""
    c = (_c_double * 3)(*[float(v) for v in center])
    v = (_c_double * 3)(*[float(x) for x in velocity])
    _check(ctx, lib.apip_set_indenter(ctx, c, v, float(radius), float(k)))


def apip_indenter_state(ctx):
    """(centre as a list, accumulated work W)."""
    c = (_c_double * 3)()
    w = _c_double()
    _check(ctx, lib.apip_indenter_state(ctx, c, ctypes.byref(w)))
    return [c[0], c[1], c[2]], w.value


def apip_descriptors(ctx, pos, box, id, n, desc_bf16, stream=None):
    _check(ctx, lib.apip_descriptors(ctx, _ptr(pos), _box(box), _ptr(id), int(n), _ptr(desc_bf16), _stream(stream)))


def apip_mlp_loss_grad(ctx, desc_bf16, y, batch, params, grad_out, loss_out, stream=None):
    _check(ctx, lib.apip_mlp_loss_grad(ctx, _ptr(desc_bf16), _ptr(y), int(batch), _ptr(params), _ptr(grad_out),
                                       _ptr(loss_out), _stream(stream)))


def apip_mlp_adam(ctx, params, grad, m, v, t, lr, stream=None):
    _check(ctx, lib.apip_mlp_adam(ctx, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr),
                                  _stream(stream)))


def mlp_flat(weights):
    """Flat float32 parameter vector (apip.h layout) from a dict of arrays."""
    parts = [np.asarray(weights[k], dtype=np.float32).reshape(-1) for k, _ in MLP_LAYOUT]
    out = np.concatenate(parts)
    assert out.size == APIP_MLP_NPARAM
    return out


def mlp_unflat(flat):
    """Inverse of mlp_flat (float64 arrays; b4 a float)."""
    flat = np.asarray(flat, dtype=np.float64).reshape(-1)
    out, k = {}, 0
    for name, shape in MLP_LAYOUT:
        size = int(np.prod(shape)) if shape else 1
        out[name] = flat[k:k + size].reshape(shape) if shape else float(flat[k])
        k += size
    return out


# ---------------------------------------------------------------- helpers
def make_params(prm, precision="fp64", lam_mode="paper", grad_lambda=True, skin=0.5, max_nb=96, cell_cap=64,
                ace_group=0, mixing="energy", deterministic=False):
    """apip_params from a parameter dict (keys eam, ace, switch, csp,
    precise_adds_eam, optional prec_shift).  The returned structure keeps the coefficient arrays
    alive through its ``_keep`` attribute."""
    e, a, s, c = prm["eam"], prm["ace"], prm["switch"], prm["csp"]
    c1 = np.ascontiguousarray(a["c1"], dtype=np.float64)
    c2 = np.ascontiguousarray(a["c2"], dtype=np.float64)
    p = ApipParams()
    p.precision = {"fp64": APIP_FP64, "fp32": APIP_FP32}[precision]
    p.lam_mode = LAM_MODES[lam_mode]
    p.grad_lambda = int(bool(grad_lambda))
    p.precise_adds_eam = int(bool(prm.get("precise_adds_eam", False)))
    p.eam_A, p.eam_beta, p.eam_re = e["A"], e["beta"], e["r_e"]
    p.eam_D, p.eam_alpha, p.eam_r0 = e["D"], e["alpha"], e["r_0"]
    p.eam_rc, p.eam_rc_width = e["rc"], e["rc_width"]
    p.ace_n_max, p.ace_l_max, p.ace_nu_max = a["n_max"], a["l_max"], a["nu_max"]
    p.ace_rc, p.ace_rc_width, p.ace_eps, p.ace_a_scale = a["rc"], a["rc_width"], a["eps"], a["a_scale"]
    p.ace_group = int(ace_group)
    nb = apip_ace_basis_size(a["n_max"], a["l_max"], a["nu_max"])
    assert len(c1) >= nb and len(c2) >= nb
    c1, c2 = np.ascontiguousarray(c1[:nb]), np.ascontiguousarray(c2[:nb])
    p.ace_c1 = c1.ctypes.data_as(ctypes.POINTER(_c_double))
    p.ace_c2 = c2.ctypes.data_as(ctypes.POINTER(_c_double))
    p.ace_n_basis = nb
    p.sw_r_w, p.sw_r_w_width = s["r_w"], s["r_w_width"]
    p.sw_d_lo, p.sw_d_hi, p.sw_d0 = s["d_lo"], s["d_hi"], s["d0"]
    p.csp_rcut, p.csp_nnb = c["rcut"], c["nnb"]
    p.skin, p.max_nb, p.cell_cap = skin, max_nb, cell_cap
    p.mixing = MIXING[mixing]
    p.deterministic = int(bool(deterministic))
    p.prec_shift = float(prm.get("prec_shift", 0.0))
    p._keep = (c1, c2)
    return p


class Apip:
    """One library context with its parameters; thin convenience over the C calls."""

    def __init__(self, prm, n_atoms_max, **kw):
        self.params = make_params(prm, **kw)
        self.ctx = apip_create(self.params, n_atoms_max)
        self.n_atoms_max = int(n_atoms_max)
        self.max_nb = self.params.max_nb
        self.csp_nnb = self.params.csp_nnb

    def close(self):
        if self.ctx:
            apip_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_csp_pairs(self, pos, box, ids, stream=None):
        apip_init_csp_pairs(self.ctx, pos, box, ids, pos.shape[0], stream)

    def set_csp_pairs(self, partner_ids, stream=None):
        """Restore saved partner ids (int32 [n][csp_nnb] device tensor, row k for atom id k)."""
        self._csp_saved = partner_ids   # kept alive until the copy on the stream has run
        apip_set_csp_pairs(self.ctx, partner_ids, partner_ids.shape[0], stream)

    def build_neighbors(self, pos, box, ids, stream=None):
        apip_build_neighbors(self.ctx, pos, box, ids, pos.shape[0], stream)

    def switch(self, pos, box, types, ids, lam_out=None, dlam_out=None, n_ace_out=None, stream=None):
        apip_switch(self.ctx, pos, box, types, ids, pos.shape[0], lam_out, dlam_out, n_ace_out, stream)

    def energy_forces(self, pos, box, types, ids, force_out, e_atom_out=None, e_total_out=None, stream=None):
        apip_energy_forces(self.ctx, pos, box, types, ids, pos.shape[0], force_out, e_atom_out, e_total_out, stream)

    def verlet_step(self, pos, vel, force, inv_mass, box, types, ids, dt, n_steps, thermo_out=None, stream=None):
        apip_verlet_step(self.ctx, pos, vel, force, inv_mass, box, types, ids, pos.shape[0], dt, n_steps,
                         thermo_out, stream)

    def sync(self, stream=None):
        apip_sync(self.ctx, stream)

    def set_mlp(self, params, stream=None):
        apip_set_mlp(self.ctx, params, stream)

    def set_indenter(self, center, velocity, radius, k):
        apip_set_indenter(self.ctx, center, velocity, radius, k)

    def indenter_state(self):
        return apip_indenter_state(self.ctx)

    def set_lam_fixed(self, lam_fixed):
        self._lam_fixed = lam_fixed   # the library reads it on later calls
        apip_set_lam_fixed(self.ctx, lam_fixed, 0 if lam_fixed is None else lam_fixed.shape[0])

    def descriptors(self, pos, box, ids, desc_bf16, stream=None):
        apip_descriptors(self.ctx, pos, box, ids, pos.shape[0], desc_bf16, stream)

    def field(self, name, n):
        """Copy an internal per-atom array into a new torch tensor."""
        import torch
        dev = torch.device("cuda")
        if name == "nblist":
            out = torch.empty((n, self.max_nb), dtype=torch.int64, device=dev)
        elif name == "csp":
            out = torch.empty((n, self.csp_nnb), dtype=torch.int64, device=dev)
        elif name in ("ace_list", "nnb"):
            out = torch.empty(n, dtype=torch.int64, device=dev)
        elif name == "build_pos":
            out = torch.empty((n, 3), dtype=torch.float64, device=dev)
        else:
            out = torch.empty(n, dtype=torch.float64, device=dev)
        apip_get_field(self.ctx, name, out, n)
        return out
