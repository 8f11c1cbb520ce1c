"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function that include/apip.h declares, and its host-side logic (basis size,
parameter validation) agrees with the oracle.  No GPU work is launched."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2512_07693_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    from paper_2512_07693_gb300 import apip
    return apip


def _declared(checked=False):
    """Function names the header declares; the declarations inside
    #ifdef APIP_CHECK_BOUNDS only with checked=True (the bounds-checked build)."""
    text = open(os.path.join(ROOT, "include", "apip.h")).read()
    if not checked:
        text = re.sub(r"#ifdef APIP_CHECK_BOUNDS.*?#endif", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(apip_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    assert "apip_check_bounds_selftest" not in names
    assert "apip_check_bounds_selftest" in _declared(checked=True)
    for n in ("apip_create", "apip_destroy", "apip_build_neighbors", "apip_init_csp_pairs", "apip_switch",
              "apip_energy_forces", "apip_verlet_step", "apip_sync", "apip_last_error", "apip_get_field",
              "apip_ace_basis_size"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (apip_\w+)", out))
    for n in _declared():
        assert n in exported, n
        getattr(lib.lib, n)


def test_build_targets_sm_103a_only(lib):
    from paper_2512_07693_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_basis_size_matches_oracle(lib):
    from oracle import ace
    for cfg in [(6, 3, 3), (4, 3, 4), (3, 2, 2), (1, 0, 1), (8, 4, 3), (2, 4, 4)]:
        assert lib.apip_ace_basis_size(*cfg) == len(ace.enumerate_basis(*cfg))
    assert lib.apip_ace_basis_size(9, 3, 3) == -1
    assert lib.apip_ace_basis_size(2, 5, 3) == -1
    assert lib.apip_ace_basis_size(2, 2, 5) == -1


def test_create_rejects_bad_parameters_before_touching_the_device(lib):
    from paper_2512_07693_gb300 import workloads as W
    s = W.config("vacancy2k", lib.apip_ace_basis_size)
    cases = [("csp_nnb", 3), ("precision", 7), ("lam_mode", 9), ("ace_n_max", 0), ("ace_l_max", 5),
             ("sw_d_hi", -1.0), ("max_nb", 0), ("ace_n_basis", 5), ("skin", -0.1), ("csp_rcut", 99.0),
             ("deterministic", 2), ("mixing", lib.APIP_MIX_FORCE), ("precision", lib.APIP_FP64)]
    for k, (field, val) in enumerate(cases):
        # (the last two are rejected only together with the deterministic mode,
        # which needs the float32 path and energy mixing)
        p = lib.make_params(s["prm"], precision="fp32", deterministic=k >= len(cases) - 2)
        setattr(p, field, val)
        ctx = ctypes.c_void_p()
        assert lib.lib.apip_create(ctypes.byref(p), 100, ctypes.byref(ctx)) == lib.APIP_ERR_ARG, field
        assert not ctx.value
    p = lib.make_params(s["prm"])
    ctx = ctypes.c_void_p()
    assert lib.lib.apip_create(ctypes.byref(p), 0, ctypes.byref(ctx)) == lib.APIP_ERR_ARG
    assert lib.lib.apip_create(None, 10, ctypes.byref(ctx)) == lib.APIP_ERR_ARG
    # calls on a NULL context are argument errors, not crashes
    assert lib.lib.apip_sync(None, None) == lib.APIP_ERR_ARG
    assert lib.lib.apip_destroy(None) == lib.APIP_OK
    assert lib.lib.apip_last_error(None) == b""

