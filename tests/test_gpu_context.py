"""One context across calls that change what it was built for, and the switch-only
entry point, through the C ABI against a fresh context and the FP64 oracle.

- The atom count may change between calls (any n up to n_atoms_max): the
  neighbour list of the last build must then be rebuilt even though no atom
  moved, or it would hold indices past the new end (n shrank) or miss the new
  atoms (n grew).
- The CSP^list partners are kept by atom id (Appendix B): when an id disappears
  and another atom takes its index, the stale id -> index entry must be reported,
  not used as a partner.
- apip_switch returns lam, dlam/dd (Eq. 2, Eq. 6, Eq. S1-S3) and |P|."""
import numpy as np
import pytest

from gpu_helpers import run_oracle, to_dev, torch_cuda
from oracle import ace
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _prm(acecfg=(6, 3, 3)):
    nb = len(ace.enumerate_basis(*acecfg))
    return dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(*acecfg, 2, nb))


def _eval(torch, m, s, n):
    """Energy, per-atom energies and forces of the first n atoms of s."""
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"][:n].contiguous(), box, t["types"][:n].contiguous(), t["ids"][:n].contiguous(),
                    F, e, E)
    m.sync()
    return F.cpu().numpy(), e.cpu().numpy(), float(E.cpu()[0])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_atom_count_change_rebuilds_the_list(prec):
    """lam = 1 everywhere (the ACE adjoint scatters into every neighbour's force):
    one context called with n, then n - k, then n + k atoms at unchanged positions,
    each call against a fresh context of that size."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=21)
    prm = _prm()
    ntot = len(s["pos"])
    k = 37
    n = ntot - k
    m = apip.Apip(prm, ntot, precision=prec, lam_mode="const1")
    tol = 1e-10 if prec == "fp64" else 1e-6
    for count in (n, n - k, ntot, n):
        F, e, E = _eval(torch, m, s, count)
        fresh = apip.Apip(prm, count, precision=prec, lam_mode="const1")
        Ff, ef, Ef = _eval(torch, fresh, s, count)
        fresh.close()
        assert np.abs(F - Ff).max() <= tol, count
        assert np.abs(e - ef).max() <= tol, count
        assert abs(E - Ef) <= tol * count, count
    m.close()


def test_vanished_partner_id_is_reported():
    """After the pairs are detected, atom id 5 leaves and the last atom takes its
    index: the atoms that had id 5 as a partner must not silently pair with the
    atom now at index 5."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=21)
    n = len(s["pos"])
    m = apip.Apip(_prm(), n, precision="fp64")
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.sync()
    partners = m.field("csp", n).cpu().numpy()
    assert np.any(partners == 5)
    order = np.arange(n - 1)
    order[5] = n - 1
    o = torch.tensor(order, device="cuda")
    F2 = torch.empty((n - 1, 3), dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"][o].contiguous(), box, t["types"][o].contiguous(), t["ids"][o].contiguous(), F2)
    with pytest.raises(apip.ApipError) as err:
        m.sync()
    assert err.value.status == apip.APIP_ERR_BAD_INPUT
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_switch_entry_point_matches_oracle(prec):
    """lam, dlam and the count of atoms with lam > 0 from apip_switch alone."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=21)
    s["prm"] = _prm()
    n = len(s["pos"])
    o = run_oracle(s)
    m = apip.Apip(s["prm"], n, precision=prec)
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    lam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    dlam = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    m.switch(t["pos"], box, t["types"], t["ids"], lam, dlam, cnt)
    m.sync()
    lam, dlam, cnt = lam.cpu().numpy(), dlam.cpu().numpy(), int(cnt.cpu()[0])
    m.close()
    assert np.count_nonzero(o["dlam"]) > 10
    if prec == "fp64":
        np.testing.assert_allclose(lam, o["lam"], atol=1e-12, rtol=0)
        np.testing.assert_allclose(dlam, o["dlam"], atol=1e-10, rtol=0)
        assert cnt == len(o["P"])
    else:
        np.testing.assert_allclose(lam, o["lam"], atol=1e-5, rtol=0)
        np.testing.assert_allclose(dlam, o["dlam"], atol=1e-4 * np.abs(o["dlam"]).max(), rtol=0)
        # the set may differ only where d lies within float32 rounding of d_lo
        assert abs(cnt - len(o["P"])) <= np.count_nonzero(np.abs(o["d"] - s["prm"]["switch"]["d_lo"]) < 1e-5)
        assert cnt == int((lam > 0).sum())
