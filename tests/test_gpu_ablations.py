"""GPU parity of the comparison modes of the paper and of constant-switch
subsets, and their conservation properties in NVE:
  - force mixing (Eq. 3) against the oracle's force mixing;
  - lam fixed on a subset of atoms (Appendix B) against the oracle's lam_const;
  - NVE: the conservative AP force keeps the total momentum and (to the
    integrator's error) the energy; force mixing breaks momentum conservation and
    dropping grad-lambda breaks energy conservation (the contrast of Fig. 5)."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, run_oracle, torch_cuda
from oracle import ace
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def mixed(seed=21, cells=(6, 6, 6), adds_eam=True, acecfg=(6, 3, 3)):
    pos, box = W.bcc(*cells)
    pos = np.delete(pos, np.random.default_rng(seed).integers(len(pos)), axis=0)
    pos = W.displace(pos, 0.06, seed)
    s = W._finish(pos, np.zeros_like(pos), box)
    nb = len(ace.enumerate_basis(*acecfg))
    s["prm"] = dict(precise_adds_eam=adds_eam, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(*acecfg, 2, nb))
    return s


@pytest.mark.parametrize("prec,tol,adds_eam,acecfg", [("fp64", 1e-9, True, (6, 3, 3)), ("fp32", 2e-4, True, (6, 3, 3)),
                                                      ("fp64", 1e-9, False, (6, 3, 3)),
                                                      ("fp64", 1e-9, True, (4, 3, 4))])
def test_force_mixing_parity(prec, tol, adds_eam, acecfg):
    s = mixed(adds_eam=adds_eam, acecfg=acecfg)
    o = run_oracle(s, mixing="force")
    assert np.count_nonzero((o["lam"] > 0) & (o["lam"] < 1)) > 10
    g = run_gpu(s, precision=prec, mixing="force")
    err = np.abs(g["F"] - o["F"]).max()
    assert err <= tol, err
    np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=1e-9 if prec == "fp64" else 1e-5)
    # the precise model's buffer: every atom within r_c of lam > 0 was evaluated
    assert g["count"] >= np.count_nonzero(o["lam"] > 0)


@pytest.mark.parametrize("mode", ["paper", "const0"])
def test_lam_fixed_subset_parity(mode):
    s = mixed()
    n = len(s["pos"])
    fixed = np.full(n, np.nan)
    rng = np.random.default_rng(3)
    idx = rng.permutation(n)
    fixed[idx[:40]] = 1.0
    fixed[idx[40:80]] = 0.0
    fixed[idx[80:100]] = 0.5
    o = run_oracle(s, lam_mode=mode, lam_const=fixed)
    g = run_gpu(s, precision="fp64", lam_mode=mode, lam_fixed=fixed)
    np.testing.assert_allclose(g["lam"], o["lam"], atol=1e-12)
    np.testing.assert_allclose(g["dlam"], o["dlam"], atol=1e-10)
    assert np.abs(g["F"] - o["F"]).max() <= 1e-9
    np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=1e-9)


def _nve(s, steps, **kw):
    torch = torch_cuda()
    s = dict(s, vel=W.maxwell(len(s["pos"]), 600.0, 11))
    g = run_gpu(s, "fp64", fields=False, **kw)
    m, t = g["model"], g["t"]
    F = torch.tensor(g["F"], device="cuda")
    thermo = torch.zeros((steps, 5), dtype=torch.float64, device="cuda")
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], g["box"], t["types"], t["ids"], 0.001, steps, thermo)
    m.sync()
    th = thermo.cpu().numpy()
    n = len(s["pos"])
    H = (th[:, 0] + th[:, 1]) / n
    dP = np.abs(th[-1, 2:] - th[0, 2:]).max()
    return np.abs(H - H[0]).max(), dP


def test_only_the_conservative_force_conserves_energy_and_momentum():
    s = mixed(seed=5)
    dh_ap, dp_ap = _nve(s, 1000)
    dh_fm, dp_fm = _nve(s, 1000, mixing="force")
    dh_ng, dp_ng = _nve(s, 1000, grad_lambda=False)
    assert dp_ap < 1e-10                     # Newton's third law, pair by pair
    assert dp_fm > 1e3 * max(dp_ap, 1e-12)   # force mixing: momentum not conserved
    assert dh_ng > 10 * dh_ap                # no grad-lambda: the energy wanders
    assert dh_fm > 10 * dh_ap
