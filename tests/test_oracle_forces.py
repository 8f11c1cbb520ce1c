"""Pins of the complete adaptive-precision oracle: F = -grad E by central finite
differences (Eq. 5), sum_i F_i = 0 (Newton's third law, Eq. A1), translation
and rotation invariance, the constant-switch special cases (lam = 1 pure ACE,
lam = 0 pure EAM, Appendix B) and bounded NVE energy (Fig. S2 / S3)."""
import math

import numpy as np
import pytest

from oracle import ace, apip, csp, verlet
from oracle.neighbors import pairs
from oracle.eam import eam_energies
from paper_2512_07693_gb300 import workloads as W


def nbasis(a, b, c):
    return len(ace.enumerate_basis(a, b, c))


def small_system(precise_adds_eam=True, nu=3, seed=21, cells=6, sigma=0.06):
    s = W.vacancy_crystal(cells=cells, sigma=sigma, seed=seed)
    prm = dict(precise_adds_eam=precise_adds_eam, eam=dict(W.EAM), csp=dict(W.CSP),
               switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9),
               ace=W.ace_params(4 if nu == 4 else 6, 3, nu, 2, nbasis(4 if nu == 4 else 6, 3, nu)))
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    return s, prm, part


@pytest.fixture(scope="module")
def sysA():
    s, prm, part = small_system()
    model = ace.AceModel(prm["ace"])
    res = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model)
    return s, prm, part, model, res


def _fd(s, prm, part, model, atoms, h=1e-5, **kw):
    out = []
    for a in atoms:
        row = []
        for c in range(3):
            pp, pm = s["pos"].copy(), s["pos"].copy()
            pp[a, c] += h
            pm[a, c] -= h
            ep = apip.energy_forces(pp, s["box"], s["ids"], part, prm, model=model, forces=False, **kw)["E"]
            em = apip.energy_forces(pm, s["box"], s["ids"], part, prm, model=model, forces=False, **kw)["E"]
            row.append(-(ep - em) / (2 * h))
        out.append(row)
    return np.array(out)


def _pick(res):
    """Atoms of every kind: pure ACE, transition, pure EAM next to ACE, bulk."""
    lam, dlam = res["lam"], res["dlam"]
    n = len(lam)
    full = np.nonzero(lam == 1.0)[0]
    trans = np.nonzero(dlam != 0.0)[0]
    zero = np.nonzero(lam == 0.0)[0]
    picks = list(full[:2]) + list(trans[:4]) + list(zero[:2]) + [n - 1]
    return sorted(set(int(a) for a in picks))


def test_mixture_has_all_regimes(sysA):
    _, _, _, _, res = sysA
    lam = res["lam"]
    assert np.any(lam == 1.0) and np.any(lam == 0.0)
    assert np.count_nonzero(res["dlam"]) >= 10


def test_total_force_is_minus_gradient(sysA):
    s, prm, part, model, res = sysA
    atoms = _pick(res)
    fd = _fd(s, prm, part, model, atoms)
    np.testing.assert_allclose(res["F"][atoms], fd, atol=2e-6, rtol=1e-6)


def test_pure_ace_precise_model_force_is_minus_gradient():
    """Same check with the precise model = ACE alone (no EAM reference)."""
    s, prm, part = small_system(precise_adds_eam=False, cells=5)
    model = ace.AceModel(prm["ace"])
    res = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model)
    atoms = _pick(res)
    fd = _fd(s, prm, part, model, atoms)
    np.testing.assert_allclose(res["F"][atoms], fd, atol=2e-6, rtol=1e-6)


def test_shifted_energy_zero_force_is_minus_gradient(sysA):
    """With the precise model's energy lowered by a constant per atom, E changes by
    -shift sum_i lam_i (Eq. 4) and the force by the matching grad-lambda term: it is
    still -grad E, and it differs from the unshifted force exactly by
    shift * sum_i grad lam_i, which no model force carries."""
    s, prm, part, model, res = sysA
    shift = 0.7
    sprm = dict(prm, prec_shift=shift)
    r2 = apip.energy_forces(s["pos"], s["box"], s["ids"], part, sprm, model=model)
    assert r2["E"] == pytest.approx(res["E"] - shift * math.fsum(res["lam"]), abs=1e-9)
    np.testing.assert_allclose(r2["lam"], res["lam"], atol=0)
    atoms = _pick(r2)
    fd = _fd(s, sprm, part, model, atoms)
    np.testing.assert_allclose(r2["F"][atoms], fd, atol=2e-6, rtol=1e-6)
    assert np.abs(r2["F"] - res["F"]).max() > 1e-3
    np.testing.assert_allclose(r2["F"].sum(axis=0), 0.0, atol=1e-9)


def test_nu4_force_is_minus_gradient():
    s, prm, part = small_system(nu=4, cells=5)
    model = ace.AceModel(prm["ace"])
    res = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model)
    atoms = _pick(res)[:4]
    fd = _fd(s, prm, part, model, atoms)
    np.testing.assert_allclose(res["F"][atoms], fd, atol=2e-6, rtol=1e-6)


def test_grad_lambda_term_is_needed(sysA):
    """Without F^(grad lambda) (Fig. 3b ablation) the force is not -grad E."""
    s, prm, part, model, res = sysA
    no = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, grad_lambda=False)
    diff = np.abs(no["F"] - res["F"]).max()
    assert diff > 1e-3
    assert np.abs(no["F"].sum(axis=0)).max() < 1e-9   # still pairwise


def test_newton_third_law(sysA):
    _, _, _, _, res = sysA
    F = res["F"]
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * max(1.0, np.abs(F).max()) * len(F)


def test_translation_and_rotation_invariance(sysA):
    s, prm, part, model, res = sysA
    shifted = s["pos"] + np.array([0.37, -1.21, 2.5])
    r2 = apip.energy_forces(shifted, s["box"], s["ids"], part, prm, model=model)
    assert r2["E"] == pytest.approx(res["E"], abs=1e-9)
    np.testing.assert_allclose(r2["F"], res["F"], atol=1e-9)
    # a cubic-lattice symmetry of the periodic box: (x, y, z) -> (y, z, x)
    rot = s["pos"][:, [1, 2, 0]]
    r3 = apip.energy_forces(rot, s["box"], s["ids"], part, prm, model=model)
    assert r3["E"] == pytest.approx(res["E"], abs=1e-9)
    np.testing.assert_allclose(r3["F"], res["F"][:, [1, 2, 0]], atol=1e-9)


def test_constant_switch_special_cases(sysA):
    s, prm, part, model, res = sysA
    n = len(s["pos"])
    i, j, rv, r = pairs(s["pos"], s["box"], apip.cutoff(prm))
    e_eam, _ = eam_energies(n, i, j, r, prm["eam"])
    e_ace, _ = ace.ace_energy_forces(model, n, i, j, rv, r, np.arange(n))
    r0 = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_mode="const0")
    assert r0["E"] == pytest.approx(math.fsum(e_eam), abs=1e-9)
    r1 = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_mode="const1")
    assert r1["E"] == pytest.approx(math.fsum(e_ace + e_eam), abs=1e-9)   # precise = EAM + ACE
    # lam fixed on a subset (Appendix B): still -grad E, dlam = 0 there
    lc = np.full(n, np.nan)
    lc[:40] = 1.0
    lc[40:80] = 0.0
    rc = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_const=lc)
    assert np.all(rc["dlam"][:80] == 0.0)
    atoms = [3, 45, int(np.nonzero(rc["dlam"])[0][0])]
    fd = _fd(s, prm, part, model, atoms, lam_const=lc)
    np.testing.assert_allclose(rc["F"][atoms], fd, atol=2e-6, rtol=1e-6)


def test_nve_energy_is_conserved():
    s = W.vacancy_crystal(cells=5, sigma=0.03, seed=4, temp=300.0)
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
               switch=dict(W.SWITCH, d_lo=0.2, d_hi=0.8),
               ace=W.ace_params(4, 2, 3, 2, nbasis(4, 2, 3)))
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    model = ace.AceModel(prm["ace"])
    H = {}
    for dt in (0.002, 0.001):
        steps = int(round(0.02 / dt))
        _, _, _, log = verlet.run(s["pos"], s["vel"], s["box"], s["ids"], part, prm, s["mass"], dt, steps, model=model)
        h = np.array([e + k for e, k, _ in log])
        H[dt] = np.abs(h - h[0]).max() / len(s["pos"])
        p = np.array([q for _, _, q in log])
        assert np.abs(p - p[0]).max() < 1e-10          # momentum conserved to rounding
    assert H[0.001] < 1e-4
    # Verlet energy error is second order in dt
    assert H[0.002] / H[0.001] == pytest.approx(4.0, rel=0.35)


def test_force_mixing_combines_the_two_complete_forces(sysA):
    """Eq. 3 (force mixing): F_i = (1 - lam_i) F_i^fast + lam_i F_i^prec with the
    complete forces of the two models, here taken from two independent constant
    switches (lam = 0: the fast model everywhere; lam = 1: the precise model
    everywhere, Appendix B), and lam from the paper's switch."""
    s, prm, part, model, res = sysA
    fm = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, mixing="force")
    f0 = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_mode="const0")["F"]
    f1 = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_mode="const1")["F"]
    lam = res["lam"][:, None]
    np.testing.assert_allclose(fm["F"], (1 - lam) * f0 + lam * f1, atol=1e-11)
    assert fm["E"] == res["E"]


def test_force_mixing_breaks_newton_and_differs_from_the_gradient(sysA):
    """Force mixing is not the gradient of Eq. 4 and does not conserve momentum
    (the qualitative statements after Eq. 3)."""
    s, prm, part, model, res = sysA
    fm = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, mixing="force")
    assert np.abs(fm["F"].sum(axis=0)).max() > 1e-3
    assert np.abs(res["F"].sum(axis=0)).max() < 1e-10
    assert np.abs(fm["F"] - res["F"]).max() > 1e-2
