"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix: the printed transition function (Eq. S1 / Fig. S1), library
special functions, exact quadrature identities and closed forms."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import ace, csp, eam, ftrans, neighbors, switch
from paper_2512_07693_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ f_trans
def test_ftrans_matches_figS1_exact_values():
    """Eq. S1 at the Fig. S1 parameter sets, against exact rationals."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "ftrans_figS1.txt")) if not l.startswith("#")]
    assert len(rows) == 114
    for lo, hi, x, v in rows:
        xv = float(Fraction(x))
        assert ftrans.f_trans(xv, float(lo), float(hi)) == pytest.approx(float(Fraction(v)), abs=1e-15)


def test_ftrans_landmarks_and_symmetry():
    lo, hi = 1.3, 2.9
    assert ftrans.f_trans(lo, lo, hi) == 1.0
    assert ftrans.f_trans(hi, lo, hi) == 0.0
    assert ftrans.f_trans(0.5 * (lo + hi), lo, hi) == pytest.approx(0.5, abs=1e-15)
    x = np.linspace(lo - 1, hi + 1, 401)
    # odd quintic around the midpoint: f(lo + hi - x) = 1 - f(x)
    np.testing.assert_allclose(ftrans.f_trans(lo + hi - x, lo, hi), 1.0 - ftrans.f_trans(x, lo, hi), atol=1e-14)
    assert np.all(np.diff(ftrans.f_trans(x, lo, hi)) <= 1e-15)


def test_ftrans_is_C2():
    lo, hi = 2.0, 4.0
    for x0 in (lo, hi):
        for h in (1e-3, 1e-4):
            assert abs(ftrans.f_trans_deriv(x0 + h, lo, hi)) < 30 * h * h
            assert abs(ftrans.f_trans_deriv(x0 - h, lo, hi)) < 30 * h * h
            assert abs(ftrans.f_trans_deriv2(x0 + h, lo, hi)) < 30 * h
            assert abs(ftrans.f_trans_deriv2(x0 - h, lo, hi)) < 30 * h
    x = np.linspace(2.01, 3.99, 57)
    h = 1e-6
    fd = (ftrans.f_trans(x + h, lo, hi) - ftrans.f_trans(x - h, lo, hi)) / (2 * h)
    np.testing.assert_allclose(ftrans.f_trans_deriv(x, lo, hi), fd, atol=1e-8)
    fd2 = (ftrans.f_trans_deriv(x + h, lo, hi) - ftrans.f_trans_deriv(x - h, lo, hi)) / (2 * h)
    np.testing.assert_allclose(ftrans.f_trans_deriv2(x, lo, hi), fd2, atol=1e-7)


# ------------------------------------------------------------ radial basis
def test_radial_is_chebyshev_times_cutoff():
    p = dict(rc=5.0, rc_width=1.0, n_max=8)
    r = np.linspace(0.3, 5.2, 101)
    R, dR = ace.radial(r, p)
    x = 1.0 - 2.0 * r / 5.0
    fc = ftrans.f_trans(r, 4.0, 5.0)
    for n in range(8):
        c = np.zeros(n + 1)
        c[n] = 1.0
        np.testing.assert_allclose(R[:, n], np.polynomial.chebyshev.chebval(x, c) * fc, atol=1e-13)
    h = 1e-6
    Rp, _ = ace.radial(r + h, p)
    Rm, _ = ace.radial(r - h, p)
    np.testing.assert_allclose(dR, (Rp - Rm) / (2 * h), atol=1e-7)


# ------------------------------------------------------ spherical harmonics
def _unit(n, seed):
    u = np.random.default_rng(seed).normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1)[:, None]


def test_real_ylm_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    u = _unit(64, 0)
    u[0] = [0.0, 0.0, 1.0]
    u[1] = [0.0, 0.0, -1.0]
    u[2] = [1.0, 0.0, 0.0]
    Y = ace.sph_harm_real(u, 6)
    th = np.arccos(np.clip(u[:, 2], -1, 1))
    ph = np.arctan2(u[:, 1], u[:, 0])
    for l in range(7):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), th, ph)
            if m == 0:
                ref = c.real
            elif m > 0:
                ref = math.sqrt(2) * (-1) ** m * c.real
            else:
                ref = math.sqrt(2) * (-1) ** m * c.imag
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, atol=1e-13)


def test_real_ylm_orthonormal_by_quadrature():
    L = 5
    zg, wz = np.polynomial.legendre.leggauss(12)
    nph = 24
    ph = 2 * np.pi * np.arange(nph) / nph
    Z, PH = np.meshgrid(zg, ph, indexing="ij")
    st = np.sqrt(1 - Z**2)
    u = np.stack([(st * np.cos(PH)).ravel(), (st * np.sin(PH)).ravel(), Z.ravel()], 1)
    wt = np.outer(wz, np.full(nph, 2 * np.pi / nph)).ravel()
    Y = ace.sph_harm_real(u, L)
    np.testing.assert_allclose(Y.T @ (wt[:, None] * Y), np.eye((L + 1) ** 2), atol=1e-13)


def test_ylm_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    rv = rng.normal(size=(40, 3)) * 2.0
    Y, dY = ace.sph_harm_real_grad_r(rv, 4)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        up = ace.sph_harm_real((rv + e) / np.linalg.norm(rv + e, axis=1)[:, None], 4)
        dn = ace.sph_harm_real((rv - e) / np.linalg.norm(rv - e, axis=1)[:, None], 4)
        np.testing.assert_allclose(dY[:, :, c], (up - dn) / (2 * h), atol=1e-8)


# ------------------------------------------------------------------- Gaunt
def test_gaunt_matches_sympy_real_gaunt():
    wig = pytest.importorskip("sympy.physics.wigner")
    G = ace.gaunt_table(3, 3, 4)
    checked = 0
    for (l1, l2, l3), g in G.items():
        for m1, m2, m3 in itertools.product(range(-l1, l1 + 1), range(-l2, l2 + 1), range(-l3, l3 + 1)):
            ref = float(wig.real_gaunt(l1, l2, l3, m1, m2, m3))
            assert g[m1 + l1, m2 + l2, m3 + l3] == pytest.approx(ref, abs=1e-14)
            checked += 1
    assert checked > 5000


def test_gaunt_product_expansion():
    """Y_l1m1 Y_l2m2 = sum_{l3 m3} G(l1m1, l2m2, l3m3) Y_l3m3 (completeness)."""
    G = ace.gaunt_table(3, 3, 6)
    u = _unit(30, 5)
    Y = ace.sph_harm_real(u, 6)
    for l1 in range(4):
        for l2 in range(4):
            for m1 in range(-l1, l1 + 1):
                for m2 in range(-l2, l2 + 1):
                    lhs = Y[:, l1 * l1 + l1 + m1] * Y[:, l2 * l2 + l2 + m2]
                    rhs = np.zeros(len(u))
                    for l3 in range(7):
                        g = G[(l1, l2, l3)][m1 + l1, m2 + l2]
                        rhs += Y[:, l3 * l3:(l3 + 1) ** 2] @ g
                    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


# --------------------------------------------------------------- basis
def test_basis_counts():
    nm, lm = 6, 3
    b = ace.enumerate_basis(nm, lm, 3)
    assert sum(1 for x in b if x[0] == 1) == nm
    assert sum(1 for x in b if x[0] == 2) == (lm + 1) * nm * (nm + 1) // 2
    # nu=3 recount from ordered triples: sorted triples of distinct/equal pairs
    P = [(n, l) for n in range(1, nm + 1) for l in range(lm + 1)]
    cnt = 0
    for a in range(len(P)):
        for bb in range(a, len(P)):
            for c in range(bb, len(P)):
                ls = sorted([P[a][1], P[bb][1], P[c][1]])
                if sum(ls) % 2 == 0 and ls[2] <= ls[0] + ls[1]:
                    cnt += 1
    assert sum(1 for x in b if x[0] == 3) == cnt
    assert len(b) == 1048


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def _ace_model(nm=4, lm=3, nu=4, seed=11, a_scale=0.3):
    nb = len(ace.enumerate_basis(nm, lm, nu))
    return ace.AceModel(W.ace_params(nm, lm, nu, seed, nb, a_scale=a_scale))


@pytest.mark.parametrize("nu", [3, 4])
def test_ace_product_basis_rotation_invariant(nu):
    m = _ace_model(nu=nu)
    rng = np.random.default_rng(2)
    env = rng.normal(size=(25, 3)) * 1.5
    env = env[np.linalg.norm(env, axis=1) < 4.8]
    for seed in range(3):
        Rm = _rot(seed)
        out = []
        for rv in (env, env @ Rm.T, env[::-1]):
            r = np.linalg.norm(rv, axis=1)
            A, *_ = m.densities(1, np.zeros(len(r), np.int64), rv, r)
            B, _ = m.products(A)
            out.append(B[0])
        scale = np.abs(out[0]).max()
        np.testing.assert_allclose(out[1], out[0], atol=1e-12 * scale)
        np.testing.assert_allclose(out[2], out[0], atol=1e-12 * scale)
        # basis functions are not identically zero
        assert np.count_nonzero(np.abs(out[0]) > 1e-10 * scale) > 0.9 * len(out[0])


def test_ace_single_atom_energy_gradient_fd():
    """dE_i/dr_j of one ACE environment against central finite differences."""
    m = _ace_model(nu=4)
    rng = np.random.default_rng(4)
    env = rng.normal(size=(14, 3)) * 1.6
    env = env[np.linalg.norm(env, axis=1) < 4.9]
    pos = np.vstack([np.zeros(3), env]) + 10.0
    box = np.array([40.0, 40.0, 40.0])
    n = len(pos)
    i, j, rv, r = neighbors.pairs_bruteforce(pos, box, 5.0)
    E, F = ace.ace_energy_forces(m, n, i, j, rv, r, np.array([0]), weights=np.array([1.0]))
    h = 1e-5
    for a in range(n):
        for c in range(3):
            pp = pos.copy()
            pp[a, c] += h
            pm = pos.copy()
            pm[a, c] -= h
            ep = ace.ace_energy_forces(m, n, *neighbors.pairs_bruteforce(pp, box, 5.0), np.array([0]))[0][0]
            em = ace.ace_energy_forces(m, n, *neighbors.pairs_bruteforce(pm, box, 5.0), np.array([0]))[0][0]
            assert F[a, c] == pytest.approx(-(ep - em) / (2 * h), abs=2e-7)
    np.testing.assert_allclose(F.sum(axis=0), 0.0, atol=1e-12)


# --------------------------------------------------------------------- EAM
def test_eam_dimer_closed_form():
    p = dict(W.EAM)
    for rr in (2.3, 3.0, 4.1, 4.3, 4.5):
        pos = np.array([[5.0, 5.0, 5.0], [5.0 + rr, 5.0, 5.0]])
        box = np.array([30.0, 30.0, 30.0])
        i, j, rv, r = neighbors.pairs_bruteforce(pos, box, 5.0)
        E, z = eam.eam_energies(2, i, j, r, p)
        fc = ftrans.f_trans(rr, p["rc"] - p["rc_width"], p["rc"])
        rho = p["A"] * math.exp(-p["beta"] * (rr - p["r_e"])) * fc
        ex = math.exp(-p["alpha"] * (rr - p["r_0"]))
        phi = p["D"] * (ex * ex - 2 * ex) * fc
        ref = (-math.sqrt(rho) if rho > 0 else 0.0) + 0.5 * phi
        np.testing.assert_allclose(E, [ref, ref], atol=1e-15)
        np.testing.assert_allclose(z, [rho, rho], atol=1e-15)


def test_eam_forces_fd_weighted():
    s = W.vacancy_crystal(cells=4, sigma=0.08, seed=9)
    pos, box = s["pos"], s["box"]
    n = len(pos)
    u = np.random.default_rng(1).uniform(0, 1, n)
    p = W.EAM

    def etot(x):
        i, j, rv, r = neighbors.pairs_bruteforce(x, box, 4.5)
        e, _ = eam.eam_energies(n, i, j, r, p)
        return math.fsum(u * e)

    i, j, rv, r = neighbors.pairs_bruteforce(pos, box, 4.5)
    _, z = eam.eam_energies(n, i, j, r, p)
    F = eam.eam_forces(n, i, j, rv, r, z, u, p)
    h = 1e-5
    for a in (0, 7, 33, 64, 100):
        for c in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, c] += h
            pm[a, c] -= h
            assert F[a, c] == pytest.approx(-(etot(pp) - etot(pm)) / (2 * h), abs=1e-7)


# --------------------------------------------------------------- neighbours
def test_neighbors_kdtree_equals_bruteforce():
    s = W.vacancy_crystal(cells=5, sigma=0.1, seed=3)
    a = neighbors.pairs_bruteforce(s["pos"], s["box"], 5.0)
    b = neighbors.pairs_kdtree(s["pos"], s["box"], 5.0)
    sa = set(zip(a[0].tolist(), a[1].tolist()))
    sb = set(zip(b[0].tolist(), b[1].tolist()))
    assert sa == sb and len(sa) > 1000
    # a few hand-placed pairs across the periodic boundary
    pos = np.array([[0.1, 0.1, 0.1], [9.9, 0.1, 0.1], [5.0, 5.0, 5.0]])
    i, j, rv, r = neighbors.pairs_bruteforce(pos, np.array([10.0, 10.0, 10.0]), 1.0)
    assert sorted(zip(i.tolist(), j.tolist())) == [(0, 1), (1, 0)]
    np.testing.assert_allclose(sorted(r), [0.2, 0.2], atol=1e-12)


# --------------------------------------------------------------------- CSP
def test_csp_perfect_bcc_is_zero_and_pairs_are_opposite():
    pos, box = W.bcc(4, 4, 4)
    ids = np.arange(len(pos))
    part = csp.init_pairs(pos, box, ids, 4.5)
    assert np.all(part >= 0)
    g = csp.csp_g(pos, box, ids, part)
    np.testing.assert_allclose(g, 0.0, atol=1e-20)
    u, ia, ib, valid = csp.pair_vectors(pos, box, ids, part)
    ra = neighbors.min_image(pos[ia] - pos[:, None, :], box)
    np.testing.assert_allclose(np.linalg.norm(ra, axis=2), math.sqrt(3) * W.LATTICE_A / 2, atol=1e-12)


def test_csp_hand_example():
    """Atom 0 with 8 neighbours; one displaced by a known vector."""
    a = 1.0
    corners = np.array(list(itertools.product((-a, a), repeat=3)), dtype=float)
    pos = np.vstack([np.zeros(3), corners]) + 10.0
    shift = np.array([0.1, -0.2, 0.05])
    pos[1] += shift
    box = np.array([40.0, 40.0, 40.0])
    ids = np.arange(9) + 100          # ids need not start at 0
    part = csp.init_pairs(pos, box, ids, 2.0)
    g = csp.csp_g(pos, box, ids, part)
    # only the pair containing the shifted corner deviates: |shift|^2
    assert g[0] == pytest.approx(float(shift @ shift), abs=1e-14)


def test_csp_force_fd():
    s = W.vacancy_crystal(cells=4, sigma=0.08, seed=5)
    pos, box, ids = s["pos"], s["box"], s["ids"]
    part = csp.init_pairs(pos, box, ids, 4.5)
    c = np.random.default_rng(0).normal(size=len(pos))
    F = csp.csp_force(pos, box, ids, part, c)
    h = 1e-6
    for a in (0, 9, 50):
        for k in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, k] += h
            pm[a, k] -= h
            fd = -(c @ csp.csp_g(pp, box, ids, part) - c @ csp.csp_g(pm, box, ids, part)) / (2 * h)
            assert F[a, k] == pytest.approx(fd, abs=1e-7)
    np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-11)


# ------------------------------------------------------------------ switch
def test_descriptor_constant_g_and_hand_example():
    p = dict(r_w=3.0, r_w_width=1.0, d_lo=0.5, d_hi=1.5, d0=0.25)
    pos = np.array([[0.0, 0, 0], [1.5, 0, 0], [0, 2.5, 0], [7.0, 7.0, 7.0]]) + 5.0
    box = np.array([30.0, 30.0, 30.0])
    i, j, rv, r = neighbors.pairs_bruteforce(pos, box, 3.0)
    g = np.full(4, 0.9)
    wbar, d, lam, dlam = switch.descriptor(4, i, j, r, g, p)
    np.testing.assert_allclose(d, 0.9 - 0.25, atol=1e-15)      # average of a constant
    assert wbar[3] == 1.0                                     # isolated: self weight only
    g = np.array([0.0, 1.0, 2.0, 5.0])
    wbar, d, lam, dlam = switch.descriptor(4, i, j, r, g, p)
    w01 = 1.0                                                 # r = 1.5 <= r_w - 1
    w02 = float(ftrans.f_trans(2.5, 2.0, 3.0))
    w12 = float(ftrans.f_trans(math.hypot(1.5, 2.5), 2.0, 3.0))
    assert wbar[0] == pytest.approx(1 + w01 + w02)
    assert d[0] == pytest.approx((0 + 1 * w01 + 2 * w02) / (1 + w01 + w02) - 0.25)
    assert d[1] == pytest.approx((1 + 0 * w01 + 2 * w12) / (1 + w01 + w12) - 0.25)
    assert d[3] == pytest.approx(5 - 0.25)
    assert lam[3] == 1.0 and dlam[3] == 0.0                   # d > d_hi -> ACE
    assert lam[0] == pytest.approx(1 - float(ftrans.f_trans(d[0], 0.5, 1.5)))


def test_indenter_closed_form_and_gradient():
    """The indenter of the indentation workload: E = K/3 (R - r)^3 inside the sphere,
    zero outside, F = -grad E (central differences), continuous at r = R."""
    from oracle import indenter
    box = np.array([30.0, 30.0, 30.0])
    c = np.array([15.0, 15.0, 15.0])
    pos = np.array([[15.0, 15.0, 12.0], [15.0, 17.5, 15.0], [22.0, 15.0, 15.0], [15.0, 15.0, 10.0001]])
    e, f = indenter.energy_forces(pos, box, c, 5.0, 10.0)
    np.testing.assert_allclose(e[0], 10.0 / 3.0 * 2.0 ** 3, rtol=1e-15)
    np.testing.assert_allclose(f[0], [0.0, 0.0, -10.0 * 2.0 ** 2], rtol=1e-15)
    assert e[2] == 0.0 and np.all(f[2] == 0.0)
    assert e[3] < 1e-11
    h = 1e-6
    for a in (0, 1, 3):
        for q in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, q] += h
            pm[a, q] -= h
            fd = -(indenter.energy_forces(pp, box, c, 5.0, 10.0)[0].sum()
                   - indenter.energy_forces(pm, box, c, 5.0, 10.0)[0].sum()) / (2 * h)
            assert abs(fd - f[a, q]) < 1e-6
