"""Closed-form pins of the oracle's ACE energy value (the precise model of Eq. 4;
the paper defines ACE only by reference, Appendix B and Eq. S14, so these pin
the reading's mathematics, not a number the paper prints).

When every neighbour of an atom lies on one line through it, at r_j along
s_j u (s_j = +1 or -1, u one unit vector), each atomic density is a multiple of
the harmonic itself, A_nlm = a rho_nl Y_lm(u) with rho_nl = sum_j s_j^l R_n(r_j)
(Y_lm(-u) = (-1)^l Y_lm(u)).  Rotating u onto z leaves every B unchanged and
keeps only m = 0, where Y_l0(z) = sqrt((2l+1)/4pi) and the real Gaunt
coefficient is the Legendre integral
    G0(l1, l2, l3) = 2 pi prod_k sqrt((2 l_k + 1)/4pi) int_{-1}^{1} P_l1 P_l2 P_l3 dx.
So, with y_l = sqrt((2l+1)/4pi):
    nu = 1:  a rho_n0 / sqrt(4 pi)
    nu = 2:  a^2 rho_n1l rho_n2l (2l+1)/4pi
    nu = 3:  a^3 G0(l1,l2,l3) prod rho_nklk y_lk
    nu = 4:  a^4 G0(l1,l2,L) G0(l3,l4,L) prod rho_nklk y_lk
and E = phi1 + (phi2^2 + eps^2)^(1/4) - sqrt(eps), phi_c = sum_b c_cb B_b.
For two neighbours in different directions the nu <= 2 functions follow from
the addition theorem, sum_m Y_lm(u1) Y_lm(u2) = (2l+1)/4pi P_l(u1 . u2).

The Legendre integrals and P_l come from numpy's Legendre module, the radial
basis from numpy's Chebyshev module: nothing here calls the oracle's harmonics,
Gaunt quadrature or product code.  The basis enumeration (which coefficient
belongs to which function, a convention of the reading) is taken from the
oracle and pinned separately by its counts.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import chebyshev as C
from numpy.polynomial import legendre as Lg

from oracle import ace, ftrans, neighbors
from paper_2512_07693_gb300 import workloads as W


def _radial(r, p):
    """R_n(r) = T_{n-1}(1 - 2r/rc) fc(r) from numpy's Chebyshev series."""
    fc = ftrans.f_trans(np.asarray([r]), p["rc"] - p["rc_width"], p["rc"])[0]
    x = 1.0 - 2.0 * r / p["rc"]
    return np.array([C.chebval(x, np.eye(p["n_max"])[n]) * fc for n in range(p["n_max"])])


def _g0(l1, l2, l3):
    """int Y_l1,0 Y_l2,0 Y_l3,0 dOmega through the Legendre product integral."""
    prod = Lg.legmul(Lg.legmul(np.eye(l1 + 1)[l1], np.eye(l2 + 1)[l2]), np.eye(l3 + 1)[l3])
    integral = 2.0 * prod[0]           # int_{-1}^{1} P_k dx = 2 delta_k0
    y = [math.sqrt((2 * l + 1) / (4 * math.pi)) for l in (l1, l2, l3)]
    return 2.0 * math.pi * y[0] * y[1] * y[2] * integral


def _closed_form_B(p, rho):
    """B_b of a collinear environment from rho[n-1, l] (module docstring)."""
    a = p["a_scale"]
    y = [math.sqrt((2 * l + 1) / (4 * math.pi)) for l in range(2 * p["l_max"] + 1)]
    out = []
    for nu, prs, L in ace.enumerate_basis(p["n_max"], p["l_max"], p["nu_max"]):
        ns = [q[0] - 1 for q in prs]
        ls = [q[1] for q in prs]
        amp = np.prod([rho[n, l] * y[l] for n, l in zip(ns, ls)])
        if nu == 1:
            out.append(a * rho[ns[0], 0] / math.sqrt(4 * math.pi))
        elif nu == 2:
            out.append(a * a * rho[ns[0], ls[0]] * rho[ns[1], ls[1]] * (2 * ls[0] + 1) / (4 * math.pi))
        elif nu == 3:
            out.append(a ** 3 * _g0(*ls) * amp)
        else:
            out.append(a ** 4 * _g0(ls[0], ls[1], L) * _g0(ls[2], ls[3], L) * amp)
    return np.array(out)


def _energy(p, B):
    phi1 = float(np.dot(p["c1"][: len(B)], B))
    phi2 = float(np.dot(p["c2"][: len(B)], B))
    return phi1 + (phi2 * phi2 + p["eps"] ** 2) ** 0.25 - math.sqrt(p["eps"])


def _oracle_e0(model, env):
    """E^ACE of an atom at the centre of a large box with neighbours at env."""
    box = np.array([60.0, 60.0, 60.0])
    pos = np.vstack([np.zeros(3), env]) + 30.0
    i, j, rv, r = neighbors.pairs_bruteforce(pos, box, model.p["rc"] + 0.5)
    E, _ = ace.ace_energy_forces(model, len(pos), i, j, rv, r, np.array([0]))
    return float(E[0])


def _model(nm, lm, nu, seed=2, a_scale=0.25):
    nb = len(ace.enumerate_basis(nm, lm, nu))
    return ace.AceModel(W.ace_params(nm, lm, nu, seed, nb, a_scale=a_scale))


@pytest.mark.parametrize("nm,lm,nu,a_scale", [(6, 3, 3, 0.25), (4, 3, 4, 0.25), (3, 2, 4, 0.7), (8, 4, 2, 0.4)])
def test_ace_energy_of_collinear_environments(nm, lm, nu, a_scale):
    """One neighbour, then three on a line through the atom (two on one side,
    one on the other, so odd and even l weight the radii differently), in a
    random direction: every basis function and E^ACE against the closed form."""
    m = _model(nm, lm, nu, a_scale=a_scale)
    p = m.p
    rng = np.random.default_rng(7 + nu)
    for radii, signs in (([2.6], [1]), ([2.45, 4.3, 3.1], [1, 1, -1]), ([4.6, 1.9], [-1, 1])):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        rho = np.zeros((nm, 2 * lm + 1))
        for r, s in zip(radii, signs):
            R = _radial(r, p)
            for l in range(lm + 1):
                rho[:, l] += (s ** l) * R
        env = np.array([s * r * u for r, s in zip(radii, signs)])
        Bc = _closed_form_B(p, rho)
        rv = env
        rr = np.linalg.norm(rv, axis=1)
        A, *_ = m.densities(1, np.zeros(len(rr), np.int64), rv, rr)
        Bo, _ = m.products(A)
        scale = np.abs(Bc).max()
        np.testing.assert_allclose(Bo[0], Bc, atol=1e-12 * scale, rtol=0)
        E = _energy(p, Bc)
        assert _oracle_e0(m, env) == pytest.approx(E, abs=1e-12 * max(1.0, abs(E)))


def test_ace_nu2_two_directions_addition_theorem():
    """Two neighbours at an angle: nu = 1 and nu = 2 functions from the addition
    theorem (numpy Legendre P_l)."""
    m = _model(6, 3, 2, a_scale=0.6)
    p = m.p
    a = p["a_scale"]
    rng = np.random.default_rng(11)
    for _ in range(4):
        u = rng.normal(size=(2, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        r = rng.uniform(1.8, 4.8, size=2)
        R1, R2 = _radial(r[0], p), _radial(r[1], p)
        c = float(u[0] @ u[1])
        ref = []
        for nu, prs, _ in ace.enumerate_basis(6, 3, 2):
            ns = [q[0] - 1 for q in prs]
            if nu == 1:
                ref.append(a * (R1[ns[0]] + R2[ns[0]]) / math.sqrt(4 * math.pi))
                continue
            l = prs[0][1]
            pl = Lg.legval(c, np.eye(l + 1)[l])
            n1, n2 = ns
            ref.append(a * a * (2 * l + 1) / (4 * math.pi) *
                       (R1[n1] * R1[n2] + R2[n1] * R2[n2] + (R1[n1] * R2[n2] + R2[n1] * R1[n2]) * pl))
        ref = np.array(ref)
        env = r[:, None] * u
        A, *_ = m.densities(1, np.zeros(2, np.int64), env, r)
        B, _ = m.products(A)
        np.testing.assert_allclose(B[0], ref, atol=1e-13 * np.abs(ref).max(), rtol=0)
        assert _oracle_e0(m, env) == pytest.approx(_energy(p, ref), abs=1e-12)


def test_ace_embedding_channels_enter_differently():
    """phi1 enters E linearly and phi2 through the smooth square root: with one
    neighbour and a single nonzero coefficient in each channel, E is
    c1 B_b + (c2^2 B_k^2 + eps^2)^(1/4) - sqrt(eps) (a swap of the channels, a
    wrong root or a dropped -sqrt(eps) changes it)."""
    m = _model(4, 2, 3)
    p = m.p
    rho = np.zeros((4, 5))
    R = _radial(2.7, p)
    for l in range(3):
        rho[:, l] = R
    Bc = _closed_form_B(p, rho)
    b, k = 3, 17
    m.c1[:] = 0.0
    m.c2[:] = 0.0
    m.c1[b] = 0.8
    m.c2[k] = -1.3
    env = np.array([[0.0, 2.7, 0.0]])
    ref = 0.8 * Bc[b] + ((1.3 * Bc[k]) ** 2 + p["eps"] ** 2) ** 0.25 - math.sqrt(p["eps"])
    assert _oracle_e0(m, env) == pytest.approx(ref, abs=1e-14)
    # an isolated atom: every B vanishes except none, so E = (eps^2)^(1/4) - sqrt(eps) = 0
    assert _oracle_e0(m, np.zeros((0, 3))) == pytest.approx(0.0, abs=1e-15)


def test_precise_model_dimer_total_energy_closed_form():
    """The whole oracle on a dimer with the constant switches (Appendix B):
    lam = 0 gives 2 E^EAM(r), lam = 1 with precise = EAM + ACE gives
    2 [E^EAM(r) + E^ACE(r)], each from its closed form."""
    from oracle import apip as oapip
    nb = len(ace.enumerate_basis(6, 3, 3))
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP), switch=dict(W.SWITCH),
               ace=W.ace_params(6, 3, 3, 2, nb))
    pe = prm["eam"]
    box = np.array([40.0, 40.0, 40.0])
    for rr in (2.4, 3.3, 4.25):
        pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0, 10.0 + rr]])
        fc = ftrans.f_trans(rr, pe["rc"] - pe["rc_width"], pe["rc"])
        rho_e = pe["A"] * math.exp(-pe["beta"] * (rr - pe["r_e"])) * fc
        ex = math.exp(-pe["alpha"] * (rr - pe["r_0"]))
        e_eam = -math.sqrt(rho_e) + 0.5 * pe["D"] * (ex * ex - 2 * ex) * fc
        rho = np.zeros((6, 7))
        R = _radial(rr, prm["ace"])
        for l in range(4):
            rho[:, l] = R
        e_ace = _energy(prm["ace"], _closed_form_B(prm["ace"], rho))
        ids = np.arange(2)
        r0 = oapip.energy_forces(pos, box, ids, None, prm, lam_mode="const0")
        r1 = oapip.energy_forces(pos, box, ids, None, prm, lam_mode="const1")
        assert r0["E"] == pytest.approx(2 * e_eam, abs=1e-12)
        assert r1["E"] == pytest.approx(2 * (e_eam + e_ace), abs=1e-12)
        # Newton's third law on the dimer, and the force along the bond is -dE/dr
        np.testing.assert_allclose(r1["F"].sum(axis=0), 0.0, atol=1e-12)
