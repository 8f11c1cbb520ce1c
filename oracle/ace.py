"""Atomic cluster expansion (ACE), the precise potential.  Oracle: test
infrastructure only.

The paper uses ACE only by reference (Appendix B; Eq. S14 cites the ACE force
contributions from the literature).  This module writes out the standard linear
+ square-root ACE in its plainest form; every choice below is a reading of the
workload definition (Chebyshev radial basis, n_max, l_max, body order nu_max,
seeded N(0, 0.1) coefficients, linear + sqrt embedding):

  radial   R_n(r) = T_{n-1}(1 - 2 r / r_c) fc(r),   n = 1..n_max,
           fc(r) = f_trans(r, r_c - width, r_c)  (Eq. S1), independent of l
  angular  real orthonormal spherical harmonics Y_lm, l <= l_max, index l^2+l+m
           (Y_l0 = N_l0 P_l; m > 0: sqrt2 N_lm P~_l^m cos(m phi); m < 0: sin),
           P~ without the Condon-Shortley phase, N_lm = sqrt((2l+1)/4pi (l-m)!/(l+m)!)
  density  A_nlm = a_scale * sum_j R_n(r_ij) Y_lm(rhat_ij)
  product  basis B_b, enumerated in a fixed canonical order (``enumerate_basis``):
           nu=1: A_n00
           nu=2: sum_m A_{n1 l m} A_{n2 l m}                (n1 <= n2)
           nu=3: sum_m G(l1m1,l2m2,l3m3) A A A            (p1 <= p2 <= p3)
           nu=4: sum_{LM} [sum G(l1m1,l2m2,LM) A A][sum G(l3m3,l4m4,LM) A A]
           with G the real Gaunt coefficient int Y Y Y dOmega
  energy   phi1 = sum_b c1_b B_b, phi2 = sum_b c2_b B_b,
           E_i^ACE = phi1 + Fs(phi2),  Fs(x) = (x^2 + eps^2)^(1/4) - sqrt(eps)

(n, l) pairs are ordered by p = (n - 1)(l_max + 1) + l.  Fs is a smooth square
root (C-infinity, equal to sqrt|x| - sqrt(eps) for |x| >> eps).
"""
import itertools
import math

import numpy as np

from .ftrans import f_trans, f_trans_deriv


# ----------------------------------------------------------------- radial basis
def radial(r, p):
    """R[k, n-1] = R_n(r_k) and its r-derivative, n = 1..n_max."""
    r = np.asarray(r, dtype=np.float64)
    rc, nmax = p["rc"], p["n_max"]
    x = 1.0 - 2.0 * r / rc
    T = np.zeros((len(r), nmax))
    dT = np.zeros((len(r), nmax))
    T[:, 0] = 1.0
    if nmax > 1:
        T[:, 1] = x
        dT[:, 1] = 1.0
    for k in range(2, nmax):
        T[:, k] = 2.0 * x * T[:, k - 1] - T[:, k - 2]
        dT[:, k] = 2.0 * T[:, k - 1] + 2.0 * x * dT[:, k - 1] - dT[:, k - 2]
    f = f_trans(r, rc - p["rc_width"], rc)[:, None]
    df = f_trans_deriv(r, rc - p["rc_width"], rc)[:, None]
    R = T * f
    dR = dT * (-2.0 / rc) * f + T * df
    return R, dR


# ------------------------------------------------------- spherical harmonics
def _norm(l, m):
    return math.sqrt((2 * l + 1) / (4.0 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def sph_harm_real(u, lmax, grad=False):
    """Real orthonormal Y_lm at the rows of u (unit vectors) and, if ``grad``,
    the gradient of the polynomial extension P_lm(x, y, z) used to write them.

    Y_lm = N_lm Pi_l^m(z) C_m(x, y)  (m >= 0; S_m for m < 0), with
    C_m + i S_m = (x + i y)^m and Pi_l^m = P~_l^m(z) / (1 - z^2)^(m/2), which
    obeys the associated-Legendre recurrence in l.
    """
    u = np.asarray(u, dtype=np.float64)
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    K = len(u)
    nlm = (lmax + 1) ** 2
    Y = np.zeros((K, nlm))
    dY = np.zeros((K, nlm, 3))
    C = [np.ones(K)]
    S = [np.zeros(K)]
    for m in range(1, lmax + 1):
        C.append(x * C[m - 1] - y * S[m - 1])
        S.append(x * S[m - 1] + y * C[m - 1])
    for m in range(0, lmax + 1):
        # Pi_l^m for l = m..lmax and d/dz
        Pi = {m: np.full(K, float(np.prod(np.arange(2 * m - 1, 0, -2)) if m > 0 else 1.0))}
        dPi = {m: np.zeros(K)}
        if m + 1 <= lmax:
            Pi[m + 1] = (2 * m + 1) * z * Pi[m]
            dPi[m + 1] = (2 * m + 1) * (Pi[m] + z * dPi[m])
        for l in range(m + 2, lmax + 1):
            Pi[l] = ((2 * l - 1) * z * Pi[l - 1] - (l + m - 1) * Pi[l - 2]) / (l - m)
            dPi[l] = ((2 * l - 1) * (Pi[l - 1] + z * dPi[l - 1]) - (l + m - 1) * dPi[l - 2]) / (l - m)
        for l in range(m, lmax + 1):
            if m == 0:
                nrm = _norm(l, 0)
                Y[:, l * l + l] = nrm * Pi[l]
                dY[:, l * l + l, 2] = nrm * dPi[l]
                continue
            nrm = math.sqrt(2.0) * _norm(l, m)
            # m > 0 (cos)
            k = l * l + l + m
            Y[:, k] = nrm * Pi[l] * C[m]
            dY[:, k, 0] = nrm * Pi[l] * m * C[m - 1]
            dY[:, k, 1] = nrm * Pi[l] * (-m) * S[m - 1]
            dY[:, k, 2] = nrm * dPi[l] * C[m]
            # m < 0 (sin)
            k = l * l + l - m
            Y[:, k] = nrm * Pi[l] * S[m]
            dY[:, k, 0] = nrm * Pi[l] * m * S[m - 1]
            dY[:, k, 1] = nrm * Pi[l] * m * C[m - 1]
            dY[:, k, 2] = nrm * dPi[l] * S[m]
    if grad:
        return Y, dY
    return Y


def sph_harm_real_grad_r(rvec, lmax):
    """Y_lm(rhat) and its gradient with respect to the vector r:
    grad_r Y(r/|r|) = (I - rhat rhat^T) grad P(rhat) / |r|."""
    r = np.sqrt(np.einsum("ij,ij->i", rvec, rvec))
    u = rvec / r[:, None]
    Y, dP = sph_harm_real(u, lmax, grad=True)
    radial_part = np.einsum("kmc,kc->km", dP, u)
    dY = (dP - radial_part[:, :, None] * u[:, None, :]) / r[:, None, None]
    return Y, dY


# ------------------------------------------------------------- Gaunt table
def gaunt_table(lmax_a, lmax_b, lmax_c):
    """Real Gaunt coefficients G[(l1,l2,l3)][m1+l1, m2+l2, m3+l3] = int Y Y Y dOmega,
    by exact quadrature: Gauss-Legendre in z (exact to degree 2k-1) times the
    trapezoid rule in phi (exact for frequencies below the point count)."""
    L = lmax_a + lmax_b + lmax_c
    kz = L // 2 + 2
    nphi = L + 2
    zg, wz = np.polynomial.legendre.leggauss(kz)
    ph = 2.0 * math.pi * np.arange(nphi) / nphi
    Z, PH = np.meshgrid(zg, ph, indexing="ij")
    W = np.meshgrid(wz, np.full(nphi, 2.0 * math.pi / nphi), indexing="ij")
    wt = (W[0] * W[1]).ravel()
    st = np.sqrt(1.0 - Z**2)
    u = np.stack([(st * np.cos(PH)).ravel(), (st * np.sin(PH)).ravel(), Z.ravel()], axis=1)
    lmax = max(lmax_a, lmax_b, lmax_c)
    Y = sph_harm_real(u, lmax)
    out = {}
    for l1 in range(lmax_a + 1):
        for l2 in range(lmax_b + 1):
            for l3 in range(lmax_c + 1):
                y1 = Y[:, l1 * l1:(l1 + 1) ** 2]
                y2 = Y[:, l2 * l2:(l2 + 1) ** 2]
                y3 = Y[:, l3 * l3:(l3 + 1) ** 2]
                g = np.einsum("q,qa,qb,qc->abc", wt, y1, y2, y3)
                g[np.abs(g) < 1e-14] = 0.0
                out[(l1, l2, l3)] = g
    return out


# ---------------------------------------------------------- basis enumeration
def enumerate_basis(n_max, l_max, nu_max):
    """Canonical list of product-basis functions.

    Each entry is (nu, pairs, L) with pairs a tuple of (n, l), sorted by
    p = (n-1)(l_max+1) + l, and L the intermediate coupling (nu = 4 only, else -1):
      nu=1: (n, 0)                          for n = 1..n_max
      nu=2: p1 <= p2 with l1 == l2           (lexicographic in p)
      nu=3: p1 <= p2 <= p3, l1+l2+l3 even, |l1-l2| <= l3 <= l1+l2
      nu=4: p1 <= p2 <= p3 <= p4 and L with |l1-l2| <= L <= l1+l2,
            |l3-l4| <= L <= l3+l4, l1+l2+L and l3+l4+L even (ascending L)
    """
    P = [(n, l) for n in range(1, n_max + 1) for l in range(l_max + 1)]
    out = []
    if nu_max >= 1:
        for n in range(1, n_max + 1):
            out.append((1, ((n, 0),), -1))
    if nu_max >= 2:
        for a, b in itertools.combinations_with_replacement(range(len(P)), 2):
            if P[a][1] == P[b][1]:
                out.append((2, (P[a], P[b]), -1))
    if nu_max >= 3:
        for a, b, c in itertools.combinations_with_replacement(range(len(P)), 3):
            l1, l2, l3 = P[a][1], P[b][1], P[c][1]
            if (l1 + l2 + l3) % 2 == 0 and abs(l1 - l2) <= l3 <= l1 + l2:
                out.append((3, (P[a], P[b], P[c]), -1))
    if nu_max >= 4:
        for a, b, c, d in itertools.combinations_with_replacement(range(len(P)), 4):
            l1, l2, l3, l4 = P[a][1], P[b][1], P[c][1], P[d][1]
            for L in range(max(abs(l1 - l2), abs(l3 - l4)), min(l1 + l2, l3 + l4) + 1):
                if (l1 + l2 + L) % 2 == 0 and (l3 + l4 + L) % 2 == 0:
                    out.append((4, (P[a], P[b], P[c], P[d]), L))
    return out


# ----------------------------------------------------------------- evaluation
def _lm(l, m):
    return l * l + l + m


def _gaunt_terms(G, l1, l2, l3):
    """Nonzero entries of G(l1 m1, l2 m2, l3 m3) as index arrays into lm and values."""
    g = G[(l1, l2, l3)]
    a, b, c = np.nonzero(g)
    return (_lm(l1, a - l1), _lm(l2, b - l2), _lm(l3, c - l3), g[a, b, c])


class AceModel:
    """Basis tables for one (n_max, l_max, nu_max) and its coefficients."""

    def __init__(self, p):
        self.p = p
        self.basis = enumerate_basis(p["n_max"], p["l_max"], p["nu_max"])
        lm = p["l_max"]
        self.G = gaunt_table(lm, lm, 2 * lm if p["nu_max"] >= 4 else lm)
        c1 = np.asarray(p["c1"], dtype=np.float64)
        c2 = np.asarray(p["c2"], dtype=np.float64)
        assert len(c1) >= len(self.basis) and len(c2) >= len(self.basis)
        self.c1 = c1[: len(self.basis)]
        self.c2 = c2[: len(self.basis)]

    # B and dB/dA ------------------------------------------------------------
    def products(self, A, want_grad_weights=None):
        """B[atoms, nb] from A[atoms, n_max, nlm].  If ``want_grad_weights``
        (kappa[atoms, nb]) is given, also return omega = sum_b kappa_b dB_b/dA."""
        nat = A.shape[0]
        B = np.zeros((nat, len(self.basis)))
        kap = want_grad_weights
        om = np.zeros_like(A) if kap is not None else None
        for b, (nu, prs, L) in enumerate(self.basis):
            ns = [q[0] - 1 for q in prs]
            ls = [q[1] for q in prs]
            if nu == 1:
                B[:, b] = A[:, ns[0], 0]
                if kap is not None:
                    om[:, ns[0], 0] += kap[:, b]
            elif nu == 2:
                l = ls[0]
                sl = slice(l * l, (l + 1) ** 2)
                a1, a2 = A[:, ns[0], sl], A[:, ns[1], sl]
                B[:, b] = np.sum(a1 * a2, axis=1)
                if kap is not None:
                    om[:, ns[0], sl] += kap[:, b, None] * a2
                    om[:, ns[1], sl] += kap[:, b, None] * a1
            elif nu == 3:
                i1, i2, i3, g = _gaunt_terms(self.G, *ls)
                x1, x2, x3 = A[:, ns[0], i1], A[:, ns[1], i2], A[:, ns[2], i3]
                B[:, b] = (x1 * x2 * x3) @ g
                if kap is not None:
                    kg = kap[:, b, None] * g[None, :]
                    _scatter(om, ns[0], i1, kg * x2 * x3)
                    _scatter(om, ns[1], i2, kg * x1 * x3)
                    _scatter(om, ns[2], i3, kg * x1 * x2)
            else:
                t12 = _gaunt_terms(self.G, ls[0], ls[1], L)
                t34 = _gaunt_terms(self.G, ls[2], ls[3], L)
                nM = 2 * L + 1
                # left[atoms, M] = sum G A_{n1 l1 m1} A_{n2 l2 m2}
                x1, x2 = A[:, ns[0], t12[0]], A[:, ns[1], t12[1]]
                x3, x4 = A[:, ns[2], t34[0]], A[:, ns[3], t34[1]]
                M12 = t12[2] - L * L
                M34 = t34[2] - L * L
                left = np.zeros((nat, nM))
                right = np.zeros((nat, nM))
                for k in range(len(M12)):
                    left[:, M12[k]] += t12[3][k] * x1[:, k] * x2[:, k]
                for k in range(len(M34)):
                    right[:, M34[k]] += t34[3][k] * x3[:, k] * x4[:, k]
                B[:, b] = np.sum(left * right, axis=1)
                if kap is not None:
                    kr = kap[:, b, None] * right[:, M12] * t12[3][None, :]
                    kl = kap[:, b, None] * left[:, M34] * t34[3][None, :]
                    _scatter(om, ns[0], t12[0], kr * x2)
                    _scatter(om, ns[1], t12[1], kr * x1)
                    _scatter(om, ns[2], t34[0], kl * x4)
                    _scatter(om, ns[3], t34[1], kl * x3)
        return B, om

    def embed(self, B):
        eps = self.p["eps"]
        phi1 = B @ self.c1
        phi2 = B @ self.c2
        E = phi1 + (phi2 * phi2 + eps * eps) ** 0.25 - math.sqrt(eps)
        dF = 0.5 * phi2 * (phi2 * phi2 + eps * eps) ** (-0.75)
        return E, dF

    # densities ----------------------------------------------------------------
    def densities(self, n_at, i, rvec, r, grad=False):
        """A[atoms, n_max, nlm] from the pairs (i, rvec) with r < rc, i local."""
        p = self.p
        R, dR = radial(r, p)
        if grad:
            Y, dY = sph_harm_real_grad_r(rvec, p["l_max"])
        else:
            u = rvec / r[:, None]
            Y = sph_harm_real(u, p["l_max"])
            dY = None
        A = np.zeros((n_at, p["n_max"], Y.shape[1]))
        prod = R[:, :, None] * Y[:, None, :]
        flat = prod.reshape(len(r), p["n_max"] * Y.shape[1])
        Af = A.reshape(n_at, p["n_max"] * Y.shape[1])
        for c in range(flat.shape[1]):
            Af[:, c] = np.bincount(i, weights=flat[:, c], minlength=n_at)
        A *= p["a_scale"]
        return A, R, dR, Y, dY


def _scatter(om, n, idx, vals):
    """om[:, n, idx[k]] += vals[:, k] with repeated idx allowed."""
    for k in range(len(idx)):
        om[:, n, idx[k]] += vals[:, k]


def ace_energy_forces(model, n, i, j, rvec, r, atoms, weights=None):
    """E_i^ACE for the atoms listed in ``atoms`` and, if ``weights`` (one per
    listed atom) is given, F = -grad sum_i weights_i E_i^ACE over all n atoms.

    With r_ij = r_j - r_i and Ecal = sum_i v_i E_i:
    dE_i/dr_j = sum_nlm omega_i,nlm grad(R_n Y_lm)(r_ij) and dE_i/dr_i = -sum_j of it
    (force contributions f_ij of Eq. S14 / A1).
    """
    p = model.p
    atoms = np.asarray(atoms, dtype=np.int64)
    local = np.full(n, -1, dtype=np.int64)
    local[atoms] = np.arange(len(atoms))
    sel = (local[i] >= 0) & (r < p["rc"])
    li, jj, rv, rr = local[i[sel]], j[sel], rvec[sel], r[sel]
    want = weights is not None
    A, R, dR, Y, dY = model.densities(len(atoms), li, rv, rr, grad=want)
    B, _ = model.products(A)
    E, dF = model.embed(B)
    if not want:
        return E, None
    kappa = model.c1[None, :] + dF[:, None] * model.c2[None, :]
    kappa = kappa * np.asarray(weights, dtype=np.float64)[:, None]
    _, om = model.products(A, want_grad_weights=kappa)
    om = om * p["a_scale"]
    Om = om[li]                                     # [pairs, n_max, nlm]
    e = rv / rr[:, None]
    s1 = np.einsum("knl,kn,kl->k", Om, dR, Y)       # radial derivative part
    v2 = np.einsum("knl,kn,klc->kc", Om, R, dY)     # angular part
    fij = s1[:, None] * e + v2                      # d(sum_i v_i E_i)/d r_j per pair
    F = np.zeros((n, 3))
    gi = atoms[li]
    for c in range(3):
        F[:, c] -= np.bincount(jj, weights=fij[:, c], minlength=n)
        F[:, c] += np.bincount(gi, weights=fij[:, c], minlength=n)
    return E, F
