"""Embedded-atom model, the fast potential (Eq. B1 = Eq. S7, S8; forces S9-S12).
Oracle: test infrastructure only.

    E_i^EAM = xi(zeta_i) + 1/2 sum_{j != i} Phi(r_ij),   zeta_i = sum_{j != i} rho(r_ij)

Analytic forms (the paper's W EAM is not available; these are the synthetic
forms of the workload definition: exponential density, Morse pair, square-root
embedding), each multiplied by the smooth cutoff fc(r) = f_trans(r, rc - width, rc):

    rho(r) = A exp(-beta (r - r_e)) fc(r)
    Phi(r) = D [exp(-2 alpha (r - r_0)) - 2 exp(-alpha (r - r_0))] fc(r)
    xi(z)  = -sqrt(z)            (xi = xi' = 0 for z <= 0: an isolated atom)
"""
import numpy as np

from .ftrans import f_trans, f_trans_deriv


def fc(r, p):
    return f_trans(r, p["rc"] - p["rc_width"], p["rc"])


def fc_deriv(r, p):
    return f_trans_deriv(r, p["rc"] - p["rc_width"], p["rc"])


def rho(r, p):
    return p["A"] * np.exp(-p["beta"] * (r - p["r_e"])) * fc(r, p)


def rho_deriv(r, p):
    e = p["A"] * np.exp(-p["beta"] * (r - p["r_e"]))
    return -p["beta"] * e * fc(r, p) + e * fc_deriv(r, p)


def phi(r, p):
    x = np.exp(-p["alpha"] * (r - p["r_0"]))
    return p["D"] * (x * x - 2.0 * x) * fc(r, p)


def phi_deriv(r, p):
    x = np.exp(-p["alpha"] * (r - p["r_0"]))
    m = p["D"] * (x * x - 2.0 * x)
    dm = p["D"] * (-2.0 * p["alpha"] * x * x + 2.0 * p["alpha"] * x)
    return dm * fc(r, p) + m * fc_deriv(r, p)


def xi(z):
    z = np.asarray(z, dtype=np.float64)
    return np.where(z > 0.0, -np.sqrt(np.maximum(z, 0.0)), 0.0)


def xi_deriv(z):
    z = np.asarray(z, dtype=np.float64)
    safe = np.where(z > 0.0, z, 1.0)
    return np.where(z > 0.0, -0.5 / np.sqrt(safe), 0.0)


def eam_energies(n, i, j, r, p):
    """Per-atom E_i^EAM (Eq. B1) and zeta_i (Eq. S8) from a full pair list."""
    inside = r < p["rc"]
    ii, rr = i[inside], r[inside]
    zeta = np.bincount(ii, weights=rho(rr, p), minlength=n)
    pair = np.bincount(ii, weights=phi(rr, p), minlength=n)
    return xi(zeta) + 0.5 * pair, zeta


def eam_forces(n, i, j, rvec, r, zeta, u, p):
    """F_i = -grad_i sum_k u_k E_k^EAM with the weights u held fixed.

    Differentiating E_k through zeta_k and the pair sum gives, for each pair
    (i, k) with unit vector e_ik = r_ik / r_ik pointing from i to k,

        F_i = sum_k (u_i a_ik + u_k a_ki) e_ik,   a_ik = xi'(zeta_i) rho'(r_ik) + Phi'(r_ik)/2,

    which is S10/S12 written with u = weight of the EAM energy (u = 1 - lam
    in the adaptive potential, u = 1 for pure EAM, S13).
    """
    inside = r < p["rc"]
    ii, jj, rv, rr = i[inside], j[inside], rvec[inside], r[inside]
    dxi = xi_deriv(zeta)
    drho = rho_deriv(rr, p)
    dphi = phi_deriv(rr, p)
    a_ij = dxi[ii] * drho + 0.5 * dphi
    a_ji = dxi[jj] * drho + 0.5 * dphi
    s = u[ii] * a_ij + u[jj] * a_ji
    f = (s / rr)[:, None] * rv
    F = np.zeros((n, 3))
    for c in range(3):
        F[:, c] = np.bincount(ii, weights=f[:, c], minlength=n)
    return F
