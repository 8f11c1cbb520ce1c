"""Locally averaged descriptor and switching parameter (Eq. 6 = Eq. S2, Eq. 2 =
Eq. S3, w(r) of Appendix B) and the force from the gradient of the switch
(Eq. S15-S27).  Oracle: test infrastructure only.

    w(r)    = f_trans(r, r_w - width, r_w)                     (Appendix B)
    wbar_i  = sum_k w(r_ik)                                    (after Eq. 6)
    d_i     = sum_k g_k w(r_ik) / wbar_i - d0                  (Eq. 6)
    lam_i   = 1 - f_trans(d_i, d_lo, d_hi)                     (Eq. 2, ACE weight)

Reading: the sums over k include k = i with w(0) = 1 (the paper leaves the
self term open); this keeps wbar_i >= 1.  lam is the ACE weight, the paper's
lambda is 1 - lam.  Atoms may carry a constant lam (Appendix B, last
paragraph); for them dlam/dd = 0.
"""
import numpy as np

from .ftrans import f_trans, f_trans_deriv
from .csp import csp_force


def w(r, p):
    return f_trans(r, p["r_w"] - p["r_w_width"], p["r_w"])


def w_deriv(r, p):
    return f_trans_deriv(r, p["r_w"] - p["r_w_width"], p["r_w"])


def descriptor(n, i, j, r, g, p, lam_const=None):
    """Return wbar, d, lam, dlam (= d lam / d d) per atom.

    ``lam_const``: optional float array, NaN where lam follows Eq. 2 and the
    constant value elsewhere (Appendix B constant-switch atoms).
    """
    inside = r < p["r_w"]
    ii, jj, rr = i[inside], j[inside], r[inside]
    wij = w(rr, p)
    wbar = 1.0 + np.bincount(ii, weights=wij, minlength=n)
    s = g + np.bincount(ii, weights=g[jj] * wij, minlength=n)
    d = s / wbar - p["d0"]
    lam = 1.0 - f_trans(d, p["d_lo"], p["d_hi"])
    dlam = -f_trans_deriv(d, p["d_lo"], p["d_hi"])
    if lam_const is not None:
        fixed = ~np.isnan(lam_const)
        lam = np.where(fixed, lam_const, lam)
        dlam = np.where(fixed, 0.0, dlam)
    return wbar, d, lam, dlam


def grad_lambda_force(n, i, j, rvec, r, g, d, wbar, dlam, delta, p, pos, box, ids, partners, g_force=None):
    """F^(grad lambda) = -grad sum_k lam_k Delta_k with Delta_k = E_k^ACE - E_k^EAM
    held fixed (Eq. S15, written for lam = ACE weight).  ``g_force(c)`` returns
    -grad sum_j c_j g_j for the atomic quantity in use (default: CSP^list).

    Chain rule through Eq. 6: with Et_k = Delta_k (dlam/dd)_k / wbar_k (Eq. S17 up
    to the sign convention of lam) and D_k = d_k + d0,

        grad_i d_k wbar_k = sum_j [ w(r_kj) grad_i g_j + (g_j - D_k) grad_i w(r_kj) ].

    The w-part (Eq. S18-S21): for each pair (k, j), j != k, with e_kj = r_kj/r_kj,
    atom j receives -Et_k (g_j - D_k) w'(r_kj) e_kj and atom k the opposite.
    The g-part (Eq. S25-S27): c_j = sum_k Et_k w(r_kj) (k = j included with
    w = 1), then F -= grad sum_j c_j g_j through the CSP pair list.
    """
    Et = delta * dlam / wbar
    D = d + p["d0"]
    inside = r < p["r_w"]
    kk, jj, rv, rr = i[inside], j[inside], rvec[inside], r[inside]
    s = Et[kk] * (g[jj] - D[kk]) * w_deriv(rr, p)
    f = (s / rr)[:, None] * rv
    F = np.zeros((n, 3))
    for comp in range(3):
        F[:, comp] += np.bincount(kk, weights=f[:, comp], minlength=n)
        F[:, comp] -= np.bincount(jj, weights=f[:, comp], minlength=n)
    c = Et + np.bincount(jj, weights=Et[kk] * w(rr, p), minlength=n)
    F += csp_force(pos, box, ids, partners, c) if g_force is None else g_force(c)
    return F
