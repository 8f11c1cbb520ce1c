"""Transition function f_trans (Eq. S1; used by Eq. 2, Eq. S3 and the weighting
function w(r) of Appendix B).  Oracle: test infrastructure only.

f_trans(x, lo, hi) is 1 for x <= lo and 0 for x >= hi.  In between it is an odd
quintic in the reduced coordinate t = (hi + lo - 2x) / (hi - lo), which runs
from +1 at x = lo to -1 at x = hi:

    f = 1/2 + (15/16) t - (5/8) t^3 + (3/16) t^5

(15/16 = 0.9375, 5/8 = 0.625, 3/16 = 0.1875 as printed in Eq. S1).  Its first
and second derivatives vanish at both ends, so f is C^2.
"""
import numpy as np


def _reduced(x, lo, hi):
    return (hi + lo - 2.0 * np.asarray(x, dtype=np.float64)) / (hi - lo)


def f_trans(x, lo, hi):
    """Eq. S1: value of the transition function (array in, array out)."""
    x = np.asarray(x, dtype=np.float64)
    t = _reduced(x, lo, hi)
    mid = 0.5 + 0.9375 * t - 0.625 * t**3 + 0.1875 * t**5
    return np.where(x <= lo, 1.0, np.where(x >= hi, 0.0, mid))


def f_trans_deriv(x, lo, hi):
    """d f_trans / d x from Eq. S1 by the chain rule (dt/dx = -2/(hi-lo))."""
    x = np.asarray(x, dtype=np.float64)
    t = _reduced(x, lo, hi)
    dfdt = 0.9375 - 1.875 * t**2 + 0.9375 * t**4
    mid = dfdt * (-2.0 / (hi - lo))
    return np.where((x <= lo) | (x >= hi), 0.0, mid)


def f_trans_deriv2(x, lo, hi):
    """Second derivative of Eq. S1 (used only to pin its C^2 property)."""
    x = np.asarray(x, dtype=np.float64)
    t = _reduced(x, lo, hi)
    d2fdt2 = -3.75 * t + 3.75 * t**3
    mid = d2fdt2 * (2.0 / (hi - lo)) ** 2
    return np.where((x <= lo) | (x >= hi), 0.0, mid)
