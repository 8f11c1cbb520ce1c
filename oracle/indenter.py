"""Spherical indenter of the indentation workload (an external potential; not part
of the AP Hamiltonian).  Oracle: test infrastructure only.

For an atom at distance r = |x_i - c| < R from the centre c:
    E_i = K/3 (R - r)^3,        F_i = -dE_i/dx_i = K (R - r)^2 (x_i - c) / r.
With the centre moving at constant velocity v_c, dE/dt at fixed positions is
(sum_i F_i) . v_c, so H - W with W = int (sum_i F_i) . v_c dt is conserved.
"""
import numpy as np

from .neighbors import min_image


def energy_forces(pos, box, center, radius, k):
    """Per-atom energies and forces (n, 3) of the indenter."""
    d = min_image(np.asarray(pos, dtype=np.float64) - np.asarray(center, dtype=np.float64), box)
    r = np.sqrt(np.sum(d * d, axis=1))
    inside = r < radius
    e = np.zeros(len(d))
    f = np.zeros_like(d)
    gap = radius - r[inside]
    e[inside] = k / 3.0 * gap ** 3
    f[inside] = (k * gap ** 2 / r[inside])[:, None] * d[inside]
    return e, f
