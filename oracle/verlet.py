"""Velocity-Verlet NVE integration (the integrator of the paper's NVE runs,
main text before Fig. 5).  Oracle: test infrastructure only.

Metal units: positions in Angstrom, velocities in Angstrom/ps, forces in eV/A,
masses in amu, time in ps.  MVV2E converts amu A^2/ps^2 to eV.
"""
import math

import numpy as np

from .apip import energy_forces
from .neighbors import wrap

MVV2E = 1.0364269e-4


def kinetic(vel, mass):
    return 0.5 * MVV2E * math.fsum((mass[:, None] * vel * vel).ravel())


def run(pos, vel, box, ids, partners, prm, mass, dt, steps, model=None, **kw):
    """Integrate ``steps`` velocity-Verlet steps; return final state and a
    per-step record of (E_pot, E_kin, total momentum)."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    inv = 1.0 / (mass * MVV2E)
    res = energy_forces(pos, box, ids, partners, prm, model=model, **kw)
    F = res["F"]
    log = [(res["E"], kinetic(vel, mass), (mass[:, None] * vel).sum(axis=0))]
    for _ in range(steps):
        vel += 0.5 * dt * F * inv[:, None]
        pos = wrap(pos + dt * vel, box)
        res = energy_forces(pos, box, ids, partners, prm, model=model, **kw)
        F = res["F"]
        vel += 0.5 * dt * F * inv[:, None]
        log.append((res["E"], kinetic(vel, mass), (mass[:, None] * vel).sum(axis=0)))
    return pos, vel, F, log
