"""Conservative adaptive-precision energy and force (Eq. 4, Eq. 5 = Eq. S4).
Oracle: test infrastructure only.

    E   = sum_i [lam_i E_i^ACE + (1 - lam_i) E_i^EAM]                 (Eq. 4)
    F_i = -grad_i E                                                    (Eq. 5)
        = F^EAM (weights 1 - lam, Eq. S12) + F^ACE (weights lam, Eq. S14)
          + F^(grad lambda) (Eq. S15-S27)

lam is the ACE weight (the paper's lambda is 1 - lam).  ``lam_mode``:
  "paper"  lam_i = 1 - f_trans(d_i, d_lo, d_hi) from the CSP descriptor (Eq. 2, 6)
  "learned" the same switch with g_k = MLP(radial descriptors) (oracle/mlp.py,
           weights in prm["mlp"])
  "const0" lam = 0 everywhere (pure EAM)
  "const1" lam = 1 everywhere (pure ACE)
and ``lam_const`` (float array, NaN = follow Eq. 2) fixes lam on a subset
(Appendix B).  ``grad_lambda=False`` drops F^(grad lambda) (the non-conservative
ablation of Fig. 3b / Fig. S2).  ``mixing="force"`` replaces Eq. 5 by force
mixing (Eq. 3, the other ablation of Fig. 5): each atom's force is the
lam-weighted combination of the full fast and full precise forces,
    F_i = (1 - lam_i) F_i^EAM + lam_i F_i^prec,   F^m = -grad sum_k E_k^m,
which is not the gradient of any energy and violates Newton's third law.  The
reported energy is still Eq. 4.
"""
import math

import numpy as np

from . import ace as ace_mod
from . import mlp
from .csp import csp_g
from .eam import eam_energies, eam_forces
from .neighbors import pairs
from .switch import descriptor, grad_lambda_force


def cutoff(prm):
    return max(prm["eam"]["rc"], prm["ace"]["rc"], prm["switch"]["r_w"])


def energy_forces(pos, box, ids, partners, prm, model=None, lam_mode="paper",
                  lam_const=None, grad_lambda=True, forces=True, mixing="energy"):
    """Return a dict with E (fsum), per-atom terms and F (n, 3)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = len(pos)
    if model is None:
        model = ace_mod.AceModel(prm["ace"])
    i, j, rvec, r = pairs(pos, box, cutoff(prm))
    e_eam, zeta = eam_energies(n, i, j, r, prm["eam"])
    sw = prm["switch"]
    rc_a, w_a = prm["ace"]["rc"], prm["ace"]["rc_width"]
    if lam_mode == "paper":
        g = csp_g(pos, box, ids, partners)
        wbar, d, lam, dlam = descriptor(n, i, j, r, g, sw, lam_const)
    elif lam_mode == "learned":
        g, _, _ = mlp.learned_g(n, i, r, prm["mlp"], rc_a, w_a)
        wbar, d, lam, dlam = descriptor(n, i, j, r, g, sw, lam_const)
    else:
        val = {"const0": 0.0, "const1": 1.0}[lam_mode]
        g = np.zeros(n)
        wbar, d = np.ones(n), np.zeros(n)
        lam, dlam = np.full(n, val), np.zeros(n)
        if lam_const is not None:
            fixed = ~np.isnan(lam_const)
            lam = np.where(fixed, lam_const, lam)
    P = np.nonzero(lam > 0.0)[0]
    e_ace = np.zeros(n)
    F = np.zeros((n, 3))
    ace_e, ace_f = ace_mod.ace_energy_forces(model, n, i, j, rvec, r, P,
                                             weights=lam[P] if forces else None)
    e_ace[P] = ace_e
    beta = 1.0 if prm.get("precise_adds_eam", False) else 0.0
    # prm["prec_shift"]: the precise model's energy zero, a constant per atom
    e_prec = e_ace + beta * e_eam - prm.get("prec_shift", 0.0)
    e_atom = lam * e_prec + (1.0 - lam) * e_eam
    out = dict(E=math.fsum(e_atom), e_atom=e_atom, e_ace=e_ace, e_eam=e_eam,
               zeta=zeta, g=g, wbar=wbar, d=d, lam=lam, dlam=dlam, P=P)
    if not forces:
        return out
    if mixing == "force":
        f_fast = eam_forces(n, i, j, rvec, r, zeta, np.ones(n), prm["eam"])
        everyone = np.arange(n)
        _, f_ace = ace_mod.ace_energy_forces(model, n, i, j, rvec, r, everyone, weights=np.ones(n))
        f_prec = beta * f_fast + f_ace
        out["F"] = (1.0 - lam)[:, None] * f_fast + lam[:, None] * f_prec
        return out
    if mixing != "energy":
        raise ValueError(mixing)
    F += eam_forces(n, i, j, rvec, r, zeta, 1.0 - lam + beta * lam, prm["eam"])
    F += ace_f
    if grad_lambda and lam_mode in ("paper", "learned"):
        delta = e_prec - e_eam
        g_force = None
        if lam_mode == "learned":
            def g_force(c):
                return mlp.learned_force(n, i, j, rvec, r, prm["mlp"], c, rc_a, w_a)
        F += grad_lambda_force(n, i, j, rvec, r, g, d, wbar, dlam, delta, sw,
                               pos, box, ids, partners, g_force=g_force)
    out["F"] = F
    return out
