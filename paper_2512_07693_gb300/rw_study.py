"""Synthetic analogue of the paper's error study against the averaging radius
(Fig. 3): on the void crystal, the adaptive-precision energies and forces are
compared with the precise model evaluated on every atom, for several cutoffs
r_w of the weighting function w (Eq. 6, Appendix B), on the atoms that the CSP
descriptor marks as defective (g_i > 1.5 A^2, the paper's selector threshold;
here the void's surface atoms).

The force error is split as in Fig. 3: the fast-model part (the AP force
without its grad-lambda term against the precise force), the grad-lambda part
(the AP force minus the force without it) and the full AP force.  The synthetic
precise model (EAM + random ACE) differs from the EAM by a constant dE^(0) per
atom even in the perfect crystal, where the paper's two fitted potentials agree;
through (E^prec - E^EAM) grad lam that offset alone makes a grad-lambda force.
Each radius is therefore evaluated twice: as defined (prec_shift = 0) and with
the precise model's energy zero aligned to the EAM's (prec_shift = dE^(0)),
which moves no force of either model.  Energies are compared with the constant
offset removed.  Float64 path, one configuration.

Usage: python -m paper_2512_07693_gb300.rw_study [--cells 24] [--rw 4 5 6 7 8]
"""
import argparse
import json

import numpy as np

from . import apip, workloads as W


def _eval(torch, s, prm, lam_mode, grad_lambda, max_nb):
    dev = torch.device("cuda")
    n = len(s["pos"])
    m = apip.Apip(prm, n, precision="fp64", lam_mode=lam_mode, grad_lambda=grad_lambda, max_nb=max_nb,
                  cell_cap=128)
    pos = torch.tensor(s["pos"], dtype=torch.float64, device=dev)
    ids = torch.tensor(s["ids"], dtype=torch.int32, device=dev)
    types = torch.zeros(n, dtype=torch.int32, device=dev)
    box = [float(x) for x in s["box"]]
    if lam_mode == "paper":
        m.init_csp_pairs(pos, box, ids)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    m.energy_forces(pos, box, types, ids, F, e)
    m.sync()
    out = dict(F=F.cpu().numpy(), e=e.cpu().numpy(), lam=m.field("lam", n).cpu().numpy(),
               g=m.field("g", n).cpu().numpy(), e_eam=m.field("e_eam", n).cpu().numpy())
    m.close()
    return out


def bulk_offset(torch, prm, cells=10):
    """dE^(0): mean E_i^prec - E_i^EAM over a perfect 0 K bcc crystal."""
    pos, box = W.bcc(cells, cells, cells)
    c = W._finish(pos, np.zeros_like(pos), box)
    r = _eval(torch, c, prm, "const1", True, 96)
    return float(np.mean(r["e"] - r["e_eam"]))


def study(torch, cells, radii):
    s = W.config("void250k", apip.apip_ace_basis_size, scale=cells)
    base = s["prm"]
    rows = []
    de0 = bulk_offset(torch, base)
    for rw in radii:
        # list capacity for the sphere of radius r_w + skin (bcc: 2 atoms per a^3) with margin
        r_list = max(rw, base["ace"]["rc"], base["eam"]["rc"]) + 0.5
        max_nb = min(256, int(1.3 * 4.18879 * r_list ** 3 * 2 / W.LATTICE_A ** 3) + 16)
        row = dict(r_w=rw)
        for tag, shift in (("", 0.0), ("aligned_", de0)):
            prm = dict(base, switch=dict(base["switch"], r_w=float(rw)), prec_shift=shift)
            ref = _eval(torch, s, prm, "const1", True, max_nb)
            ap = _eval(torch, s, prm, "paper", True, max_nb)
            nog = _eval(torch, s, prm, "paper", False, max_nb)
            sel = np.flatnonzero(ap["g"] > 1.5)
            # -(1 - lam_i)(dE_i - dE^(0)): the constant offset removed (already so when aligned)
            err_e = ap["e"] - ref["e"] + (1.0 - ap["lam"]) * (de0 - shift)
            rms = lambda f: float(np.sqrt(np.mean(f[sel] ** 2)))
            row.update({"atoms_selected": int(len(sel)), "x": float((ap["lam"] > 0).mean()),
                        tag + "rmse_e_ev": rms(err_e[:, None]),
                        tag + "rmse_f_ev_per_a": rms(ap["F"] - ref["F"]),
                        tag + "rmse_f_fast_model_part_ev_per_a": rms(nog["F"] - ref["F"]),
                        tag + "rmse_f_grad_lambda_part_ev_per_a": rms(ap["F"] - nog["F"]),
                        tag + "rmse_f_all_atoms_ev_per_a": float(np.sqrt(np.mean((ap["F"] - ref["F"]) ** 2)))})
        rows.append(row)
    return dict(workload=f"void recipe at {cells}^3 cells ({len(s['pos'])} atoms)", bulk_offset_ev=de0, rows=rows)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=24)
    ap.add_argument("--rw", type=float, nargs="+", default=[4.0, 5.0, 6.0, 7.0, 8.0])
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    print(json.dumps(study(torch, args.cells, args.rw)))


if __name__ == "__main__":
    main()
