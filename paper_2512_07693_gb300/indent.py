"""The indentation run: a 4 M-atom bcc slab under a moving spherical indenter,
advanced by NVE velocity Verlet with three force models on the same GPU:

  paper    adaptive precision with the paper's switch (CSP^list descriptor, Eq. 2, 6)
  learned  adaptive precision with the learned indicator g = MLP(radial descriptors),
           its switch window placed so that the ACE fraction x equals the paper
           switch's at the start
  ace      the precise model on every atom (lam = 1)

For each it reports atom-steps/s (CUDA events around the step calls), the ACE
fraction x at the start and the end, the drift of H - W (W the indenter's work,
which the library accumulates; H alone is not conserved while the indenter
moves), the change of the total momentum, and the per-atom energy error of the
final configuration against the precise model evaluated on every atom (the
constant bulk offset between the two models removed).

Usage: python -m paper_2512_07693_gb300.indent [--steps 5000] [--ace-steps 500]
       [--mlp weights.npy] [--cells N]
"""
import argparse
import json
import time

import numpy as np

from . import apip, workloads as W

MODES = {"paper": "paper", "learned": "learned", "ace": "const1"}


def _device(torch, s):
    dev = torch.device("cuda")
    n = len(s["pos"])
    return dict(pos=torch.tensor(s["pos"], dtype=torch.float64, device=dev),
                vel=torch.tensor(s["vel"], dtype=torch.float64, device=dev),
                ids=torch.tensor(s["ids"], dtype=torch.int32, device=dev),
                types=torch.zeros(n, dtype=torch.int32, device=dev),
                inv_mass=torch.tensor(1.0 / (s["mass"] * apip.MVV2E), dtype=torch.float64, device=dev),
                F=torch.empty((n, 3), dtype=torch.float64, device=dev),
                e=torch.empty(n, dtype=torch.float64, device=dev),
                lam_fixed=torch.tensor(s["lam_fixed"], dtype=torch.float64, device=dev))


def model(torch, s, arm, t, prm=None, mlp_flat=None, max_nb=80, cell_cap=48):
    """A library context for one arm, set up on the slab's initial positions
    (pinned surfaces, indenter, CSP pairs or network), forces evaluated."""
    prm = prm or s["prm"]
    n = len(s["pos"])
    m = apip.Apip(prm, n, precision="fp32", lam_mode=MODES[arm], max_nb=max_nb, cell_cap=cell_cap)
    if arm != "ace":
        m.set_lam_fixed(t["lam_fixed"])
    ind = s["indenter"]
    m.set_indenter(ind["center"], ind["velocity"], ind["radius"], ind["k"])
    box = [float(x) for x in s["box"]]
    if arm == "paper":
        m.init_csp_pairs(t["pos"], box, t["ids"])
    if arm == "learned":
        m.set_mlp(mlp_flat)
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"], t["e"])
    m.sync()
    return m, box


def learned_window(torch, s, t, mlp_flat, x_free):
    """(d_lo, d_hi) for the learned switch such that the fraction of the free
    (not pinned) atoms with lam > 0 is x_free: d_lo at the (1 - x_free) quantile of
    the learned descriptor d over the free atoms.  The width is half of d_lo (at
    least a quarter of d's spread): like the paper's window it scales with the
    descriptor values it separates, not with the spread of a nearly uniform
    crystal, which would make the switch, and the grad-lambda forces, stiff."""
    wide = dict(s["prm"], switch=dict(s["prm"]["switch"], d_lo=-1e3, d_hi=1e3))
    m, _ = model(torch, s, "learned", t, prm=wide, mlp_flat=mlp_flat)
    n = len(s["pos"])
    d = m.field("d", n).cpu().numpy()
    m.close()
    free = ~np.isfinite(s["lam_fixed"])
    lo = float(np.quantile(d[free], 1.0 - x_free))
    return lo, lo + max(0.5 * abs(lo), 0.25 * float(np.std(d[free])))


def bulk_offset(torch, prm, cells=10):
    """dE^(0): the mean of E_i^prec - E_i^EAM over a perfect 0 K bcc crystal, the
    constant by which the two models' per-atom energies differ in the bulk."""
    pos, box = W.bcc(cells, cells, cells)
    n = len(pos)
    dev = torch.device("cuda")
    m = apip.Apip(prm, n, precision="fp32", lam_mode="const1")
    e = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    m.energy_forces(torch.tensor(pos, device=dev), [float(b) for b in box], torch.zeros(n, dtype=torch.int32, device=dev),
                    torch.arange(n, dtype=torch.int32, device=dev), F, e)
    m.sync()
    d0 = float((e - m.field("e_eam", n)).mean())
    m.close()
    return d0


def run_arm(torch, s, arm, steps, chunk=100, dt=0.001, prm=None, mlp_flat=None, de0=0.0):
    t = _device(torch, s)
    n = len(s["pos"])
    m, box = model(torch, s, arm, t, prm=prm, mlp_flat=mlp_flat)
    lam0 = m.field("lam", n).cpu().numpy()
    steps = max(chunk, steps // chunk * chunk)
    thermo = torch.zeros((steps, 5), dtype=torch.float64, device="cuda")
    work = [0.0]
    stream = torch.cuda.current_stream()
    ms = 0.0
    for q in range(0, steps, chunk):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], dt, chunk,
                      thermo[q:q + chunk])
        b.record(stream)
        work.append(m.indenter_state()[1])   # synchronises
        ms += a.elapsed_time(b)
    m.sync()
    th = thermo.cpu().numpy()
    H = th[:, 0] + th[:, 1]
    Wk = np.interp(np.arange(1, steps + 1), np.arange(0, steps + 1, chunk), np.array(work))
    hw = (H - Wk) / n
    tps = np.arange(1, steps + 1) * dt
    lam1 = m.field("lam", n).cpu().numpy()
    # per-atom energy of the final configuration: this arm against lam = 1 everywhere
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"], t["e"])
    e_arm = t["e"].cpu().numpy()
    centre = m.indenter_state()[0]
    m.close()
    ref = apip.Apip(prm or s["prm"], n, precision="fp32", lam_mode="const1", max_nb=80, cell_cap=48)
    ind = s["indenter"]
    ref.set_indenter(centre, [0.0, 0.0, 0.0], ind["radius"], ind["k"])
    Fr = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    er = torch.empty(n, dtype=torch.float64, device="cuda")
    ref.energy_forces(t["pos"], box, t["types"], t["ids"], Fr, er)
    ref.sync()
    err = e_arm - er.cpu().numpy()
    ref.close()
    # E_i^AP - E_i^prec = -(1 - lam_i)(dE_i): without the bulk offset dE^(0), which
    # shifts every fast atom's energy by the same constant (no force, no dynamics)
    err_b = err + (1.0 - lam1) * de0
    contact = np.flatnonzero(lam1 > 0)
    return {
        "arm": arm, "atoms": n, "steps": steps, "atom_steps_per_s": n * steps / (ms * 1e-3),
        "ms_per_step": ms / steps,
        "x_start": float((lam0 > 0).mean()), "x_end": float((lam1 > 0).mean()),
        "drift_h_minus_w_ev_per_atom_ps": float(np.polyfit(tps, hw, 1)[0]),
        "h_minus_w_range_ev_per_atom": float(hw.max() - hw.min()),
        "indenter_work_ev": float(work[-1]), "indenter_depth_a": float(s["indenter"]["center"][2] - centre[2]),
        "momentum_change": [float(v) for v in th[-1, 2:] - th[0, 2:]],
        "energy_error_vs_ace_ev_per_atom": {
            "rms": float(np.sqrt(np.mean(err_b ** 2))), "max": float(np.abs(err_b).max()),
            "rms_where_lam_pos": float(np.sqrt(np.mean(err_b[contact] ** 2))) if len(contact) else 0.0,
            "bulk_offset_removed": de0, "rms_with_offset": float(np.sqrt(np.mean(err ** 2)))},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--ace-steps", type=int, default=500)
    ap.add_argument("--mlp", default=None, help="float32 flat network weights (.npy) for the learned arm")
    ap.add_argument("--cells", type=int, default=None)
    args = ap.parse_args()
    import torch
    from . import build
    build.build()
    t0 = time.time()
    s = W.config("indent4m", apip.apip_ace_basis_size, scale=args.cells)
    de0 = bulk_offset(torch, s["prm"])
    out = [run_arm(torch, s, "paper", args.steps, de0=de0)]
    if args.mlp:
        flat = torch.tensor(np.load(args.mlp).astype(np.float32), device="cuda")
        free = ~np.isfinite(s["lam_fixed"])
        x_free = out[0]["x_start"] * len(s["pos"]) / free.sum()
        lo, hi = learned_window(torch, s, _device(torch, s), flat, x_free)
        prm = dict(s["prm"], switch=dict(s["prm"]["switch"], d_lo=lo, d_hi=hi))
        r = run_arm(torch, s, "learned", args.steps, prm=prm, mlp_flat=flat, de0=de0)
        r["switch_window"] = [lo, hi]
        out.append(r)
    out.append(run_arm(torch, s, "ace", args.ace_steps, de0=de0))
    for r in out:
        r["speedup_vs_all_ace"] = r["atom_steps_per_s"] / out[-1]["atom_steps_per_s"]
    print(json.dumps({"workload": "indent4m" if args.cells is None else f"indent recipe at {args.cells} cells",
                      "arms": out, "wall_s": time.time() - t0}))


if __name__ == "__main__":
    main()
