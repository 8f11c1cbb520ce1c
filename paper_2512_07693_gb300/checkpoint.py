"""Checkpoint and resume of an adaptive-precision MD run.

A run's state is the caller's arrays (positions, velocities, ids, types, inverse
masses), the box and the step count, plus three pieces the library holds: the
CSP^list partner ids, detected once at t = 0 and fixed by ID afterwards
(Appendix B); the positions the current neighbour list was built from, so that
the resumed run rebuilds the same list (same entries in the same order) and
triggers its next rebuild at the same step; and, with an indenter, its centre and
accumulated work.  With apip_params.deterministic set, a resumed run then
continues the trajectory bit for bit.  A resumed
run must reuse the saved partners (detecting them again at the resumed
configuration could pair atoms differently).  The parameters (the context's
apip_params, the network weights, a constant-lam mask) belong to the caller and
are given again when the context is created for the resumed run.  The format is a
numpy .npz archive.
"""
import numpy as np

STATE = ("pos", "vel", "ids", "types", "inv_mass")


def save(path, model, t, box, step, csp=True, indenter=False):
    """Write the state of ``model`` (an apip.Apip) and its device arrays ``t``
    (keys pos, vel, ids, types, inv_mass) after ``step`` steps."""
    n = t["pos"].shape[0]
    arrays = {k: t[k].detach().cpu().numpy() for k in STATE}
    arrays["box"] = np.asarray(box, dtype=np.float64)
    arrays["step"] = np.int64(step)
    if csp:   # rows by atom id, for every id in use
        rows = int(arrays["ids"].max()) + 1 if n else 0
        arrays["csp"] = model.field("csp", rows).cpu().numpy().astype(np.int32)
    if n:
        arrays["build_pos"] = model.field("build_pos", n).cpu().numpy()
    if indenter:
        centre, work = model.indenter_state()
        arrays["ind_centre"] = np.asarray(centre, dtype=np.float64)
        arrays["ind_work"] = np.float64(work)
    np.savez(path, **arrays)


def load(path):
    with np.load(path) as f:
        return {k: f[k] for k in f.files}


def resume(model, ck, device="cuda", indenter=None):
    """Device tensors of the saved state; restores the saved partner ids into
    ``model`` (a new context with the run's parameters), rebuilds its neighbour
    list from the saved build positions and, when ``indenter`` (dict of velocity,
    radius, k) is given, places the indenter at its saved centre.
    Returns (t, box, step, indenter work so far); the caller evaluates the forces
    (apip_energy_forces) before the next Verlet step."""
    import torch
    t = {k: torch.tensor(ck[k], device=device) for k in STATE}
    if "csp" in ck:   # rows by atom id, as the library keeps them
        model.set_csp_pairs(torch.tensor(ck["csp"], dtype=torch.int32, device=device).contiguous())
    box = [float(x) for x in ck["box"]]
    if "build_pos" in ck:
        model.build_neighbors(torch.tensor(ck["build_pos"], device=device).contiguous(), box, t["ids"])
    work = 0.0
    if indenter is not None and "ind_centre" in ck:
        model.set_indenter(ck["ind_centre"], indenter["velocity"], indenter["radius"], indenter["k"])
        work = float(ck["ind_work"])
    return t, box, int(ck["step"]), work
