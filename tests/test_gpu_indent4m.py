"""The indentation slab at full size: 3 993 600 atoms under a spherical indenter,
the float32 path with the bottom surface and the top surface outside the
contact zone pinned to the fast model (a constant-switch subset, Appendix B).

The slab is evaluated once with the sphere pressed 1 A into the top surface, with
the paper's switch and with the learned one, and sampled atoms are checked one by
one against the oracle.  As in the full-size void test, the AP energy and force of
an atom depend on positions within 9.5 A of it, so the oracle runs on the cluster
of all atoms within 20 A (pinned atoms keep their constant lam there); the
indenter's energy and force act on each atom alone and come from its closed form.
"""
import numpy as np
import pytest

from gpu_helpers import run_oracle, torch_cuda
from oracle import ace, indenter, mlp
from oracle.neighbors import pairs
from oracle.switch import descriptor
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu

R_CLUSTER = 20.0
DEPTH = 1.0


def _cluster(s, i, prm):
    d = s["pos"] - s["pos"][i]
    d -= s["box"] * np.rint(d / s["box"])
    keep = np.flatnonzero(np.sum(d * d, axis=1) < R_CLUSTER ** 2)
    box = np.full(3, 2 * R_CLUSTER + 40.0)
    c = W._finish(d[keep] + 0.5 * box, np.zeros((len(keep), 3)), box)
    c["ids"] = s["ids"][keep].copy()
    c["prm"] = prm
    return c, int(np.flatnonzero(keep == i)[0]), s["lam_fixed"][keep]


def _learned_prm(s, centre):
    """An untrained network with its output layer scaled by 30 (g then varies like a
    trained indicator's) and a switch window from the oracle's descriptor d near the
    contact point: on the cluster of the atoms within 20 A of the surface atom
    nearest the indenter axis, d is exact for the atoms within 10 A of that atom
    (it depends on positions within r_w + r_c = 10 A); d_lo is the 30 % quantile of
    those values, the width half their range."""
    from paper_2512_07693_gb300 import apip
    net = W.mlp_params(7)
    net["w4"] = 30.0 * net["w4"]
    net = apip.mlp_unflat(apip.mlp_flat(net))       # the float32 weights the library holds
    prm = dict(s["prm"], mlp=net)
    top = np.argmin(np.sum((s["pos"] - centre) ** 2, axis=1))
    c, k, _ = _cluster(s, top, prm)
    n = len(c["pos"])
    i, j, _, r = pairs(c["pos"], c["box"], 5.5)
    g, _, _ = mlp.learned_g(n, i, r, net, 5.0, 1.0)
    _, d, _, _ = descriptor(n, i, j, r, g, dict(prm["switch"], d_lo=-1e9, d_hi=1e9))
    inner = np.sum((c["pos"] - c["pos"][k]) ** 2, axis=1) < 100.0
    lo = float(np.quantile(d[inner], 0.3))
    return dict(prm, switch=dict(prm["switch"], d_lo=lo, d_hi=lo + 0.5 * float(np.ptp(d[inner]))))


@pytest.mark.parametrize("lam_mode", ["paper", "learned"])
def test_indent4m_full_size_sampled_atoms_fp32(lam_mode):
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.config("indent4m", apip.apip_ace_basis_size)
    n = len(s["pos"])
    assert n == 3_993_600
    ind = s["indenter"]
    centre = ind["center"] - np.array([0.0, 0.0, DEPTH])
    prm = s["prm"] if lam_mode == "paper" else _learned_prm(s, centre)
    m = apip.Apip(prm, n, precision="fp32", lam_mode=lam_mode, max_nb=80, cell_cap=48)
    dev = torch.device("cuda")
    pos = torch.tensor(s["pos"], dtype=torch.float64, device=dev)
    ids = torch.tensor(s["ids"], dtype=torch.int32, device=dev)
    types = torch.zeros(n, dtype=torch.int32, device=dev)
    box = [float(x) for x in s["box"]]
    m.set_lam_fixed(torch.tensor(s["lam_fixed"], dtype=torch.float64, device=dev))
    m.set_indenter(centre, [0.0, 0.0, 0.0], ind["radius"], ind["k"])
    if lam_mode == "paper":
        m.init_csp_pairs(pos, box, ids)
    else:
        m.set_mlp(torch.tensor(apip.mlp_flat(prm["mlp"]), device=dev))
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    m.energy_forces(pos, box, types, ids, F, e, E)
    m.sync()
    F = F.cpu().numpy()
    e = e.cpu().numpy()
    # the total is the sum of the per-atom energies (float32 warp sums round at 1e-7)
    assert abs(float(E.cpu()[0]) - e.sum()) < 1e-6 * n
    lam = m.field("lam", n).cpu().numpy()
    dlam = m.field("dlam", n).cpu().numpy()
    m.close()
    e_ind, f_ind = indenter.energy_forces(s["pos"], s["box"], centre, ind["radius"], ind["k"])
    pinned = np.isfinite(s["lam_fixed"])
    assert np.all(lam[pinned] == 0.0)
    touched = np.flatnonzero(e_ind > 0)
    assert len(touched) > 20
    rng = np.random.default_rng(17)
    core = np.flatnonzero(lam == 1.0)
    trans = np.flatnonzero((lam > 0) & (lam < 1) & (dlam != 0))
    assert len(core) and len(trans)
    sample = np.concatenate([rng.choice(touched, 2, replace=False), rng.choice(core, 2, replace=False),
                             rng.choice(trans, 2, replace=False), rng.choice(np.flatnonzero(pinned), 1),
                             rng.choice(np.flatnonzero(~pinned & (lam == 0.0)), 1)])
    model = ace.AceModel(prm["ace"])
    for i in sample:
        c, k, fixed = _cluster(s, i, prm)
        o = run_oracle(c, lam_mode=lam_mode, model=model, lam_const=fixed)
        assert abs(lam[i] - o["lam"][k]) < 1e-5, (i, lam[i], o["lam"][k])
        assert abs(e[i] - (o["e_atom"][k] + e_ind[i])) <= 1e-5, (i, e[i], o["e_atom"][k] + e_ind[i])
        err = np.abs(F[i] - (o["F"][k] + f_ind[i])).max()
        assert err <= 2e-4, (i, lam[i], err)
