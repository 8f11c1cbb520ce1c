"""The cracked slab at full size: about 2.0 M atoms, a wedge crack through the
thickness, ACE with n_max 8, l_max 4, body order 4 (90 970 basis functions),
the float32 path.

The whole slab is evaluated once, and its forces are taken through the
torch.autograd.Function (dE/dpos = -F).  On 64 seeded atoms they are compared
with central finite differences (h = 1e-5 A) of the float64 energy.  The energy
of the full slab cannot resolve such a difference (float64 at 1e7 eV), so each
difference is taken on the cluster of all atoms within 20 A of the displaced
atom.  Every energy term that moves with that atom is then exact: it depends on
positions within r_w + CSP reach = 9.5 A of its atom (the cluster premise is
pinned on CPU by test_oracle_locality).  The float64 library path itself is
pinned against the oracle at this basis by test_crack_basis_nu4_lmax4.
"""
import numpy as np
import pytest

from gpu_helpers import to_dev, torch_cuda
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu

R_CLUSTER = 20.0


def _cluster(s, i):
    d = s["pos"] - s["pos"][i]
    d -= s["box"] * np.rint(d / s["box"])
    keep = np.flatnonzero(np.sum(d * d, axis=1) < R_CLUSTER ** 2)
    box = np.full(3, 2 * R_CLUSTER + 40.0)
    pos = d[keep] + 0.5 * box
    return pos, box, int(np.flatnonzero(keep == i)[0]), s["lam_fixed"][keep]


def test_crack2m_forces_match_cluster_finite_differences():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    from paper_2512_07693_gb300.autograd import energy
    s = W.config("crack2m", apip.apip_ace_basis_size)
    prm = s["prm"]
    n = len(s["pos"])
    assert n > 1_900_000
    m = apip.Apip(prm, n, precision="fp32", lam_mode="paper", max_nb=80, cell_cap=64)
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.set_lam_fixed(torch.tensor(s["lam_fixed"], dtype=torch.float64, device="cuda"))
    m.init_csp_pairs(t["pos"], box, t["ids"])
    pos = t["pos"].clone().requires_grad_(True)
    E = energy(pos, m, box, t["types"], t["ids"])
    (grad,) = torch.autograd.grad(E, pos)
    F = -grad.cpu().numpy()
    lam = m.field("lam", n).cpu().numpy()
    m.close()
    x = float((lam > 0).mean())
    # the crack faces run through the whole thickness: a few per cent of the slab
    assert 0.001 < x < 0.06, x
    # 64 seeded atoms: half among those evaluated with ACE, half anywhere
    rng = np.random.default_rng(4)
    ace_atoms = np.flatnonzero(lam > 0)
    sample = np.concatenate([rng.choice(ace_atoms, 32, replace=False), rng.choice(n, 32, replace=False)])
    clusters = [_cluster(s, i) for i in sample]
    nc = max(len(c[0]) for c in clusters)
    mc = apip.Apip(prm, nc, precision="fp64", lam_mode="paper", max_nb=96, cell_cap=64)
    h = 1e-5
    worst = 0.0
    for (cpos, cbox, k, cfix), i in zip(clusters, sample):
        nloc = len(cpos)
        mc.set_lam_fixed(torch.tensor(cfix, dtype=torch.float64, device="cuda"))
        ids = torch.arange(nloc, dtype=torch.int32, device="cuda")
        types = torch.zeros(nloc, dtype=torch.int32, device="cuda")
        p0 = torch.tensor(cpos, dtype=torch.float64, device="cuda")
        cb = [float(v) for v in cbox]
        mc.init_csp_pairs(p0, cb, ids)
        fd = np.zeros(3)
        for c in range(3):
            es = []
            for sgn in (1.0, -1.0):
                p = p0.clone()
                p[k, c] += sgn * h
                Fo = torch.empty((nloc, 3), dtype=torch.float64, device="cuda")
                e = torch.zeros(1, dtype=torch.float64, device="cuda")
                mc.energy_forces(p, cb, types, ids, Fo, e_total_out=e)
                mc.sync()
                es.append(float(e.cpu()[0]))
            fd[c] = -(es[0] - es[1]) / (2 * h)
        err = np.abs(F[i] - fd).max()
        worst = max(worst, err)
        # float32 forces (2e-4 eV/A) plus the difference quotient's own error
        assert err < 3e-4, (int(i), float(lam[i]), F[i], fd)
    mc.close()
