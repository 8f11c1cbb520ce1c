"""Parity at full size: the 248 757-atom void crystal (float32 path, the launch
configuration that bench.py times) evaluated once on the GPU, and sampled atoms
checked one by one against the oracle.

The oracle cannot run the whole crystal, but every per-atom output is local.
E_j depends on the atoms within r_w = 5 A of j (ACE, EAM, the weights of d_j)
and on the CSP partners of those atoms (detected within 4.5 A), so it depends
on positions within 9.5 A of j; F_i = -dE/dx_i involves the E_j with j within
9.5 A of i.  A cluster of all atoms within 20 A of the sampled atom, placed in
an empty box, therefore reproduces E_i, lam_i and F_i exactly (up to rounding).
"""
import numpy as np
import pytest

from gpu_helpers import run_oracle, to_dev, torch_cuda
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu

R_CLUSTER = 20.0


def _cluster(s, i):
    d = s["pos"] - s["pos"][i]
    d -= s["box"] * np.rint(d / s["box"])
    keep = np.flatnonzero(np.sum(d * d, axis=1) < R_CLUSTER ** 2)
    box = np.full(3, 2 * R_CLUSTER + 40.0)
    pos = d[keep] + 0.5 * box
    c = W._finish(pos, np.zeros_like(pos), box)
    c["ids"] = s["ids"][keep].copy()
    c["prm"] = s["prm"]
    return c, int(np.flatnonzero(keep == i)[0])


@pytest.fixture(scope="module")
def void250k_fp32():
    """The whole crystal evaluated once on the GPU (float32 path, bench launch
    configuration): the workload, forces, per-atom energies, lam and dlam."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.config("void250k", apip.apip_ace_basis_size)
    n = len(s["pos"])
    assert n == 248757
    m = apip.Apip(s["prm"], n, precision="fp32", lam_mode="paper", max_nb=80, cell_cap=48)
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, e)
    m.sync()
    out = dict(s=s, F=F.cpu().numpy(), e=e.cpu().numpy(), lam=m.field("lam", n).cpu().numpy(),
               dlam=m.field("dlam", n).cpu().numpy())
    m.close()
    return out


def test_void250k_full_size_sampled_atoms_fp32(void250k_fp32):
    s, F, e, lam, dlam = (void250k_fp32[k] for k in ("s", "F", "e", "lam", "dlam"))
    assert np.abs(F.sum(axis=0)).max() < 1e-2     # 249 k atoms, float32 pair terms
    rng = np.random.default_rng(11)
    core = np.flatnonzero(lam == 1.0)
    trans = np.flatnonzero((lam > 0) & (lam < 1) & (dlam != 0))
    # fast atoms within r_w of the transition region carry grad-lambda forces
    near = np.flatnonzero(lam == 0.0)
    dc = s["pos"][near][:, None, :] - s["pos"][trans[:200]][None, :, :]
    dc -= s["box"] * np.rint(dc / s["box"])
    near = near[np.min(np.sum(dc * dc, axis=2), axis=1) < 25.0]
    bulk = np.flatnonzero(lam == 0.0)
    assert len(core) and len(trans) and len(near)
    sample = np.concatenate([rng.choice(core, 2, replace=False), rng.choice(trans, 3, replace=False),
                             rng.choice(near, 2, replace=False), rng.choice(bulk, 1)])
    for i in sample:
        c, k = _cluster(s, i)
        o = run_oracle(c)
        assert abs(lam[i] - o["lam"][k]) < 1e-5, (i, lam[i], o["lam"][k])
        assert abs(e[i] - o["e_atom"][k]) <= 1e-5, (i, e[i], o["e_atom"][k])
        err = np.abs(F[i] - o["F"][k]).max()
        assert err <= 2e-4, (i, lam[i], err)


SUBBOX_HALF = 16.0     # half edge of the sub-box (A): ~2 100 atoms
SUBBOX_HALO = 20.0     # every dependency of its atoms' outputs (module docstring)
SUBBOX_FREE = 10.0     # atoms farther than this from the sub-box do not affect them


def test_void250k_subbox_every_atom_fp32(void250k_fp32):
    """Every atom of a ~2 100-atom cube straddling the void surface (centred on the
    surface, so it holds precise, transition and fast atoms) against one oracle run
    on the cube and a 20 A halo.  The halo's outer atoms (farther than 10 A from
    the cube) neither enter the cube's energies nor, beyond 9.5 A, its forces;
    the oracle holds them at lam = 0 (a constant-switch subset) so that it does
    not evaluate ACE on the free surface of the cut-out."""
    s, F, e, lam = (void250k_fp32[k] for k in ("s", "F", "e", "lam"))
    centre = 0.5 * s["box"] + np.array([15.0, 0.0, 0.0])
    d = s["pos"] - centre
    d -= s["box"] * np.rint(d / s["box"])
    out = np.maximum(np.abs(d) - SUBBOX_HALF, 0.0)
    dist = np.sqrt(np.sum(out * out, axis=1))     # distance to the cube, 0 inside
    inside = np.flatnonzero(dist == 0.0)
    keep = np.flatnonzero(dist < SUBBOX_HALO)
    assert 1900 < len(inside) < 2400
    assert np.any(lam[inside] == 1.0) and np.any((lam[inside] > 0) & (lam[inside] < 1)) and np.any(lam[inside] == 0)
    box = np.full(3, 2 * (SUBBOX_HALF + SUBBOX_HALO) + 40.0)
    pos = d[keep] + 0.5 * box
    c = W._finish(pos, np.zeros_like(pos), box)
    c["ids"] = s["ids"][keep].copy()
    c["prm"] = s["prm"]
    lam_const = np.where(dist[keep] > SUBBOX_FREE, 0.0, np.nan)
    o = run_oracle(c, lam_const=lam_const)
    loc = np.searchsorted(keep, inside)
    assert np.array_equal(keep[loc], inside)
    np.testing.assert_allclose(lam[inside], o["lam"][loc], atol=1e-5, rtol=0)
    np.testing.assert_allclose(e[inside], o["e_atom"][loc], atol=1e-5, rtol=0)
    err = np.abs(F[inside] - o["F"][loc]).max()
    assert err <= 2e-4, err


def test_void250k_fp32_against_fp64_all_atoms():
    """Every atom of the full crystal: the float32 path (the benchmarked one)
    against the float64 path, which the parity tests pin to the oracle at 1e-9 eV/A,
    within the float32 tolerances (2e-4 eV/A, 1e-5 eV per atom)."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.config("void250k", apip.apip_ace_basis_size)
    n = len(s["pos"])
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    out = {}
    for prec in ("fp32", "fp64"):
        m = apip.Apip(s["prm"], n, precision=prec, lam_mode="paper", max_nb=80, cell_cap=48)
        m.init_csp_pairs(t["pos"], box, t["ids"])
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        m.energy_forces(t["pos"], box, t["types"], t["ids"], F, e)
        m.sync()
        out[prec] = (F.cpu().numpy(), e.cpu().numpy(), m.field("lam", n).cpu().numpy())
        m.close()
    F32, e32, l32 = out["fp32"]
    F64, e64, l64 = out["fp64"]
    assert int((l64 > 0).sum()) > 1000
    assert np.abs(F32 - F64).max() <= 2e-4
    assert np.abs(e32 - e64).max() <= 1e-5
    assert np.abs(l32 - l64).max() <= 1e-5
    assert np.abs(F64.sum(axis=0)).max() < 1e-9                  # Newton's third law in float64
