"""Deterministic mode (apip_params.deterministic = 1, float32 path, body order
<= 3): cells sorted by index after binning, the compacted list written in index
order and every scattered force and c-vector contribution summed as 64-bit fixed
point (2^-40).  Checked here:
- it is still the method: forces, energies and lam against the FP64 oracle at the
  plain float32 parity bars (2e-4 eV/A, 1e-5 eV), and against the default (float64
  atomic) mode, paper and learned switch;
- two contexts running the same 30 MD steps give the same bits (positions,
  velocities, forces, per-atom energies), paper and learned switch;
- a run stopped after 10 steps, checkpointed (with the neighbour list's build
  positions) and resumed in a new context continues the uninterrupted trajectory
  bit for bit."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, run_oracle, to_dev, torch_cuda
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(seed=11):
    from oracle import ace
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=seed, temp=600.0)
    nb = len(ace.enumerate_basis(6, 3, 3))
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    return s


@pytest.mark.parametrize("prec,tolF,tolE", [("fp32", 2e-4, 1e-5)])
def test_deterministic_mode_matches_oracle(prec, tolF, tolE):
    s = _system()
    o = run_oracle(s)
    g = run_gpu(s, precision=prec, deterministic=True)
    assert np.count_nonzero(o["dlam"]) > 10
    assert np.abs(g["F"] - o["F"]).max() <= tolF
    assert np.abs(g["e_atom"] - o["e_atom"]).max() <= tolE
    assert abs(g["E"] - o["E"]) <= tolE * len(s["pos"])
    # the compacted list in index order
    lst = g["ace_list"][:g["count"]]
    assert np.all(np.diff(lst) > 0)
    np.testing.assert_array_equal(lst, np.flatnonzero(g["lam"] > 0))
    # the default mode differs by summation order (neighbour order within a cell,
    # the ACE groups' composition, the atomics) and the 2^-40 rounding: at the
    # rounding level of the path's precision
    d = run_gpu(s, precision=prec)
    bound = (1e-10, 1e-12) if prec == "fp64" else (1e-4, 5e-6)
    assert np.abs(g["F"] - d["F"]).max() < bound[0]
    assert np.abs(g["e_atom"] - d["e_atom"]).max() < bound[1]


def _learned_prm(s):
    """An untrained network with its output layer scaled by 30 (so that g varies
    like a trained indicator's) and a switch window from the 20 % quantile of d."""
    from oracle import mlp
    from oracle.neighbors import pairs
    from oracle.switch import descriptor
    from paper_2512_07693_gb300 import apip
    net = W.mlp_params(7)
    net["w4"] = 30.0 * net["w4"]
    prm = dict(s["prm"], mlp=apip.mlp_unflat(apip.mlp_flat(net)))
    n = len(s["pos"])
    i, j, rv, r = pairs(s["pos"], s["box"], 5.5)
    g, _, _ = mlp.learned_g(n, i, r, prm["mlp"], 5.0, 1.0)
    _, d, _, _ = descriptor(n, i, j, r, g, dict(prm["switch"], d_lo=-1e9, d_hi=1e9))
    lo = float(np.quantile(d, 0.2))
    prm["switch"] = dict(prm["switch"], d_lo=lo, d_hi=lo + 0.5 * float(g.max() - g.min()))
    return prm


def test_deterministic_learned_switch_matches_default_mode():
    s = _system()
    prm = _learned_prm(s)
    g = run_gpu(s, precision="fp32", lam_mode="learned", prm=prm, deterministic=True)
    d = run_gpu(s, precision="fp32", lam_mode="learned", prm=prm)
    assert np.count_nonzero(d["dlam"]) > 10
    assert np.abs(g["F"] - d["F"]).max() < 1e-4
    np.testing.assert_allclose(g["lam"], d["lam"], atol=1e-5)


def _run(torch, s, prec, lam_mode="paper", prm=None, steps=30):
    from paper_2512_07693_gb300 import apip
    prm = prm or s["prm"]
    n = len(s["pos"])
    box = [float(x) for x in s["box"]]
    m = apip.Apip(prm, n, precision=prec, lam_mode=lam_mode, deterministic=True)
    t = to_dev(torch, s)
    if lam_mode == "paper":
        m.init_csp_pairs(t["pos"], box, t["ids"])
    else:
        m.set_mlp(torch.tensor(apip.mlp_flat(prm["mlp"]), device="cuda"))
    F = torch.empty_like(t["pos"])
    e = torch.empty(n, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], box, t["types"], t["ids"], 0.001, steps)
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, e)
    m.sync()
    out = [x.cpu().numpy() for x in (t["pos"], t["vel"], F, e)]
    m.close()
    return out


@pytest.mark.parametrize("prec,lam_mode", [("fp32", "paper"), ("fp32", "learned")])
def test_repeated_runs_give_the_same_bits(prec, lam_mode):
    torch = torch_cuda()
    s = _system(seed=12)
    prm = _learned_prm(s) if lam_mode == "learned" else None
    a = _run(torch, s, prec, lam_mode, prm)
    b = _run(torch, s, prec, lam_mode, prm)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def _steps(torch, m, t, box, k):
    F = torch.empty_like(t["pos"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], box, t["types"], t["ids"], 0.001, k)
    m.sync()


@pytest.mark.parametrize("prec", ["fp32"])
def test_resume_is_bit_for_bit(tmp_path, prec):
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip, checkpoint
    s = _system()
    n = len(s["pos"])
    box = [float(x) for x in s["box"]]
    a = apip.Apip(s["prm"], n, precision=prec, deterministic=True)
    ta = to_dev(torch, s)
    a.init_csp_pairs(ta["pos"], box, ta["ids"])
    _steps(torch, a, ta, box, 10)
    path = str(tmp_path / "run.npz")
    checkpoint.save(path, a, ta, box, 10)
    _steps(torch, a, ta, box, 25)
    a.close()

    b = apip.Apip(s["prm"], n, precision=prec, deterministic=True)
    tb, box_b, step, _ = checkpoint.resume(b, checkpoint.load(path))
    _steps(torch, b, tb, box_b, 25)
    b.close()
    np.testing.assert_array_equal(tb["pos"].cpu().numpy(), ta["pos"].cpu().numpy())
    np.testing.assert_array_equal(tb["vel"].cpu().numpy(), ta["vel"].cpu().numpy())
