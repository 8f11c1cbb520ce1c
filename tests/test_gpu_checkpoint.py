"""Checkpoint and resume: a run stopped after 10 steps and resumed in a new
context (saved CSP^list partners restored, not detected again) continues the
uninterrupted trajectory (float64 path, 600 K crystal with a vacancy, the
paper's switch with a transition region)."""
import numpy as np
import pytest

from gpu_helpers import to_dev, torch_cuda
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system():
    from oracle import ace
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=11, temp=600.0)
    nb = len(ace.enumerate_basis(6, 3, 3))
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    return s


def _steps(torch, m, t, box, k):
    F = torch.empty_like(t["pos"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], box, t["types"], t["ids"], 0.001, k)
    m.sync()


def test_resume_continues_the_trajectory(tmp_path):
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip, checkpoint
    s = _system()
    n = len(s["pos"])
    box = [float(x) for x in s["box"]]
    a = apip.Apip(s["prm"], n, precision="fp64")
    ta = to_dev(torch, s)
    a.init_csp_pairs(ta["pos"], box, ta["ids"])
    _steps(torch, a, ta, box, 10)
    assert int((a.field("dlam", n) != 0).sum()) > 10
    path = str(tmp_path / "run.npz")
    checkpoint.save(path, a, ta, box, 10)
    _steps(torch, a, ta, box, 10)
    partners = a.field("csp", n).cpu().numpy()
    a.close()

    b = apip.Apip(s["prm"], n, precision="fp64")
    tb, box_b, step, _ = checkpoint.resume(b, checkpoint.load(path))
    assert step == 10 and box_b == box
    _steps(torch, b, tb, box_b, 10)
    np.testing.assert_array_equal(b.field("csp", n).cpu().numpy(), partners)
    assert np.abs(tb["pos"].cpu().numpy() - ta["pos"].cpu().numpy()).max() < 1e-9
    assert np.abs(tb["vel"].cpu().numpy() - ta["vel"].cpu().numpy()).max() < 1e-7
    b.close()
    # without the saved partners the paper's switch refuses to run
    c = apip.Apip(s["prm"], n, precision="fp64")
    tc, _, _, _ = checkpoint.resume(c, {k: v for k, v in checkpoint.load(path).items() if k != "csp"})
    with pytest.raises(apip.ApipError) as e:
        c.energy_forces(tc["pos"], box, tc["types"], tc["ids"], torch.empty_like(tc["pos"]))
    assert e.value.status == apip.APIP_ERR_STATE
    c.close()
