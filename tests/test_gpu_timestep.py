"""Time-step dependence of the energy change (the study of Fig. S3): with the
velocity-Verlet integrator the change of H between two consecutive steps scales
as dt^3, for the fast model (lam = 0), the precise model (lam = 1) and the
conservative AP potential alike."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, torch_cuda
from oracle import ace
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system():
    pos, box = W.bcc(6, 6, 6)
    pos = np.delete(pos, np.random.default_rng(21).integers(len(pos)), axis=0)
    pos = W.displace(pos, 0.06, 21)
    s = W._finish(pos, W.maxwell(len(pos), 600.0, 11), box)
    nb = len(ace.enumerate_basis(6, 3, 3))
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    return s


def _mean_step_change(s, dt, t_total, lam_mode):
    torch = torch_cuda()
    steps = int(round(t_total / dt))
    g = run_gpu(s, "fp64", lam_mode=lam_mode, fields=False)
    m, t = g["model"], g["t"]
    F = torch.tensor(g["F"], device="cuda")
    thermo = torch.zeros((steps, 5), dtype=torch.float64, device="cuda")
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], g["box"], t["types"], t["ids"], dt, steps, thermo)
    m.sync()
    th = thermo.cpu().numpy()
    H = (th[:, 0] + th[:, 1]) / len(s["pos"])
    m.close()
    return float(np.mean(np.abs(np.diff(H))))


@pytest.mark.parametrize("lam_mode", ["const0", "paper", "const1"])
def test_energy_change_per_step_scales_as_dt_cubed(lam_mode):
    s = _system()
    dts = np.array([0.00025, 0.0005, 0.001, 0.002])
    dh = np.array([_mean_step_change(s, dt, 0.5, lam_mode) for dt in dts])
    slope = np.polyfit(np.log(dts), np.log(dh), 1)[0]
    assert 2.6 < slope < 3.4, (slope, dh)
