"""The spherical indenter of the indentation workload on the GPU: forces and
energies against the oracle (AP potential plus the indenter's closed form), and
NVE with a moving indenter, where H - W (W the work accumulated by the library)
is conserved while H itself changes by W."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, run_oracle, to_dev, torch_cuda
from oracle import ace, indenter
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu

K = 10.0
R = 4.5


def mixed(seed=21):
    pos, box = W.bcc(6, 6, 6)
    site = int(np.random.default_rng(seed).integers(len(pos)))
    hole = pos[site].copy()
    pos = np.delete(pos, site, axis=0)
    pos = W.displace(pos, 0.06, seed)
    s = W._finish(pos, np.zeros_like(pos), box, vacancy=hole)
    nb = len(ace.enumerate_basis(6, 3, 3))
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    return s


@pytest.mark.parametrize("prec,tolF,tolE", [("fp64", 1e-9, 1e-9), ("fp32", 2e-4, 1e-5)])
def test_indenter_forces_and_energies(prec, tolF, tolE):
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = mixed()
    c = 0.5 * s["box"] + np.array([0.3, -0.2, 0.1])
    o = run_oracle(s)
    e_ind, f_ind = indenter.energy_forces(s["pos"], s["box"], c, R, K)
    assert np.count_nonzero(e_ind) > 10
    n = len(s["pos"])
    m = apip.Apip(s["prm"], n, precision=prec)
    m.set_indenter(c, [0.0, 0.0, 0.0], R, K)
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ea = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, ea, E)
    m.sync()
    assert np.abs(F.cpu().numpy() - (o["F"] + f_ind)).max() <= tolF
    np.testing.assert_allclose(ea.cpu().numpy(), o["e_atom"] + e_ind, atol=tolE)
    assert abs(float(E.cpu()[0]) - (o["E"] + e_ind.sum())) <= tolE * n
    # removing it restores the plain potential
    m.set_indenter(c, [0.0, 0.0, 0.0], 0.0, K)
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, ea, E)
    m.sync()
    assert np.abs(F.cpu().numpy() - o["F"]).max() <= tolF


def test_moving_indenter_conserves_h_minus_w():
    """A small sphere starts in the vacancy (no atom inside) and moves at 4 A/ps
    into the neighbour shells for 0.5 ps."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = mixed(seed=5)
    s["vel"] = W.maxwell(len(s["pos"]), 300.0, 9)
    n = len(s["pos"])
    m = apip.Apip(s["prm"], n, precision="fp64")
    c0 = s["vacancy"]
    v = np.array([0.0, 0.0, 4.0])
    m.set_indenter(c0, v, 2.0, K)
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.sync()
    steps, dt = 1000, 0.0005
    thermo = torch.zeros((steps, 5), dtype=torch.float64, device="cuda")
    works = []   # the work after each step, read between one-step calls
    for k in range(steps):
        m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], box, t["types"], t["ids"], dt, 1, thermo[k:k + 1])
        works.append(m.indenter_state()[1])
    th = thermo.cpu().numpy()
    H = th[:, 0] + th[:, 1]
    Wk = np.array(works)
    centre, _ = m.indenter_state()
    np.testing.assert_allclose(centre, c0 + v * dt * steps, atol=1e-9)
    dw = abs(Wk[-1] - Wk[0])
    assert dw > 0.02, dw                                      # the indenter did work
    drift = np.abs((H - Wk) - (H[0] - Wk[0])).max()
    assert drift < 0.02 * dw, (drift, dw)                     # H - W is conserved, H is not
    assert np.abs(H - H[0]).max() > 0.5 * dw
