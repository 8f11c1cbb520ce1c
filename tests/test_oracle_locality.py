"""The premise of the full-size sampled parity test: an atom's energy, lam and
force depend only on the atoms within 20 A of it, so the oracle on a cluster cut
out of a periodic crystal reproduces them.  Checked against the oracle on the
whole periodic crystal (6685 atoms with a void), for atoms of every regime."""
import numpy as np

from gpu_helpers import run_oracle
from oracle import ace
from paper_2512_07693_gb300 import workloads as W
from test_gpu_full_size import _cluster


def test_cluster_of_20_angstrom_reproduces_the_periodic_crystal():
    nb = len(ace.enumerate_basis(6, 3, 3))
    s = W.void_crystal(cells=15, void_radius=6.0, sigma=0.03, temp=300.0, seed=3)
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), switch=dict(W.SWITCH), csp=dict(W.CSP),
                    ace=W.ace_params(6, 3, 3, 2, nb))
    o = run_oracle(s)
    lam = o["lam"]
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.flatnonzero(lam == 1), 2),
                          rng.choice(np.flatnonzero((lam > 0) & (lam < 1)), 2),
                          rng.choice(np.flatnonzero(lam == 0), 2)])
    for i in idx:
        c, k = _cluster(s, i)
        oc = run_oracle(c)
        assert abs(oc["lam"][k] - lam[i]) < 1e-13
        assert abs(oc["e_atom"][k] - o["e_atom"][i]) < 1e-12
        assert np.abs(oc["F"][k] - o["F"][i]).max() < 1e-12
