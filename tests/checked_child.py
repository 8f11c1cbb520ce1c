"""Run by test_gpu_checked_build.py in a process of its own, with APIP_LIBRARY
naming the bounds-checked library (libapip_checked.so): a few small cases of
every evaluation path through that library, each of which must finish without
a bounds report (apip_sync would raise APIP_ERR_BOUNDS), two of them also against
the FP64 oracle; then the self-test, whose report must arrive and leave the
context usable.  Prints CHECKED OK at the end."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

from gpu_helpers import run_gpu, run_oracle, to_dev  # noqa: E402
from paper_2512_07693_gb300 import apip  # noqa: E402
from paper_2512_07693_gb300 import workloads as W  # noqa: E402


def system(seed=11, nu=3):
    from oracle import ace
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=seed, temp=600.0)
    nb = len(ace.enumerate_basis(6 if nu == 3 else 4, 3, nu))
    s["prm"] = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9),
                    ace=W.ace_params(6 if nu == 3 else 4, 3, nu, 2, nb))
    return s


def main():
    import torch
    assert os.path.basename(apip.LIB_PATH) == "libapip_checked.so", apip.LIB_PATH
    assert hasattr(apip.lib, "apip_check_bounds_selftest")
    s = system()
    n = len(s["pos"])
    # float64 paper switch against the oracle (the plain bar)
    o = run_oracle(s)
    g = run_gpu(s, precision="fp64")
    assert np.abs(g["F"] - o["F"]).max() <= 1e-9
    # float32: paper switch, deterministic mode, all-ACE (32-atom groups)
    g32 = run_gpu(s, precision="fp32")
    assert np.abs(g32["F"] - o["F"]).max() <= 2e-4
    run_gpu(s, precision="fp32", deterministic=True)
    run_gpu(s, precision="fp32", lam_mode="const1", fields=False)
    # body order 4 (pool evaluation), both precisions
    s4 = system(nu=4)
    run_gpu(s4, precision="fp32", fields=False)
    run_gpu(s4, precision="fp64", fields=False)
    # learned switch, float32 (tensor-core network) against the oracle
    net = W.mlp_params(7)
    net["w4"] = 30.0 * net["w4"]
    prm = dict(s["prm"], mlp=apip.mlp_unflat(apip.mlp_flat(net)), switch=dict(s["prm"]["switch"], d_lo=-1e3, d_hi=1e3))
    ol = run_oracle(s, lam_mode="learned", prm=prm)
    gl = run_gpu(s, precision="fp32", lam_mode="learned", prm=prm)
    assert np.abs(gl["F"] - ol["F"]).max() <= 2e-4
    # MD: 40 steps with neighbour-list rebuilds, float32 paper switch
    m = apip.Apip(s["prm"], n, precision="fp32")
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty_like(t["pos"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], box, t["types"], t["ids"], 0.002, 40)
    m.sync()
    # the self-test's report arrives, names the site, and the context stays usable
    st = apip.lib.apip_check_bounds_selftest(m.ctx, None)
    assert st == apip.APIP_OK, st
    try:
        m.sync()
        raise AssertionError("the self-test's violation was not reported")
    except apip.ApipError as e:
        assert e.status == apip.APIP_ERR_BOUNDS, e.status
        assert "self-test 7 outside [0, 5)" in str(e), str(e)
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    m.sync()
    m.close()
    print("CHECKED OK")


if __name__ == "__main__":
    main()
