"""apip_reduce_energy_static, the allocation-free total-energy entry point for
callers that cannot call cudaMalloc (a host program whose device memory is owned
by its own pool allocator, or a loop that must never enter the allocator).

Its float64 total of the per-atom energies must equal the total that
apip_energy_forces reduces with context scratch, within the float64 energy
tolerance of the parity tests, on consecutive calls that reuse the same fixed
scratch array.  This file is named to be collected last, so that a failure here
comes after every other test has run.
"""
import numpy as np
import pytest

from gpu_helpers import to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TOL_E = 1e-9   # float64 energy tolerance of the parity tests (per atom), applied to the total


def _energies(torch, cells):
    from paper_2512_07693_gb300 import apip, workloads as W
    s = W.vacancy_crystal(cells=cells, sigma=0.06, seed=21)
    nb = apip.apip_ace_basis_size(6, 3, 3)
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
               switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    n = len(s["pos"])
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m = apip.Apip(prm, n, precision="fp64")
    m.init_csp_pairs(t["pos"], box, t["ids"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    e_atom = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, e_atom, E)
    m.sync()
    m.close()
    return e_atom, float(E.cpu()[0])


def test_static_reduction_matches_energy_forces_on_consecutive_calls():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    big, E_big = _energies(torch, 14)       # 5487 atoms: two blocks of partials
    small, E_small = _energies(torch, 6)    # 431 atoms: one block
    assert len(big) > 4096 > len(small)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    apip.apip_reduce_energy_static(big, len(big), out[0:1])
    apip.apip_reduce_energy_static(big, len(big), out[1:2])
    apip.apip_reduce_energy_static(small, len(small), out[2:3])
    apip.apip_reduce_energy_static(small, len(small), out[3:4])
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    np.testing.assert_allclose(got[:2], E_big, rtol=0, atol=TOL_E * len(big))
    np.testing.assert_allclose(got[2:], E_small, rtol=0, atol=TOL_E * len(small))


def test_static_reduction_rejects_oversize_and_bad_arguments():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    e = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(apip.ApipError) as err:
        apip.apip_reduce_energy_static(e, apip.APIP_STATIC_MAX_ATOMS + 1, out)
    assert err.value.status == apip.APIP_ERR_SIZE
    with pytest.raises(apip.ApipError) as err:
        apip.apip_reduce_energy_static(e, -1, out)
    assert err.value.status == apip.APIP_ERR_ARG
    apip.apip_reduce_energy_static(e, 0, out)           # empty input: total 0
    torch.cuda.synchronize()
    assert float(out.cpu()[0]) == 0.0
