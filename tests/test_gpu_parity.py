"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.  Bars: float64 path |dF| <= 1e-9 eV/A and per-atom energy
<= 1e-9 eV; float32 path |dF| <= 2e-4 eV/A and |dE|/atom <= 1e-5 eV; neighbour
sets, CSP pairs and the compacted ACE set exact."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, run_oracle, to_dev, torch_cuda
from oracle import ace
from oracle.neighbors import pairs
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-9, e=1e-9), "fp32": dict(F=2e-4, e=1e-5)}


def nbasis(a, b, c):
    return len(ace.enumerate_basis(a, b, c))


def small(cells=(6, 6, 6), sigma=0.06, seed=21, adds_eam=True, acecfg=(6, 3, 3), d_lo=0.25, d_hi=0.9, vac=True):
    pos, box = W.bcc(*cells)
    if vac:
        pos = np.delete(pos, np.random.default_rng(seed).integers(len(pos)), axis=0)
    pos = W.displace(pos, sigma, seed)
    s = W._finish(pos, np.zeros_like(pos), box)
    s["prm"] = dict(precise_adds_eam=adds_eam, eam=dict(W.EAM), csp=dict(W.CSP),
                    switch=dict(W.SWITCH, d_lo=d_lo, d_hi=d_hi),
                    ace=W.ace_params(*acecfg, 2, nbasis(*acecfg)))
    return s


def compare(g, o, prec, check_sets=True):
    tol = TOL[prec]
    lam = o["lam"]
    if prec == "fp64":
        np.testing.assert_allclose(g["lam"], lam, atol=1e-12)
        np.testing.assert_allclose(g["dlam"], o["dlam"], atol=1e-10)
        np.testing.assert_allclose(g["g"], o["g"], atol=1e-12)
        np.testing.assert_allclose(g["d"], o["d"], atol=1e-12)
        np.testing.assert_allclose(g["wbar"], o["wbar"], atol=1e-12)
    P = o["P"]
    Pg = np.sort(g["ace_list"][: g["count"]])
    if check_sets:
        if prec == "fp64":
            assert np.array_equal(Pg, np.sort(P))
        else:
            # float32 may only disagree where d is within its rounding of d_lo
            # (there lam ~ (d - d_lo)^3 is negligible)
            diff = np.setxor1d(Pg, P)
            assert np.all((np.abs(o["d"][diff] - o["switch_dlo"]) < 1e-5) | (lam[diff] < 1e-12)), diff
    np.testing.assert_allclose(g["e_eam"], o["e_eam"], atol=tol["e"])
    both = np.intersect1d(Pg, P)
    np.testing.assert_allclose(g["e_ace"][both], o["e_ace"][both], atol=tol["e"])
    np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=tol["e"])
    assert abs(g["E"] - o["E"]) <= tol["e"] * len(lam)
    err = np.abs(g["F"] - o["F"]).max()
    assert err <= tol["F"], f"max |dF| = {err:.3e}"


def _check(s, prec="fp64", **kw):
    o = run_oracle(s, lam_mode=kw.get("lam_mode", "paper"), grad_lambda=kw.get("grad_lambda", True))
    o["switch_dlo"] = s["prm"]["switch"]["d_lo"]
    g = run_gpu(s, precision=prec, **kw)
    compare(g, o, prec)
    return g, o


@pytest.mark.parametrize("prec,group", [("fp64", 0), ("fp64", 32), ("fp64", 4), ("fp32", 0), ("fp32", 4),
                                        ("fp32", 8), ("fp32", 32)])
def test_mixed_system_parity(prec, group):
    """Body order 3 (the streamed kernel); group = compacted atoms per ACE thread
    block (0: automatic)."""
    s = small()
    g, o = _check(s, prec, ace_group=group)
    # every regime is exercised
    assert np.any(o["lam"] == 1.0) and np.any(o["lam"] == 0.0) and np.count_nonzero(o["dlam"]) > 10


@pytest.mark.parametrize("prec,group", [("fp64", 0), ("fp32", 0), ("fp64", 1), ("fp32", 2), ("fp64", 4),
                                        ("fp32", 8)])
def test_nu4_ragged(prec, group):
    """4-body terms (the pool kernel) with every group size, N not a multiple of 32
    (precise = EAM + ACE as in the workloads)."""
    s = small(cells=(7, 6, 6), adds_eam=True, acecfg=(4, 3, 4), seed=5)
    assert len(s["pos"]) % 32 != 0
    _check(s, prec, ace_group=group)


_ORACLE_844 = {}


def _crack_basis_system():
    """The crack workload's basis (n_max 8, l_max 4, nu <= 4: 90970 functions,
    a pool of 13188 values per atom) on a small vacancy crystal; the oracle result
    is shared by the float64 and float32 cases."""
    s = small(cells=(6, 6, 6), acecfg=(8, 4, 4), seed=9, d_lo=0.3, d_hi=0.9)
    if "o" not in _ORACLE_844:
        o = run_oracle(s)
        o["switch_dlo"] = s["prm"]["switch"]["d_lo"]
        _ORACLE_844["o"] = o
    return s, _ORACLE_844["o"]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_crack_basis_nu4_lmax4(prec):
    s, o = _crack_basis_system()
    assert len(o["P"]) > 10
    g = run_gpu(s, precision=prec)
    compare(g, o, prec)


def test_pure_ace_precise_model_nu4_fp64():
    """precise = ACE alone (EAM weights 1 - lam, the paper's literal structure)."""
    s = small(cells=(7, 6, 6), adds_eam=False, acecfg=(4, 3, 4), seed=5)
    _check(s, "fp64")


def test_pure_ace_precise_model_nu4_fp32():
    """precise = ACE alone, float32, at the plain bars (2e-4 eV/A, 1e-5 eV per atom).
    |E^prec - E^EAM| reaches 6 eV on this random ACE, so the switch must carry lam
    to ~1e-6: the float32 sums of w-bar and sum g w are compensated and the CSP
    vectors are formed from the integer separations."""
    s = small(cells=(7, 6, 6), adds_eam=False, acecfg=(4, 3, 4), seed=5)
    o = run_oracle(s)
    assert np.abs(o["e_ace"] - o["e_eam"]).max() > 3.0
    o["switch_dlo"] = s["prm"]["switch"]["d_lo"]
    g = run_gpu(s, precision="fp32")
    compare(g, o, "fp32")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shifted_energy_zero_parity(prec):
    """The precise model's energy lowered by a constant per atom (prec_shift)."""
    s = small()
    s["prm"]["prec_shift"] = 0.7
    _check(s, prec)


@pytest.mark.parametrize("mode", ["const0", "const1"])
def test_constant_switch_modes(mode):
    s = small(cells=(6, 6, 6), adds_eam=False)
    _check(s, "fp64", lam_mode=mode)


def test_without_grad_lambda_ablation():
    s = small()
    _check(s, "fp64", grad_lambda=False)


def test_neighbour_list_and_csp_pairs_exact():
    s = small(cells=(6, 7, 6), sigma=0.1)
    g = run_gpu(s, "fp64")
    o = run_oracle(s)
    rl = 5.5
    i, j, rv, r = pairs(s["pos"], s["box"], rl)
    n = len(s["pos"])
    sets = [set() for _ in range(n)]
    for a, b in zip(i.tolist(), j.tolist()):
        sets[a].add(b)
    for a in range(n):
        got = set(g["nblist"][a][: g["nnb"][a]].tolist())
        assert got == sets[a], a
    assert np.array_equal(g["csp"], o["partners"])


def test_neighbour_list_fp32_brackets_the_cutoff():
    """The float32 list (fixed-point pair vectors, float distances) holds every
    pair within r_list - 1e-4 A and none beyond r_list + 1e-4 A."""
    s = small(cells=(6, 7, 6), sigma=0.1)
    g = run_gpu(s, "fp32")
    n = len(s["pos"])
    rl = 5.5
    inner = [set() for _ in range(n)]
    outer = [set() for _ in range(n)]
    for cut, sets in ((rl - 1e-4, inner), (rl + 1e-4, outer)):
        i, j, _, _ = pairs(s["pos"], s["box"], cut)
        for a, b in zip(i.tolist(), j.tolist()):
            sets[a].add(b)
    for a in range(n):
        got = set(g["nblist"][a][: g["nnb"][a]].tolist())
        assert inner[a] <= got <= outer[a], a


def test_vacancy2k_config_fp64():
    s = W.config("vacancy2k", nbasis)
    g, o = _check(s, "fp64")
    x = len(o["P"]) / len(s["pos"])
    assert 0.02 < x < 0.12


def test_vacancy2k_config_fp32():
    s = W.config("vacancy2k", nbasis)
    _check(s, "fp32")


def test_newton_third_law_on_gpu():
    s = small()
    g = run_gpu(s, "fp64", fields=False)
    assert np.abs(g["F"].sum(axis=0)).max() < 1e-9


def test_verlet_matches_oracle_fp64():
    torch = torch_cuda()
    from oracle import csp, verlet
    s = small(cells=(6, 6, 6))
    s["vel"] = W.maxwell(len(s["pos"]), 300.0, 7)
    steps, dt = 10, 0.001
    g = run_gpu(s, "fp64", fields=False)
    m, t = g["model"], g["t"]
    F = torch.tensor(g["F"], device="cuda")
    thermo = torch.zeros((steps, 5), dtype=torch.float64, device="cuda")
    m.verlet_step(t["pos"], t["vel"], F, t["inv_mass"], g["box"], t["types"], t["ids"], dt, steps, thermo)
    m.sync()
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    pos, vel, Fo, log = verlet.run(s["pos"], s["vel"], s["box"], s["ids"], part, s["prm"], s["mass"], dt, steps,
                                   model=ace.AceModel(s["prm"]["ace"]))
    from oracle.neighbors import min_image
    np.testing.assert_allclose(min_image(t["pos"].cpu().numpy() - pos, s["box"]), 0.0, atol=1e-9)
    np.testing.assert_allclose(t["vel"].cpu().numpy(), vel, atol=1e-7)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, atol=1e-8)
    th = thermo.cpu().numpy()
    np.testing.assert_allclose(th[:, 0], [e for e, _, _ in log[1:]], atol=1e-8)
    np.testing.assert_allclose(th[:, 1], [k for _, k, _ in log[1:]], rtol=1e-10, atol=1e-10)
    p_ref = np.array([p for _, _, p in log[1:]]) * 1.0364269e-4
    np.testing.assert_allclose(th[:, 2:], p_ref, atol=1e-8)


def test_autograd_function_matches_finite_differences():
    torch = torch_cuda()
    from paper_2512_07693_gb300.autograd import energy
    s = small()
    g = run_gpu(s, "fp64", fields=False)
    m, t, box = g["model"], g["t"], g["box"]
    pos = t["pos"].clone().requires_grad_(True)
    E = energy(pos, m, box, t["types"], t["ids"])
    (grad,) = torch.autograd.grad(E, pos)
    np.testing.assert_allclose(grad.cpu().numpy(), -g["F"], atol=1e-12)
    h = 1e-5
    rng = np.random.default_rng(0)
    for a in rng.choice(len(s["pos"]), 6, replace=False):
        for c in range(3):
            pp = t["pos"].clone(); pp[a, c] += h
            pm = t["pos"].clone(); pm[a, c] -= h
            ep = float(energy(pp, m, box, t["types"], t["ids"]))
            em = float(energy(pm, m, box, t["types"], t["ids"]))
            assert float(grad[a, c]) == pytest.approx((ep - em) / (2 * h), abs=2e-6)


def test_error_paths():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = small()
    n = len(s["pos"])
    from gpu_helpers import to_dev
    t = to_dev(torch, s)
    box = list(s["box"])
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    m = apip.Apip(s["prm"], n)
    with pytest.raises(apip.ApipError) as e:          # switch before CSP pair detection
        m.energy_forces(t["pos"], box, t["types"], t["ids"], F)
    assert e.value.status == apip.APIP_ERR_STATE
    with pytest.raises(apip.ApipError) as e:          # box smaller than 3 (cutoff + skin)
        m.init_csp_pairs(t["pos"], [10.0, 10.0, 10.0], t["ids"])
    assert e.value.status == apip.APIP_ERR_ARG
    m.init_csp_pairs(t["pos"], box, t["ids"])
    m.sync()
    bad = t["pos"].clone()
    bad[3, 1] = float("nan")
    m.energy_forces(bad, box, t["types"], t["ids"], F)
    with pytest.raises(apip.ApipError) as e:
        m.sync()
    assert e.value.status == apip.APIP_ERR_BAD_INPUT
    small_nb = apip.Apip(s["prm"], n, max_nb=20)
    small_nb.init_csp_pairs(t["pos"], box, t["ids"])
    with pytest.raises(apip.ApipError) as e:
        small_nb.sync()
    assert e.value.status == apip.APIP_ERR_NB_OVERFLOW and "max_nb = 20" in str(e.value)
    # group sizes that are rejected at creation: one the streamed (body order 3)
    # kernel does not provide, and pools that exceed shared memory (the crack
    # basis in float64: 2 atoms x 2 pools x 13188 values x 8 bytes = 422 KB)
    with pytest.raises(apip.ApipError) as e:
        apip.Apip(s["prm"], n, precision="fp64", ace_group=2)
    assert e.value.status == apip.APIP_ERR_ARG
    crack = dict(s["prm"], ace=W.ace_params(8, 4, 4, 2, nbasis(8, 4, 4)))
    with pytest.raises(apip.ApipError) as e:
        apip.Apip(crack, n, precision="fp64", ace_group=2)
    assert e.value.status == apip.APIP_ERR_ARG
    # empty system
    E = torch.ones(1, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"][:0], box, t["types"][:0], t["ids"][:0], F[:0], e_total_out=E)
    m.sync()
    assert float(E.cpu()[0]) == 0.0


def test_atoms_reordered_after_pair_detection():
    """The CSP^list partners are kept by atom id: after the pairs are detected, the
    same atoms passed in another order give the same energies and forces, permuted."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = W.vacancy_crystal(cells=6, sigma=0.06, seed=21)
    nb = nbasis(6, 3, 3)
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP),
               switch=dict(W.SWITCH, d_lo=0.25, d_hi=0.9), ace=W.ace_params(6, 3, 3, 2, nb))
    n = len(s["pos"])
    m = apip.Apip(prm, n, precision="fp64")
    t = to_dev(torch, s)
    box = [float(x) for x in s["box"]]
    m.init_csp_pairs(t["pos"], box, t["ids"])
    out = []
    perm = np.random.default_rng(5).permutation(n)
    for order in (np.arange(n), perm):
        o = torch.tensor(order, device="cuda")
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        m.energy_forces(t["pos"][o].contiguous(), box, t["types"][o].contiguous(), t["ids"][o].contiguous(), F, e)
        m.sync()
        out.append((F.cpu().numpy(), e.cpu().numpy(), m.field("dlam", n).cpu().numpy()))
    m.close()
    (F0, e0, dl0), (F1, e1, dl1) = out
    assert np.count_nonzero(dl0) > 10
    assert np.abs(F1 - F0[perm]).max() < 1e-10
    assert np.abs(e1 - e0[perm]).max() < 1e-10
    np.testing.assert_allclose(dl1, dl0[perm], atol=1e-12)
