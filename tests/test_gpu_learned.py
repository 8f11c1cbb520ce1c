"""GPU parity of the learned indicator: descriptors, the adaptive energy and
forces with g = MLP(G), the training gradient and the Adam update, against the
FP64 oracle on the same inputs (float32-rounded weights, bfloat16-rounded
descriptors)."""
import numpy as np
import pytest

from gpu_helpers import run_gpu, run_oracle, to_dev, torch_cuda
from oracle import ace, mlp
from oracle.neighbors import pairs
from oracle.switch import descriptor
from paper_2512_07693_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def f32(params):
    """Weights as the library holds them (float32), back in float64 for the oracle."""
    from paper_2512_07693_gb300 import apip
    return apip.mlp_unflat(apip.mlp_flat(params))


def learned_system(seed=31, cells=6):
    """An untrained network with its output layer scaled by 30, so that g varies over
    a range like a trained indicator's (an untrained one is nearly constant, and a
    switch window inside its tiny spread would amplify float32 rounding by ~1e3);
    the window spans the 5-95 % quantiles of the resulting d."""
    s = W.vacancy_crystal(cells=cells, sigma=0.08, seed=seed)
    nb = len(ace.enumerate_basis(6, 3, 3))
    net = W.mlp_params(7)
    net["w4"] = 30.0 * net["w4"]
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP), mlp=f32(net),
               switch=dict(W.SWITCH), ace=W.ace_params(6, 3, 3, 2, nb))
    n = len(s["pos"])
    i, j, rv, r = pairs(s["pos"], s["box"], 5.5)
    g, _, _ = mlp.learned_g(n, i, r, prm["mlp"], 5.0, 1.0)
    _, d, _, _ = descriptor(n, i, j, r, g, dict(prm["switch"], d_lo=-1e9, d_hi=1e9))
    lo = float(np.quantile(d, 0.2))
    prm["switch"].update(d_lo=lo, d_hi=lo + 0.5 * float(g.max() - g.min()))
    s["prm"] = prm
    return s


@pytest.mark.parametrize("prec,tolF,tolE", [("fp64", 1e-9, 1e-9), ("fp32", 2e-4, 1e-5)])
def test_learned_switch_parity(prec, tolF, tolE):
    s = learned_system()
    o = run_oracle(s, lam_mode="learned")
    assert np.count_nonzero(o["dlam"]) > 50
    g = run_gpu(s, precision=prec, lam_mode="learned")
    err = np.abs(g["F"] - o["F"]).max()
    assert err <= tolF, err
    # float64: pair terms cancel to rounding; float32: both atoms of a gathered
    # pair evaluate it separately in float32, so the sum is ~N eps |F|
    assert np.abs(g["F"].sum(axis=0)).max() < (1e-8 if prec == "fp64" else 1e-4)
    if prec == "fp64":
        np.testing.assert_allclose(g["g"], o["g"], atol=1e-12)
        np.testing.assert_allclose(g["lam"], o["lam"], atol=1e-12)
        np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=tolE)
    else:
        # float32 g: ~1e-6 of its range from the network's multiply-adds
        np.testing.assert_allclose(g["g"], o["g"], atol=1e-5 * np.abs(o["g"]).max())
        np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=tolE, rtol=0)
    # the total is the sum of every atom's energy: one partial per block of the
    # learned pass 1 (its blocks are smaller than the other passes')
    n = len(s["pos"])
    assert abs(g["E"] - g["e_atom"].sum()) <= (1e-9 if prec == "fp64" else 1e-6) * n
    assert abs(g["E"] - o["E"]) <= tolE * n


def _ap_energy_error(s, prm, lam_mode, params=None):
    """x = |{lam > 0}| / N and the RMS over atoms of the adaptive energy error
    relative to the precise model, the constant bulk offset removed:
    err_i = E_i^AP - E_i^prec + (1 - lam_i) dE^(0) = -(1 - lam_i)(dE_i - dE^(0))."""
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    n = len(s["pos"])
    t = to_dev(torch, s)
    box = [float(b) for b in s["box"]]
    out = {}
    for mode in ("const1", lam_mode):
        m = apip.Apip(prm, n, precision="fp32", lam_mode=mode)
        if mode == "paper":
            m.init_csp_pairs(t["pos"], box, t["ids"])
        if mode == "learned":
            m.set_mlp(params)
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        e = torch.empty(n, dtype=torch.float64, device="cuda")
        m.energy_forces(t["pos"], box, t["types"], t["ids"], F, e_atom_out=e)
        m.sync()
        out[mode] = (e.cpu().numpy(), m.field("lam", n).cpu().numpy(), m.field("e_eam", n).cpu().numpy(),
                     m.field("d", n).cpu().numpy())
        m.close()
    return out


def test_trained_indicator_beats_csp_at_equal_ace_fraction():
    """The network trained on the method's own |dE - dE^(0)| selects the atoms
    whose fast-model energy is wrong better than CSP^list does: at the same ACE
    fraction x it leaves a smaller energy error."""
    torch_cuda()
    from paper_2512_07693_gb300 import apip, train
    prm = W.config("vacancy2k", apip.apip_ace_basis_size)["prm"]
    G, y, ref = train.make_dataset(prm, n_configs=60, cells=10)
    params, hist = train.train(G, y, epochs=20, batch=4096, lr=1e-3, prm=prm)
    assert len(hist) == 21 and hist[-1] < 0.5 * hist[0]   # against the untrained network
    rms = {"paper": [], "learned": []}
    held_out = [k for k in range(1000, 1100) if W.training_config(k, cells=10)["temp"] < 700.0][:4]
    for k in held_out:
        s = W.training_config(k, cells=10)
        paper = _ap_energy_error(s, prm, "paper")
        e_prec, _, e_eam, _ = paper["const1"]
        dE = e_prec - e_eam
        e_ap, lam_p, _, _ = paper["paper"]
        x = float((lam_p > 0).mean())
        rms["paper"].append(np.sqrt(np.mean(((1 - lam_p) * (dE - ref)) ** 2)))
        # learned switch with its window placed to give the same x
        wide = dict(prm, switch=dict(prm["switch"], d_lo=-1e3, d_hi=1e3))
        d = _ap_energy_error(s, wide, "learned", params)["learned"][3]
        lo = float(np.quantile(d, 1.0 - x))
        width = 0.25 * float(np.std(d))
        tuned = dict(prm, switch=dict(prm["switch"], d_lo=lo, d_hi=lo + width))
        lam_l = _ap_energy_error(s, tuned, "learned", params)["learned"][1]
        assert abs((lam_l > 0).mean() - x) < 0.02
        rms["learned"].append(np.sqrt(np.mean(((1 - lam_l) * (dE - ref)) ** 2)))
    assert np.mean(rms["learned"]) < np.mean(rms["paper"]), rms


def _bf16(x):
    """Round float64 -> float32 -> bfloat16 (nearest even) -> float64."""
    f = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_descriptors_bf16():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    s = learned_system(cells=6)
    n = len(s["pos"])
    m = apip.Apip(s["prm"], n, precision="fp32", lam_mode="const0")
    t = to_dev(torch, s)
    out = torch.empty((n, 32), dtype=torch.int16, device="cuda")
    m.descriptors(t["pos"], list(s["box"]), t["ids"], out)
    m.sync()
    got = out.cpu().numpy().astype(np.int16).view(np.uint16).astype(np.uint32) << 16
    got = got.view(np.float32).astype(np.float64)
    i, j, rv, r = pairs(s["pos"], s["box"], 5.5)
    ref = mlp.descriptors(n, i, r, 5.0, 1.0)
    # float32 descriptors may straddle a bfloat16 rounding boundary: one bf16 ulp
    np.testing.assert_allclose(got, _bf16(ref), rtol=2 ** -7, atol=1e-30)
    assert np.mean(got == _bf16(ref)) > 0.98


def test_training_gradient_and_adam_match_oracle():
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    rng = np.random.default_rng(5)
    B = 1000
    G = _bf16(rng.uniform(0, 6, (B, 32)))
    y = rng.uniform(0, 0.5, B).astype(np.float32)
    w = f32(W.mlp_params(9))
    # the training step's reading: bfloat16 GEMM operands, float32 accumulation
    loss_ref, grads_ref = mlp.loss_and_grads_bf16(w, G, y.astype(np.float64))
    flat = torch.tensor(apip.mlp_flat(w), device="cuda")
    Gd = torch.tensor(G.astype(np.float32), device="cuda").to(torch.bfloat16).contiguous()
    yd = torch.tensor(y, device="cuda")
    grad = torch.empty(apip.APIP_MLP_NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    s = learned_system(cells=6)
    m = apip.Apip(s["prm"], 8, precision="fp32", lam_mode="const0")
    apip.apip_mlp_loss_grad(m.ctx, Gd, yd, B, flat, grad, loss)
    torch.cuda.synchronize()
    assert float(loss.cpu()[0]) == pytest.approx(loss_ref, rel=1e-5)
    g_ref = apip.mlp_flat(grads_ref).astype(np.float64)
    g_got = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(g_ref).max()
    np.testing.assert_allclose(g_got, g_ref, atol=2e-5 * scale)
    # one Adam step from zero moments, compared with the oracle's float64 update
    mom = torch.zeros_like(grad)
    var = torch.zeros_like(grad)
    apip.apip_mlp_adam(m.ctx, flat, grad, mom, var, 1, 1e-3)
    torch.cuda.synchronize()
    zeros = {k: np.zeros_like(np.asarray(v, dtype=np.float64)) for k, v in w.items()}
    new = mlp.adam_step(w, apip.mlp_unflat(g_got), dict(zeros), {k: np.zeros_like(v) for k, v in zeros.items()}, 1)
    np.testing.assert_allclose(flat.cpu().numpy(), apip.mlp_flat(new), atol=2e-7)
