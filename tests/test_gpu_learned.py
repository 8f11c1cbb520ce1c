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
    s = W.vacancy_crystal(cells=cells, sigma=0.08, seed=seed)
    nb = len(ace.enumerate_basis(6, 3, 3))
    prm = dict(precise_adds_eam=True, eam=dict(W.EAM), csp=dict(W.CSP), mlp=f32(W.mlp_params(7)),
               switch=dict(W.SWITCH), ace=W.ace_params(6, 3, 3, 2, nb))
    n = len(s["pos"])
    i, j, rv, r = pairs(s["pos"], s["box"], 5.5)
    g, _, _ = mlp.learned_g(n, i, r, prm["mlp"], 5.0, 1.0)
    _, d, _, _ = descriptor(n, i, j, r, g, dict(prm["switch"], d_lo=-1e9, d_hi=1e9))
    lo, hi = np.quantile(d, [0.3, 0.8])
    prm["switch"].update(d_lo=float(lo), d_hi=float(hi))
    s["prm"] = prm
    return s


@pytest.mark.parametrize("prec,tolF,tolE", [("fp64", 1e-9, 1e-9), ("fp32", 2e-4, 1e-5)])
def test_learned_switch_parity(prec, tolF, tolE):
    s = learned_system()
    o = run_oracle(s, lam_mode="learned")
    assert np.count_nonzero(o["dlam"]) > 50
    g = run_gpu(s, precision=prec, lam_mode="learned")
    if prec == "fp64":
        np.testing.assert_allclose(g["g"], o["g"], atol=1e-12)
        np.testing.assert_allclose(g["lam"], o["lam"], atol=1e-12)
    else:
        np.testing.assert_allclose(g["g"], o["g"], atol=1e-5)
    np.testing.assert_allclose(g["e_atom"], o["e_atom"], atol=tolE + 1e-6 * (prec == "fp32"))
    err = np.abs(g["F"] - o["F"]).max()
    assert err <= tolF, err
    assert np.abs(g["F"].sum(axis=0)).max() < 1e-8


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
    loss_ref, grads_ref = mlp.loss_and_grads(w, G, y.astype(np.float64))
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
