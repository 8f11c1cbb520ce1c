"""Pins of the oracle's learned indicator (oracle/mlp.py): the activation
against scipy, descriptors in closed form, back-propagation against finite
differences, Adam against its closed-form first steps, and the full adaptive
force with the learned g against finite differences of the energy."""
import math

import numpy as np
import pytest

from oracle import ace, apip, mlp
from oracle.ftrans import f_trans
from oracle.neighbors import pairs_bruteforce
from paper_2512_07693_gb300 import workloads as W


def test_silu_matches_library():
    sp = pytest.importorskip("scipy.special")
    x = np.linspace(-30, 30, 601)
    np.testing.assert_allclose(mlp.silu(x), x * sp.expit(x), rtol=1e-14, atol=1e-300)
    h = 1e-6
    np.testing.assert_allclose(mlp.silu_deriv(x), (mlp.silu(x + h) - mlp.silu(x - h)) / (2 * h), atol=1e-8)


def test_descriptor_dimer_closed_form():
    r0 = 2.7
    pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0 + r0]])
    i, j, rv, r = pairs_bruteforce(pos, np.array([30.0, 30.0, 30.0]), 5.0)
    G = mlp.descriptors(2, i, r, 5.0, 1.0)
    ref = np.exp(-mlp.ETA * (r0 - mlp.MU) ** 2) * f_trans(r0, 4.0, 5.0)
    np.testing.assert_allclose(G, [ref, ref], atol=1e-15)
    assert mlp.MU[0] == 1.5 and mlp.MU[-1] == 5.0 and mlp.ETA == pytest.approx(1 / (2 * 0.15**2))


def _rand_batch(n=40, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 6, (n, mlp.N_DESC)), rng.uniform(0, 1, n)


def test_input_gradient_fd():
    p = W.mlp_params(3)
    G, _ = _rand_batch()
    g, cache = mlp.forward(p, G)
    dG = mlp.backward(p, cache, np.ones(len(G)))["G"]
    h = 1e-6
    for m in (0, 7, 31):
        Gp, Gm = G.copy(), G.copy()
        Gp[:, m] += h
        Gm[:, m] -= h
        fd = (mlp.forward(p, Gp)[0] - mlp.forward(p, Gm)[0]) / (2 * h)
        np.testing.assert_allclose(dG[:, m], fd, atol=1e-8)


def test_weight_gradients_fd():
    p = W.mlp_params(4)
    G, y = _rand_batch(seed=1)
    loss, grads = mlp.loss_and_grads(p, G, y)
    rng = np.random.default_rng(2)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        for _ in range(3):
            q = {kk: (np.array(v, copy=True) if not isinstance(v, float) else v) for kk, v in p.items()}
            if k == "b4":
                qp, qm = dict(q, b4=q["b4"] + h), dict(q, b4=q["b4"] - h)
                fd = (mlp.loss_and_grads(qp, G, y)[0] - mlp.loss_and_grads(qm, G, y)[0]) / (2 * h)
                assert grads["b4"] == pytest.approx(fd, abs=1e-8)
                break
            idx = tuple(rng.integers(s) for s in q[k].shape)
            qp = {kk: np.array(v, copy=True) if not isinstance(v, float) else v for kk, v in q.items()}
            qm = {kk: np.array(v, copy=True) if not isinstance(v, float) else v for kk, v in q.items()}
            qp[k][idx] += h
            qm[k][idx] -= h
            fd = (mlp.loss_and_grads(qp, G, y)[0] - mlp.loss_and_grads(qm, G, y)[0]) / (2 * h)
            assert grads[k][idx] == pytest.approx(fd, abs=1e-8)


def test_adam_closed_form_first_steps():
    p = dict(a=np.array([1.0, -2.0, 0.5]))
    m = dict(a=np.zeros(3))
    v = dict(a=np.zeros(3))
    g1 = np.array([0.3, -4.0, 1e-3])
    p1 = mlp.adam_step(p, dict(a=g1), m, v, 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, update = -lr g / (|g| + eps)
    np.testing.assert_allclose(p1["a"], p["a"] - 0.01 * g1 / (np.abs(g1) + 1e-8), rtol=1e-12)
    g2 = np.array([-0.1, 1.0, 2e-3])
    p2 = mlp.adam_step(p1, dict(a=g2), m, v, 2, lr=0.01)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.9**2)
    vh = (0.999 * 0.001 * g1**2 + 0.001 * g2**2) / (1 - 0.999**2)
    np.testing.assert_allclose(p2["a"], p1["a"] - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-12)


def learned_system(adds_eam=True):
    s = W.vacancy_crystal(cells=5, sigma=0.08, seed=31)
    nb = len(ace.enumerate_basis(4, 2, 3))
    prm = dict(precise_adds_eam=adds_eam, eam=dict(W.EAM), csp=dict(W.CSP), mlp=W.mlp_params(7),
               switch=dict(W.SWITCH), ace=W.ace_params(4, 2, 3, 2, nb))
    # place the switch window inside the spread of the untrained network's d
    n = len(s["pos"])
    from oracle.neighbors import pairs
    i, j, rv, r = pairs(s["pos"], s["box"], 5.5)
    g, _, _ = mlp.learned_g(n, i, r, prm["mlp"], 5.0, 1.0)
    from oracle.switch import descriptor
    _, d, _, _ = descriptor(n, i, j, r, g, dict(prm["switch"], d_lo=-1e9, d_hi=1e9))
    lo, hi = np.quantile(d, [0.3, 0.8])
    prm["switch"].update(d_lo=float(lo), d_hi=float(hi))
    return s, prm


def test_learned_switch_force_is_minus_gradient():
    s, prm = learned_system()
    model = ace.AceModel(prm["ace"])
    res = apip.energy_forces(s["pos"], s["box"], s["ids"], None, prm, model=model, lam_mode="learned")
    assert np.count_nonzero(res["dlam"]) > 20
    trans = np.nonzero(res["dlam"])[0]
    atoms = [int(trans[0]), int(trans[5]), int(np.nonzero(res["lam"] == 0)[0][0])]
    h = 1e-5
    for a in atoms:
        for c in range(3):
            pp, pm = s["pos"].copy(), s["pos"].copy()
            pp[a, c] += h
            pm[a, c] -= h
            ep = apip.energy_forces(pp, s["box"], s["ids"], None, prm, model=model, lam_mode="learned",
                                    forces=False)["E"]
            em = apip.energy_forces(pm, s["box"], s["ids"], None, prm, model=model, lam_mode="learned",
                                    forces=False)["E"]
            assert res["F"][a, c] == pytest.approx(-(ep - em) / (2 * h), abs=2e-6)
    assert np.abs(res["F"].sum(axis=0)).max() < 1e-10


def test_bf16_rounding_matches_library():
    """The oracle's bfloat16 rounding against torch's (round to nearest even)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.normal(0, 1, 4000), rng.normal(0, 1e-3, 1000) * 1e3, [0.0, -0.0, 1.0, 3.0, 1e-30]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_bf16_training_step_is_the_exact_chain_without_rounding(monkeypatch):
    """With the bfloat16 rounding replaced by the identity, the mixed-precision
    training step is the exact loss and gradient (same chain, no term dropped)."""
    p = W.mlp_params(4)
    G, y = _rand_batch(seed=1)
    loss, grads = mlp.loss_and_grads(p, G, y)
    monkeypatch.setattr(mlp, "bf16", lambda x: np.asarray(x, dtype=np.float64))
    loss_b, grads_b = mlp.loss_and_grads_bf16(p, G, y)
    assert loss_b == pytest.approx(loss, rel=1e-14)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4"):
        np.testing.assert_allclose(grads_b[k], grads[k], rtol=1e-12, atol=1e-15)
    assert grads_b["b4"] == pytest.approx(grads["b4"], rel=1e-12)


def test_bf16_training_step_is_close_to_the_exact_one():
    """bfloat16 operands move each gradient by a few bfloat16 roundings (2^-9)."""
    p = W.mlp_params(4)
    G, y = _rand_batch(seed=1)
    loss, grads = mlp.loss_and_grads(p, G, y)
    loss_b, grads_b = mlp.loss_and_grads_bf16(p, G, y)
    assert loss_b == pytest.approx(loss, rel=2e-2)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4"):
        scale = np.abs(grads[k]).max()
        np.testing.assert_allclose(grads_b[k], grads[k], atol=3e-2 * scale)
