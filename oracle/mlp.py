"""Learned switching quantity: a small MLP on radial descriptors whose output
is used as the atomic quantity g_k of the locally averaged descriptor (Eq. 6).
Oracle: test infrastructure only.

The paper allows any differentiable atomic quantity g_k that depends on
interatomic distances only (main text after Eq. 5); the workload definition
asks for an MLP on cheap radial descriptors trained on the per-atom energy
difference of the two models.  Readings (none of this is in the paper):

  descriptors  G_im = sum_{j, r_ij < rc} exp(-eta (r_ij - mu_m)^2) fc(r_ij),
               m = 0..31, mu_m evenly spaced on [1.5, 5.0] A, eta = 1/(2 * 0.15^2) A^-2,
               fc(r) = f_trans(r, rc - 1, rc), rc = 5 A (the ACE cutoff)
  network      x0 = s_in G;  h_k = silu(W_k h_{k-1} + b_k), k = 1..3 (64 wide);
               g = w4 . h3 + b4,  silu(x) = x / (1 + exp(-x)),  s_in = 0.25
  label        y_i = |dE_i - dE^(0)|, dE = E^prec - E^EAM, dE^(0) its value in the
               perfect 0 K lattice (the energy analogue of the reference d^(0) of Eq. 6)
  loss         mean over the batch of (g_i - y_i)^2
  optimiser    Adam (Kingma & Ba 2015): lr 1e-3, beta1 0.9, beta2 0.999, eps 1e-8
  training     "BF16 inputs, FP32 accumulate" (the workload): every matrix product of
               the training step takes its operands rounded to bfloat16 (round to
               nearest even) -- the weights W1, W2, W3, the activations x0, h1, h2,
               h3 and the back-propagated gradients dz1, dz2, dz3, dg -- and sums
               exactly; the elementwise steps (bias, SiLU, its derivative, the
               output layer's dot product g = w4 . h3 + b4 and the loss) are not
               rounded (``loss_and_grads_bf16``).  Inference (the switch and its
               forces) keeps the plain float64 definition above.
"""
import numpy as np

from .ftrans import f_trans, f_trans_deriv

N_DESC = 32
MU = np.linspace(1.5, 5.0, N_DESC)
ETA = 1.0 / (2.0 * 0.15 ** 2)
S_IN = 0.25
WIDTH = 64


def _fc(r, rc, width):
    return f_trans(r, rc - width, rc), f_trans_deriv(r, rc - width, rc)


def radial_features(r, rc, width):
    """phi[k, m] = exp(-eta (r_k - mu_m)^2) fc(r_k) and d phi / d r."""
    r = np.asarray(r, dtype=np.float64)
    fc, dfc = _fc(r, rc, width)
    x = r[:, None] - MU[None, :]
    e = np.exp(-ETA * x * x)
    phi = e * fc[:, None]
    dphi = e * (-2.0 * ETA * x) * fc[:, None] + e * dfc[:, None]
    return phi, dphi


def descriptors(n, i, r, rc, width):
    """G[n, 32] from a full pair list (i, r), pairs with r < rc."""
    sel = r < rc
    phi, _ = radial_features(r[sel], rc, width)
    G = np.zeros((n, N_DESC))
    for m in range(N_DESC):
        G[:, m] = np.bincount(i[sel], weights=phi[:, m], minlength=n)
    return G


def silu(x):
    return x / (1.0 + np.exp(-x))


def silu_deriv(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def forward(p, G):
    """g[n] and the cache for backward."""
    x0 = S_IN * np.asarray(G, dtype=np.float64)
    z1 = x0 @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = silu(z3)
    g = h3 @ p["w4"] + p["b4"]
    return g, (x0, z1, h1, z2, h2, z3, h3)


def backward(p, cache, dg):
    """Gradients of sum_i dg_i g_i with respect to the weights and to G."""
    x0, z1, h1, z2, h2, z3, h3 = cache
    out = {}
    out["w4"] = h3.T @ dg
    out["b4"] = float(np.sum(dg))
    d3 = np.outer(dg, p["w4"]) * silu_deriv(z3)
    out["W3"] = d3.T @ h2
    out["b3"] = d3.sum(axis=0)
    d2 = (d3 @ p["W3"]) * silu_deriv(z2)
    out["W2"] = d2.T @ h1
    out["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * silu_deriv(z1)
    out["W1"] = d1.T @ x0
    out["b1"] = d1.sum(axis=0)
    out["G"] = S_IN * (d1 @ p["W1"])
    return out


def loss_and_grads(p, G, y):
    g, cache = forward(p, G)
    r = g - y
    loss = float(np.mean(r * r))
    grads = backward(p, cache, 2.0 * r / len(y))
    return loss, grads


def bf16(x):
    """Round to the nearest bfloat16 (ties to even) through float32, as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def loss_and_grads_bf16(p, G, y):
    """Loss and weight gradients of one training step with bfloat16 GEMM operands
    (module docstring): the same chain as forward/backward, each matrix product's
    inputs rounded to bfloat16.  Bias gradients are sums of the rounded dz; the
    output layer's weight gradient pairs the rounded dg with the rounded h3."""
    x0 = S_IN * np.asarray(G, dtype=np.float64)          # G holds bfloat16 values; 0.25 G is exact
    W1, W2, W3 = bf16(p["W1"]), bf16(p["W2"]), bf16(p["W3"])
    z1 = x0 @ W1.T + p["b1"]
    h1 = bf16(silu(z1))
    z2 = h1 @ W2.T + p["b2"]
    h2 = bf16(silu(z2))
    z3 = h2 @ W3.T + p["b3"]
    h3 = silu(z3)
    g = h3 @ p["w4"] + p["b4"]
    r = g - y
    loss = float(np.mean(r * r))
    dg = 2.0 * r / len(y)
    d3 = bf16(np.outer(dg, p["w4"]) * silu_deriv(z3))
    d2 = bf16((d3 @ W3) * silu_deriv(z2))
    d1 = bf16((d2 @ W2) * silu_deriv(z1))
    dgb, h3b = bf16(dg), bf16(h3)
    out = {"W3": d3.T @ h2, "b3": d3.sum(axis=0), "W2": d2.T @ h1, "b2": d2.sum(axis=0),
           "W1": d1.T @ x0, "b1": d1.sum(axis=0), "w4": h3b.T @ dgb, "b4": float(np.sum(dgb))}
    return loss, out


def adam_step(p, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); m, v dicts updated in place."""
    new = {}
    for k in p:
        gk = np.asarray(grads[k], dtype=np.float64)
        m[k] = b1 * m[k] + (1.0 - b1) * gk
        v[k] = b2 * v[k] + (1.0 - b2) * gk * gk
        mh = m[k] / (1.0 - b1 ** t)
        vh = v[k] / (1.0 - b2 ** t)
        new[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
        if k == "b4":
            new[k] = float(new[k])
    return new


def learned_g(n, i, r, p, rc, width):
    G = descriptors(n, i, r, rc, width)
    g, cache = forward(p, G)
    return g, G, cache


def learned_force(n, i, j, rvec, r, p, c, rc, width):
    """-grad sum_j c_j g_j with c held fixed: for each pair (j, k) with r < rc,
    v = c_j sum_m (dg_j/dG_jm) phi_m'(r_jk), F_k -= v e_jk, F_j += v e_jk."""
    G = descriptors(n, i, r, rc, width)
    _, cache = forward(p, G)
    dG = backward(p, cache, np.asarray(c, dtype=np.float64))["G"]      # c_j dg_j/dG_jm
    sel = r < rc
    jj, kk, rv, rr = i[sel], j[sel], rvec[sel], r[sel]
    _, dphi = radial_features(rr, rc, width)
    v = np.einsum("km,km->k", dG[jj], dphi)
    f = (v / rr)[:, None] * rv
    F = np.zeros((n, 3))
    for comp in range(3):
        F[:, comp] -= np.bincount(kk, weights=f[:, comp], minlength=n)
        F[:, comp] += np.bincount(jj, weights=f[:, comp], minlength=n)
    return F
