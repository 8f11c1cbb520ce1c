"""Training of the learned indicator with the library's own kernels.

Labels are generated by the method itself: for every training configuration
the library evaluates the precise model on all atoms (lam = 1) and the fast
model, and the label of atom i is y_i = |dE_i - dE^(0)| with dE = E^prec - E^EAM
and dE^(0) its value in the perfect 0 K lattice; the inputs are the atoms'
radial descriptors (bfloat16).  The network is then fitted on the GPU with the
library's loss-gradient and Adam kernels.  PyTorch only holds device memory.
"""
import numpy as np

from . import apip, workloads as W


def _delta(model, n, e_atom, torch):
    """dE_i = E_i^prec - E_i^EAM of the last lam = 1 call: with lam = 1 the per-atom
    energy is E^prec, and the EAM part is the e_eam field."""
    return e_atom - model.field("e_eam", n)


def make_dataset(prm, n_configs, cells=10, base_seed=5, precision="fp32"):
    """Descriptors (torch bfloat16 [N, 32]) and labels (float32 [N]) on the GPU."""
    import torch
    dev = torch.device("cuda")
    nmax = 2 * cells ** 3 + 8
    model = apip.Apip(prm, nmax, precision=precision, lam_mode="const1")
    types = torch.zeros(nmax, dtype=torch.int32, device=dev)

    def run(pos, box, ids):
        n = pos.shape[0]
        F = torch.empty((n, 3), dtype=torch.float64, device=dev)
        e = torch.empty(n, dtype=torch.float64, device=dev)
        model.energy_forces(pos, box, types[:n], ids, F, e_atom_out=e)
        d = _delta(model, n, e, torch)
        G = torch.empty((n, 32), dtype=torch.bfloat16, device=dev)
        model.descriptors(pos, box, ids, G)
        model.sync()
        return d, G

    pos0, box0 = W.bcc(cells, cells, cells)
    n0 = len(pos0)
    d0, _ = run(torch.tensor(pos0, device=dev), list(box0), torch.arange(n0, dtype=torch.int32, device=dev))
    ref = float(d0.mean())
    Gs, ys = [], []
    for k in range(n_configs):
        s = W.training_config(k, cells=cells, base_seed=base_seed)
        n = len(s["pos"])
        d, G = run(torch.tensor(s["pos"], device=dev), list(s["box"]),
                   torch.arange(n, dtype=torch.int32, device=dev))
        Gs.append(G)
        ys.append((d - ref).abs().to(torch.float32))
    model.close()
    G = torch.cat(Gs)
    y = torch.cat(ys)
    perm = torch.tensor(np.random.default_rng(base_seed).permutation(len(y)), device=dev)
    return G[perm].contiguous(), y[perm].contiguous(), ref


def train(G, y, epochs=20, batch=65536, lr=1e-3, seed=7, prm=None, log_every=0):
    """Adam on mean squared error; returns (float32 parameter tensor, losses per epoch)."""
    import torch
    dev = G.device
    ctx_prm = prm if prm is not None else W.config("vacancy2k", apip.apip_ace_basis_size, scale=6)["prm"]
    holder = apip.Apip(ctx_prm, 8, precision="fp32", lam_mode="const0")
    p = torch.tensor(apip.mlp_flat(W.mlp_params(seed)), device=dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grad = torch.empty_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    n = len(y)
    batch = min(batch, n)
    nb = n // batch
    t = 0
    history = []
    for ep in range(epochs):
        acc = 0.0
        for b in range(nb):
            t += 1
            apip.apip_mlp_loss_grad(holder.ctx, G[b * batch:(b + 1) * batch], y[b * batch:(b + 1) * batch], batch,
                                    p, grad, loss)
            apip.apip_mlp_adam(holder.ctx, p, grad, m, v, t, lr)
            acc += float(loss.item()) if (log_every and b % log_every == 0) else 0.0
        apip.apip_mlp_loss_grad(holder.ctx, G[:batch], y[:batch], batch, p, grad, loss)
        history.append(float(loss.item()))
    holder.close()
    return p, history
