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
    """Adam on mean squared error; returns (float32 parameter tensor, losses): the
    loss on the first batch before training, then after each epoch."""
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
    apip.apip_mlp_loss_grad(holder.ctx, G[:batch], y[:batch], batch, p, grad, loss)
    history = [float(loss.item())]
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


# Algorithmic flops of one training sample: the forward products (32*64 + 2*64*64
# + 64 multiply-adds), the back-propagation to h1 (2*64*64) and the weight
# gradients (as many as the forward), two flops per multiply-add.
FLOP_PER_SAMPLE = 2 * ((32 * 64 + 2 * 64 * 64 + 64) * 2 + 2 * 64 * 64)


def step_time(batch=65536, steps=50, warmup=5, seed=3):
    """Device time of one training step (loss and gradient, then Adam) on a batch
    of seeded synthetic descriptors, timed with CUDA events on the stream the
    kernels run on; returns (microseconds per step, TFLOP/s algorithmic)."""
    import torch
    dev = torch.device("cuda")
    rng = np.random.default_rng(seed)
    G = torch.tensor(rng.uniform(0.0, 3.0, (batch, 32)).astype(np.float32), device=dev).to(torch.bfloat16)
    y = torch.tensor(rng.uniform(0.0, 0.5, batch).astype(np.float32), device=dev)
    prm = W.config("vacancy2k", apip.apip_ace_basis_size, scale=6)["prm"]
    holder = apip.Apip(prm, 8, precision="fp32", lam_mode="const0")
    p = torch.tensor(apip.mlp_flat(W.mlp_params(7)), device=dev)
    m, v, grad = torch.zeros_like(p), torch.zeros_like(p), torch.empty_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()   # the kernels' stream (the bindings' default)
    t = 0
    for _ in range(warmup):
        t += 1
        apip.apip_mlp_loss_grad(holder.ctx, G, y, batch, p, grad, loss)
        apip.apip_mlp_adam(holder.ctx, p, grad, m, v, t, 1e-4)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        t += 1
        apip.apip_mlp_loss_grad(holder.ctx, G, y, batch, p, grad, loss)
        apip.apip_mlp_adam(holder.ctx, p, grad, m, v, t, 1e-4)
    b.record(stream)
    torch.cuda.synchronize()
    holder.sync()
    holder.close()
    us = a.elapsed_time(b) * 1e3 / steps
    return us, FLOP_PER_SAMPLE * batch / (us * 1e-6) / 1e12


def _energies(prm, s, lam_mode, params=None):
    """Per-atom energies, lam, E^EAM and d of one configuration (float32 path)."""
    import torch
    dev = torch.device("cuda")
    n = len(s["pos"])
    pos = torch.tensor(s["pos"], dtype=torch.float64, device=dev)
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    types = torch.zeros(n, dtype=torch.int32, device=dev)
    box = [float(b) for b in s["box"]]
    m = apip.Apip(prm, n, precision="fp32", lam_mode=lam_mode)
    if lam_mode == "paper":
        m.init_csp_pairs(pos, box, ids)
    if lam_mode == "learned":
        m.set_mlp(params)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    m.energy_forces(pos, box, types, ids, F, e_atom_out=e)
    m.sync()
    out = (e.cpu().numpy(), m.field("lam", n).cpu().numpy(), m.field("e_eam", n).cpu().numpy(),
           m.field("d", n).cpu().numpy())
    m.close()
    return out


def compare_switches(prm, params, ref, configs, cells=10):
    """On held-out configurations: the RMS over atoms of the adaptive energy error
    against the precise model, bulk offset removed, -(1 - lam_i)(dE_i - dE^(0)),
    for the paper's switch and for the learned switch with its window placed at
    the same ACE fraction x."""
    rows = []
    for k in configs:
        s = W.training_config(k, cells=cells)
        e_prec, _, e_eam, _ = _energies(prm, s, "const1")
        dE = e_prec - e_eam
        _, lam_p, _, _ = _energies(prm, s, "paper")
        x = float((lam_p > 0).mean())
        wide = dict(prm, switch=dict(prm["switch"], d_lo=-1e3, d_hi=1e3))
        d = _energies(wide, s, "learned", params)[3]
        lo = float(np.quantile(d, 1.0 - x))
        tuned = dict(prm, switch=dict(prm["switch"], d_lo=lo, d_hi=lo + 0.25 * float(np.std(d))))
        lam_l = _energies(tuned, s, "learned", params)[1]
        rows.append(dict(config=k, temp=s["temp"], x_paper=x, x_learned=float((lam_l > 0).mean()),
                         rms_paper=float(np.sqrt(np.mean(((1 - lam_p) * (dE - ref)) ** 2))),
                         rms_learned=float(np.sqrt(np.mean(((1 - lam_l) * (dE - ref)) ** 2)))))
    return rows


def main():
    """The learned-indicator training workload: label generation on n_configs
    2000-site crystals with point defects, then Adam epochs; prints a JSON summary
    and saves the float32 weights."""
    import argparse
    import json
    import time
    import torch
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--configs", type=int, default=50000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default="mlp_weights.npy")
    ap.add_argument("--held-out", type=int, default=8, help="configurations for the switch comparison")
    ap.add_argument("--step-bench", action="store_true",
                    help="only time the training step on synthetic descriptors (--batch, --steps)")
    ap.add_argument("--steps", type=int, default=50)
    args = ap.parse_args()
    build.build()
    if args.step_bench:
        us, tf = step_time(args.batch, args.steps)
        print(json.dumps({"batch": args.batch, "steps": args.steps, "us_per_step": us, "tflops": tf}))
        return
    prm = W.config("vacancy2k", apip.apip_ace_basis_size)["prm"]
    torch.cuda.synchronize()
    t0 = time.time()
    G, y, ref = make_dataset(prm, args.configs)
    torch.cuda.synchronize()
    t1 = time.time()
    params, hist = train(G, y, epochs=args.epochs, batch=args.batch, lr=args.lr, prm=prm)
    torch.cuda.synchronize()
    t2 = time.time()
    np.save(args.out, params.cpu().numpy())
    n_atoms = int(len(y))
    del G, y
    held = [k for k in range(10 ** 6, 10 ** 6 + 400) if W.training_config(k)["temp"] < 700.0][:args.held_out]
    rows = compare_switches(prm, params, ref, held)
    print(json.dumps({
        "configs": args.configs, "atoms": n_atoms, "epochs": args.epochs, "batch": args.batch,
        "label_and_descriptor_s": t1 - t0, "training_s": t2 - t1,
        "label_atoms_per_s": n_atoms / (t1 - t0), "training_atom_epochs_per_s": n_atoms * args.epochs / (t2 - t1),
        "loss_per_epoch": hist, "dE0": ref,
        "switch_comparison": rows,
        "mean_rms_paper": float(np.mean([r["rms_paper"] for r in rows])),
        "mean_rms_learned": float(np.mean([r["rms_learned"] for r in rows]))}))


if __name__ == "__main__":
    main()
