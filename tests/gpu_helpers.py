"""Shared helpers of the GPU tests: run one configuration through the C ABI
and through the CPU oracle on the same seeded inputs."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(torch, s):
    dev = torch.device("cuda")
    return dict(pos=torch.tensor(s["pos"], dtype=torch.float64, device=dev).contiguous(),
                ids=torch.tensor(s["ids"], dtype=torch.int32, device=dev),
                types=torch.tensor(s["types"], dtype=torch.int32, device=dev),
                vel=torch.tensor(s["vel"], dtype=torch.float64, device=dev).contiguous(),
                inv_mass=torch.tensor(1.0 / (s["mass"] * 1.0364269e-4), dtype=torch.float64, device=dev))


def run_gpu(s, precision="fp64", lam_mode="paper", grad_lambda=True, max_nb=96, fields=True, prm=None, ace_group=0,
            mixing="energy", lam_fixed=None, deterministic=False):
    torch = torch_cuda()
    from paper_2512_07693_gb300 import apip
    prm = prm or s["prm"]
    n = len(s["pos"])
    m = apip.Apip(prm, n, precision=precision, lam_mode=lam_mode, grad_lambda=grad_lambda, max_nb=max_nb,
                  ace_group=ace_group, mixing=mixing, deterministic=deterministic)
    t = to_dev(torch, s)
    if lam_fixed is not None:
        m.set_lam_fixed(torch.tensor(lam_fixed, dtype=torch.float64, device="cuda"))
    box = [float(x) for x in s["box"]]
    if lam_mode == "paper":
        m.init_csp_pairs(t["pos"], box, t["ids"])
    if lam_mode == "learned":
        flat = torch.tensor(apip.mlp_flat(prm["mlp"]), device="cuda")
        m.set_mlp(flat)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    ea = torch.empty(n, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.energy_forces(t["pos"], box, t["types"], t["ids"], F, ea, E)
    m.sync()
    out = dict(F=F.cpu().numpy(), e_atom=ea.cpu().numpy(), E=float(E.cpu()[0]), model=m, t=t, box=box)
    if fields:
        for k in ("g", "d", "wbar", "lam", "dlam", "e_eam", "e_ace", "zeta", "nnb", "ace_list"):
            out[k] = m.field(k, n).cpu().numpy()
        out["nblist"] = m.field("nblist", n).cpu().numpy()
        out["csp"] = m.field("csp", n).cpu().numpy()
        out["count"] = int((out["lam"] > 0).sum())
    return out


def run_oracle(s, lam_mode="paper", grad_lambda=True, prm=None, model=None, mixing="energy", lam_const=None):
    from oracle import ace, apip, csp
    prm = prm or s["prm"]
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], prm["csp"]["rcut"], prm["csp"]["nnb"])
    model = model or ace.AceModel(prm["ace"])
    res = apip.energy_forces(s["pos"], s["box"], s["ids"], part, prm, model=model, lam_mode=lam_mode,
                             grad_lambda=grad_lambda, mixing=mixing, lam_const=lam_const)
    res["partners"] = part
    return res
