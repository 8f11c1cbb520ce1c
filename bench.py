#!/usr/bin/env python
"""Throughput of the adaptive-precision (AP) EAM+ACE MD step on one GB300.

One "step" is one velocity-Verlet NVE step of the whole hot path (neighbour
check/rebuild, EAM pass, CSP^list g, switch, compaction, ACE forward+adjoint on
the compacted atoms, grad-lambda forces, float64 reductions, integrator) on the
void250k workload: a 50^3-cell bcc crystal with a central void of radius 15 A
(248 757 atoms, 300 K), ACE n_max 6 / l_max 3 / nu <= 3, float32 pair
arithmetic with float64 positions, velocities, forces and reductions.

Prints one JSON line (rank 0).  Metric: atom-steps/s of the adaptive run; the
all-ACE run on the same GPU, the NVE drift and the roofline of the dominant
kernel are reported beside it.  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (a bounded sample of the same workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): replicas only, one independent system per rank.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "void250k"
METRIC = "atom-steps/s adaptive EAM+ACE vs all-ACE on 1 GB300; NVE drift eV/atom/ps"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2, written between timed steps
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes (read + write) per launch of the step's dominant kernels on this
# workload, from one ncu capture of the current kernels (profiles/*_void250k.md),
# per launch (the Verlet one per half-step launch); a kernel changed since its
# capture has no entry
NCU_TRAFFIC = {"ace": 3.370752e6, "pass2": 69.671680e6 + 1.681664e6, "prep": 13.949184e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ace-steps", type=int, default=5, help="steps of the all-ACE comparison run")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--drift-steps", type=int, default=10000,
                    help="NVE steps after the timed run over which the energy drift is fitted (10 ps)")
    ap.add_argument("--ace-group", type=int, default=0, choices=[0, 1, 2, 4, 8, 32],
                    help="compacted atoms per ACE thread block (0: library default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=None,
                    help="scale the void workload to cells^3 (small cases for profiling; not the metric)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_ms(torch, total_ms, world, device):
    """The job's timed total: the maximum over the ranks (all-reduce MAX); each rank
    runs an independent replica, so the job ends with its slowest rank."""
    if world <= 1:
        return total_ms
    tt = torch.tensor([total_ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
    return float(tt)


def job_value(world, n_atoms, steps, total_ms):
    """Whole-job atom-steps/s: the atom-steps of all ranks over the job's time."""
    return world * n_atoms * steps / (total_ms * 1e-3)


# ------------------------------------------------------------------ oracle
def oracle_sample(steps_budget_s, target_s):
    """Time the FP64 CPU oracle on a shrunken copy of the workload recipe
    (same lattice, void radius scaled with the box, same potentials)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import ace, apip as oapip, csp
    from paper_2512_07693_gb300 import workloads as W
    nb = lambda a, b, c: len(ace.enumerate_basis(a, b, c))
    cells = 12
    s = W.config(WORKLOAD, nb, scale=cells)
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    model = ace.AceModel(s["prm"]["ace"])
    t0 = time.perf_counter()
    reps = 0
    while True:
        res = oapip.energy_forces(s["pos"], s["box"], s["ids"], part, s["prm"], model=model)
        reps += 1
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    n = len(s["pos"])
    return dict(value=n * reps / dt, n=n, reps=reps, seconds=dt, x=len(res["P"]) / n, cells=cells)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import ace, apip as oapip, csp
    from paper_2512_07693_gb300 import workloads as W
    nb = lambda a, b, c: len(ace.enumerate_basis(a, b, c))
    cells = 6
    s = W.config(WORKLOAD, nb, scale=cells)
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    model = ace.AceModel(s["prm"]["ace"])
    from oracle import verlet
    n = len(s["pos"])
    pos, vel = s["pos"], s["vel"]
    _, _, _, _ = verlet.run(pos, vel, s["box"], s["ids"], part, s["prm"], s["mass"], 0.001, args.warmup, model=model)
    t0 = time.perf_counter()
    _, _, _, log = verlet.run(pos, vel, s["box"], s["ids"], part, s["prm"], s["mass"], 0.001, args.steps, model=model)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    sample = f"{WORKLOAD} recipe at {cells}^3 cells ({n} atoms), FP64 numpy oracle, velocity-Verlet steps"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "atoms": n, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# -------------------------------------------------------------------- clocks
def clocks_start():
    path = tempfile.mktemp(prefix="clk_", suffix=".csv")
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        fh = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=fh, stderr=subprocess.DEVNULL)
        return p, fh, path
    except Exception:
        return None, None, path


def clocks_stop(handle, gpu_index):
    p, fh, path = handle
    if p is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    p.terminate()
    p.wait()
    fh.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if f[5 + k].lower().startswith("active"):
                reasons.add(nm)
    os.unlink(path)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------- ours
ACE_GROUP = 0


def setup(torch, prm, s, lam_mode, precision="fp32"):
    from paper_2512_07693_gb300 import apip
    n = len(s["pos"])
    dev = torch.device("cuda")
    m = apip.Apip(prm, n, precision=precision, lam_mode=lam_mode, max_nb=80, cell_cap=48, ace_group=ACE_GROUP)
    t = dict(pos=torch.tensor(s["pos"], dtype=torch.float64, device=dev),
             vel=torch.tensor(s["vel"], dtype=torch.float64, device=dev),
             ids=torch.tensor(s["ids"], dtype=torch.int32, device=dev),
             types=torch.zeros(n, dtype=torch.int32, device=dev),
             inv_mass=torch.tensor(1.0 / (s["mass"] * apip.MVV2E), dtype=torch.float64, device=dev),
             F=torch.empty((n, 3), dtype=torch.float64, device=dev))
    box = [float(x) for x in s["box"]]
    if lam_mode == "paper":
        m.init_csp_pairs(t["pos"], box, t["ids"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"])
    m.sync()
    return m, t, box


def timed_steps(torch, m, t, box, steps, flush, thermo=None):
    """Per-step CUDA-event timing on the launching stream, L2 flushed between steps."""
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xff)
        starts[k].record(stream)
        m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], 0.001, 1,
                      None if thermo is None else thermo[k])
        ends[k].record(stream)
    torch.cuda.synchronize()
    m.sync()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def ace_flops_per_atom(s, nnb_rc, info):
    """Algorithmic float32 operations of the ACE kernel per compacted atom, a
    multiply-add counted as 2: per neighbour within r_c, A accumulation 2 n NLM and
    the force contraction (u, v) 4 n NLM + 8 NLM; plus the basis work forward and
    adjoint as the library counts it from its tables (apip_ace_info
    "table_flops").  Basis-function evaluation (R, Y) is not counted."""
    a = s["prm"]["ace"]
    nlm = (a["l_max"] + 1) ** 2
    per_nb = 2 * a["n_max"] * nlm + 4 * a["n_max"] * nlm + 8 * nlm
    return nnb_rc * per_nb + info["table_flops"], per_nb


def run_ours(args):
    import numpy as np
    import torch
    global ACE_GROUP
    ACE_GROUP = args.ace_group
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_2512_07693_gb300 import build
    build.build()
    from paper_2512_07693_gb300 import apip, workloads as W

    s = W.config(WORKLOAD, apip.apip_ace_basis_size, scale=args.cells)
    n = len(s["pos"])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    # --- adaptive run (the metric)
    m, t, box = setup(torch, s["prm"], s, "paper")
    timed_steps(torch, m, t, box, args.warmup, flush)
    thermo = torch.zeros((args.steps, 5), dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = clocks_start()
    per = timed_steps(torch, m, t, box, args.steps, flush, thermo)
    clocks = clocks_stop(clk, local)
    total_ms = job_ms(torch, sum(per), world, "cuda")
    value = job_value(world, n, args.steps, total_ms)
    th = thermo.cpu().numpy()
    H = (th[:, 0] + th[:, 1]) / n
    tps = np.arange(args.steps) * 0.001
    drift_timed = float(np.polyfit(tps, H, 1)[0]) if args.steps > 2 else None
    # energy drift: least-squares slope of H/N over a 10 ps NVE continuation (untimed;
    # 100 steps per call), after the timed steps let the start-up transient decay
    drift, drift_window = None, None
    if args.drift_steps >= 100:
        nd = args.drift_steps // 100 * 100
        thd = torch.zeros((nd, 5), dtype=torch.float64, device="cuda")
        for q in range(0, nd, 100):
            m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], 0.001, 100,
                          thd[q:q + 100])
        torch.cuda.synchronize()
        m.sync()
        hd = thd.cpu().numpy()
        Hd = (hd[:, 0] + hd[:, 1]) / n
        drift = float(np.polyfit(np.arange(nd) * 0.001, Hd, 1)[0])
        drift_window = {"ps": nd * 0.001, "start_ps": (args.warmup + args.steps) * 0.001,
                        "H_std_ev_per_atom": float(Hd.std()),
                        "momentum_change": [float(v) for v in hd[-1, 2:] - th[0, 2:]]}
    lam = m.field("lam", n).cpu().numpy()
    x_ace = float((lam > 0).mean())
    pmom = th[-1, 2:] - th[0, 2:]

    # --- per-phase device time (profiled pass, same workload)
    apip.apip_profile(m.ctx, 1)
    apip.apip_profile_read(m.ctx)
    prof_steps = min(args.steps, 50)
    timed_steps(torch, m, t, box, prof_steps, flush)
    prof = apip.apip_profile_read(m.ctx)
    apip.apip_profile(m.ctx, 0)
    launches_per_step = sum(v[1] for v in prof.values()) / prof_steps
    nnb = m.field("nnb", n).cpu().numpy()
    P = m.field("ace_list", n).cpu().numpy()[: int((lam > 0).sum())]
    ace_info = apip.apip_ace_info(m.ctx)
    # neighbours within the ACE cutoff of the compacted atoms (the per-pair work)
    nbl = m.field("nblist", n)[torch.as_tensor(P, device="cuda")].cpu().numpy()
    pos_now = t["pos"].cpu().numpy()
    jj = np.where(nbl >= 0, nbl, P[:, None])
    dv = pos_now[jj] - pos_now[P][:, None, :]
    dv -= np.asarray(box) * np.rint(dv / np.asarray(box))
    r2 = np.sum(dv * dv, axis=2)
    rc = s["prm"]["ace"]["rc"]
    nb_rc_ace = float(np.mean(np.sum((nbl >= 0) & (r2 < rc * rc) & (jj != P[:, None]), axis=1))) if len(P) else 0.0
    del m

    # --- all-ACE run on the same GPU (lam = 1 everywhere)
    ma, ta, boxa = setup(torch, s["prm"], s, "const1")
    timed_steps(torch, ma, ta, boxa, 1, flush)
    per_a = timed_steps(torch, ma, ta, boxa, args.ace_steps, flush)
    all_ace = n * args.ace_steps / (sum(per_a) * 1e-3)
    apip.apip_profile(ma.ctx, 1)
    timed_steps(torch, ma, ta, boxa, 2, flush)
    prof_a = apip.apip_profile_read(ma.ctx)
    del ma

    # --- end to end through the public API with host buffers
    me, te, boxe = setup(torch, s["prm"], s, "paper")
    h_pos = torch.tensor(s["pos"], dtype=torch.float64).pin_memory()
    h_vel = torch.tensor(s["vel"], dtype=torch.float64).pin_memory()
    h_th = torch.zeros(5, dtype=torch.float64).pin_memory()
    th_d = torch.zeros(5, dtype=torch.float64, device="cuda")
    e2e_steps = args.e2e_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        te["pos"].copy_(h_pos, non_blocking=True)
        te["vel"].copy_(h_vel, non_blocking=True)
        me.verlet_step(te["pos"], te["vel"], te["F"], te["inv_mass"], boxe, te["types"], te["ids"], 0.001, 1, th_d)
        h_pos.copy_(te["pos"], non_blocking=True)
        h_vel.copy_(te["vel"], non_blocking=True)
        h_th.copy_(th_d, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_dt = time.perf_counter() - t0
    me.sync()
    del me
    e2e = dict(value=world * n * e2e_steps / e2e_dt, unit="atom-steps/s", h2d_bytes_per_step=2 * 24 * n,
               d2h_bytes_per_step=2 * 24 * n + 40)

    # --- roofline of the dominant kernel
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM)
    dom = max((k for k in prof if k != "reduce"), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(1, prof[dom][1] if dom != "neighbor" else prof_steps)
    mean_nnb = float(nnb.mean())
    if dom in ("pass1", "pass2", "prep", "neighbor"):
        # algorithmic bytes per atom: neighbour indices 4 B each + nnb + own position
        # (hi/lo 32 B) + per-atom inputs/outputs (pass1: 8 partner ids 32 B + 4 outputs 16 B;
        # pass2: g, xi' 8 B + lam, dlam, wbar, d 16 B + force 24 B)
        extra = {"pass1": 32 + 16, "pass2": 8 + 16 + 24, "prep": 0, "neighbor": 0}[dom]
        per_atom = 4 * mean_nnb + 4 + 32 + extra
        if dom == "prep":
            per_atom = 2 * 48 + 24 + 24 + 32 + 8      # Verlet: pos, vel r/w, F, ref, hi/lo, inv_mass
        traffic_alg = per_atom * n
        achieved = traffic_alg / (dom_ms * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": NCU_TRAFFIC.get(dom) if args.cells is None else None,
                "algorithmic_bytes_per_launch": traffic_alg,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"}
    else:
        nb_rc = nb_rc_ace
        fl_atom, _ = ace_flops_per_atom(s, nb_rc, ace_info)
        fl = fl_atom * len(P)
        peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
        achieved = fl / (dom_ms * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dom) if args.cells is None else None,
                "traffic_unit": "DRAM bytes per launch (ncu)", "algorithmic_flops_per_launch": fl,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}

    out = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.cells is None else f"void recipe at {args.cells}^3 cells",
                   "atoms": n, "ace": "n_max 6, l_max 3, nu<=3", "x_ace": x_ace,
                   "precision": "fp32 pair arithmetic, fp64 positions/velocities/forces/reductions",
                   "l2": "flushed (512 MB write) between timed steps", "parallelism": "replicas" if world > 1 else "1 GPU"},
        "all_ace_atom_steps_per_s": all_ace * world,
        "speedup_vs_all_ace": value / (all_ace * world),
        "nve_drift_ev_per_atom_ps": drift,
        "nve_drift_window": drift_window,
        "nve_drift_timed_steps_ev_per_atom_ps": drift_timed,
        "momentum_change": [float(v) for v in pmom],
        "phase_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()},
        "phase_ms_per_step_all_ace": {k: v[0] / 2 for k, v in prof_a.items()},
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "ace_tables": ace_info,
    }
    if rank == 0 and not args.no_cpu_baseline:
        cb = oracle_sample(None, 15.0)
        out["cpu_baseline"] = {"value": cb["value"], "unit": "atom-steps/s", "cores": 1, "kind": "oracle",
                               "sample": f"{cb['reps']} FP64 numpy energy/force call(s) on the {WORKLOAD} recipe "
                                         f"at {cb['cells']}^3 cells ({cb['n']} atoms, x = {cb['x']:.3f}), "
                                         f"{cb['seconds']:.1f} s, single thread"}
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
