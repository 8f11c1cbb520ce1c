#!/usr/bin/env python
"""Throughput of the adaptive-precision (AP) EAM+ACE MD step on one GB300.

One "step" is one velocity-Verlet NVE step of the whole hot path (neighbour
check/rebuild, EAM pass, CSP^list g, switch, compaction, ACE forward+adjoint on
the compacted atoms, grad-lambda forces, float64 reductions, integrator) on the
void250k workload: a 50^3-cell bcc crystal with a central void of radius 15 A
(248 757 atoms, 300 K), ACE n_max 6 / l_max 3 / nu <= 3, float32 pair
arithmetic with float64 positions, velocities, forces and reductions.

Prints one JSON line (rank 0).  Metric: atom-steps/s of the adaptive run; the
all-ACE run on the same GPU, the NVE drift, the rooflines of the dominant kernel
and of the ACE kernel against measured peaks, and one line per other workload
(the 2 k-atom vacancy crystal in float64, the void crystal in float64, the 2 M-atom
cracked slab, learned-indicator training, the 4 M-atom indentation slab with the
paper's switch, the learned switch and all-ACE) are reported beside it.
``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): replicas only, one independent system per rank.
"""
import argparse
import json
import math
import multiprocessing
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
FALLBACK_BF16 = 1900.0


def measured_peaks():
    """The measured peaks of this machine's GPUs (empty if the file is absent)."""
    return json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
L2_FLUSH_BYTES = 512 << 20          # > 129 MB L2, written between timed steps
# DRAM bytes (read + write) per launch of the step's dominant kernel on this
# workload from an ncu capture, with the commit of the kernel's source it was
# taken at; reported beside the roofline while that kernel is unchanged
NCU_TRAFFIC_CURRENT = {"pass2": (69.683968e6 + 0.957696e6, "ncu capture of k_pass2 at commit 513b48c")}


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
    ap.add_argument("--no-extra", action="store_true", help="skip the lines of the other workloads")
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
def _oracle_system(cells):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import ace, csp
    from paper_2512_07693_gb300 import workloads as W
    s = W.config(WORKLOAD, lambda a, b, c: len(ace.enumerate_basis(a, b, c)), scale=cells)
    part = csp.init_pairs(s["pos"], s["box"], s["ids"], W.CSP["rcut"])
    return s, part, ace.AceModel(s["prm"]["ace"])


def _oracle_forces_worker(job):
    """One host process: repeated FP64 oracle energy/force calls on the shrunken
    recipe for about target_s seconds."""
    target_s, cells = job
    from oracle import apip as oapip
    s, part, model = _oracle_system(cells)
    t0 = time.perf_counter()
    reps = 0
    while True:
        res = oapip.energy_forces(s["pos"], s["box"], s["ids"], part, s["prm"], model=model)
        reps += 1
        if time.perf_counter() - t0 >= target_s:
            break
    return len(s["pos"]), reps, time.perf_counter() - t0, len(res["P"]) / len(s["pos"])


def _oracle_verlet_worker(job):
    """One host process: warm-up then timed FP64 oracle velocity-Verlet steps."""
    cells, warmup, steps = job
    from oracle import verlet
    s, part, model = _oracle_system(cells)
    pos, vel = s["pos"], s["vel"]
    pos, vel, _, _ = verlet.run(pos, vel, s["box"], s["ids"], part, s["prm"], s["mass"], 0.001, warmup, model=model)
    t0 = time.perf_counter()
    verlet.run(pos, vel, s["box"], s["ids"], part, s["prm"], s["mass"], 0.001, steps, model=model)
    return len(s["pos"]), steps, time.perf_counter() - t0


def host_workers():
    return max(1, os.cpu_count() or 1)


def _pool_map(fn, jobs):
    """Run the oracle in spawned processes (a fresh interpreter each: the parent's
    CUDA context is never forked), one numpy thread per process."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(len(jobs)) as pool:
        return pool.map(fn, jobs)


def oracle_sample(target_s, cells=12):
    """The FP64 CPU oracle on every host core: one independent copy of a shrunken
    void recipe (same lattice, void radius scaled with the box, same potentials)
    per core, timed together; atom-steps/s summed over the copies."""
    workers = host_workers()
    res = _pool_map(_oracle_forces_worker, [(target_s, cells)] * workers)
    value = sum(n * reps / dt for n, reps, dt, _ in res)
    n, reps, dt, x = res[0]
    return dict(value=value, n=n, reps=sum(r[1] for r in res), seconds=max(r[2] for r in res), x=x,
                cells=cells, workers=workers)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cells = 6
    workers = host_workers()
    t0 = time.perf_counter()
    res = _pool_map(_oracle_verlet_worker, [(cells, args.warmup, args.steps)] * workers)
    wall = time.perf_counter() - t0
    value = sum(n * steps / dt for n, steps, dt in res)
    n = res[0][0]
    sample = (f"{WORKLOAD} recipe at {cells}^3 cells ({n} atoms), FP64 numpy oracle, velocity-Verlet steps; "
              f"{workers} independent copies, one per host core, atom-steps/s summed")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * max(r[2] for r in res) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "atoms": n, "sample": sample, "wall_s": wall},
        "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": workers, "kind": "oracle", "sample": sample},
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


def device_arrays(torch, s):
    from paper_2512_07693_gb300 import apip
    n = len(s["pos"])
    dev = torch.device("cuda")
    return dict(pos=torch.tensor(s["pos"], dtype=torch.float64, device=dev),
                vel=torch.tensor(s["vel"], dtype=torch.float64, device=dev),
                ids=torch.tensor(s["ids"], dtype=torch.int32, device=dev),
                types=torch.zeros(n, dtype=torch.int32, device=dev),
                inv_mass=torch.tensor(1.0 / (s["mass"] * apip.MVV2E), dtype=torch.float64, device=dev),
                F=torch.empty((n, 3), dtype=torch.float64, device=dev))


def setup(torch, prm, s, lam_mode, precision="fp32"):
    from paper_2512_07693_gb300 import apip
    n = len(s["pos"])
    m = apip.Apip(prm, n, precision=precision, lam_mode=lam_mode, max_nb=80, cell_cap=48, ace_group=ACE_GROUP)
    t = device_arrays(torch, s)
    box = [float(x) for x in s["box"]]
    if lam_mode == "paper":
        m.init_csp_pairs(t["pos"], box, t["ids"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"])
    m.sync()
    return m, t, box


THERMO_EVERY = 10   # thermo output (E_pot, E_kin, momentum) every 10th step, as an MD log does


def timed_steps(torch, m, t, box, steps, flush, thermo=None):
    """Per-step CUDA-event timing on the launching stream, L2 flushed between steps.
    With ``thermo`` (rows of 5), step k writes row k // THERMO_EVERY when
    k % THERMO_EVERY == THERMO_EVERY - 1."""
    stream = torch.cuda.current_stream()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xff)
        log = thermo is not None and k % THERMO_EVERY == THERMO_EVERY - 1
        starts[k].record(stream)
        m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], 0.001, 1,
                      thermo[k // THERMO_EVERY] if log else None)
        ends[k].record(stream)
    torch.cuda.synchronize()
    m.sync()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def nve_drift(torch, m, t, box, n, steps, chunk=100):
    """Least-squares slope of H/N (eV/atom/ps) over ``steps`` NVE steps of 1 fs
    (untimed; thermo every step), and the momentum change over them."""
    import numpy as np
    nd = max(chunk, steps // chunk * chunk)
    thd = torch.zeros((nd, 5), dtype=torch.float64, device="cuda")
    for q in range(0, nd, chunk):
        m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], 0.001, chunk,
                      thd[q:q + chunk])
    torch.cuda.synchronize()
    m.sync()
    hd = thd.cpu().numpy()
    Hd = (hd[:, 0] + hd[:, 1]) / n
    return (float(np.polyfit(np.arange(nd) * 0.001, Hd, 1)[0]),
            {"ps": nd * 0.001, "H_std_ev_per_atom": float(Hd.std()),
             "momentum_change": [float(v) for v in hd[-1, 2:] - hd[0, 2:]]})


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


def neighbours_within(torch, m, t, box, atoms, rc, n):
    """Mean number of neighbours within rc of the given atoms (the ACE pair work)."""
    import numpy as np
    if len(atoms) == 0:
        return 0.0
    nbl = m.field("nblist", n)[torch.as_tensor(atoms, device="cuda")].cpu().numpy()
    pos_now = t["pos"].cpu().numpy()
    jj = np.where(nbl >= 0, nbl, atoms[:, None])
    dv = pos_now[jj] - pos_now[atoms][:, None, :]
    dv -= np.asarray(box) * np.rint(dv / np.asarray(box))
    r2 = np.sum(dv * dv, axis=2)
    return float(np.mean(np.sum((nbl >= 0) & (r2 < rc * rc) & (jj != atoms[:, None]), axis=1)))


def ace_roofline(s, nb_rc, info, atoms, ms, peak, source):
    fl_atom, _ = ace_flops_per_atom(s, nb_rc, info)
    fl = fl_atom * atoms
    achieved = fl / (ms * 1e-3) / 1e12 if ms > 0 else 0.0
    return {"kernel": "ace", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None, "traffic": None, "atoms": int(atoms),
            "algorithmic_flops_per_launch": fl, "flops_per_atom": fl_atom, "peak_source": source}


# ------------------------------------------------------- the other workloads
def extra_vacancy2k(torch, W, apip):
    """C1: 1 999 atoms, float64, one energy/force call and 100 Verlet steps."""
    s = W.config("vacancy2k", apip.apip_ace_basis_size)
    n = len(s["pos"])
    m, t, box = setup(torch, s["prm"], s, "paper", precision="fp64")
    stream = torch.cuda.current_stream()
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record(stream)
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"])
    b.record(stream)
    m.verlet_step(t["pos"], t["vel"], t["F"], t["inv_mass"], box, t["types"], t["ids"], 0.001, 100)
    c.record(stream)
    torch.cuda.synchronize()
    m.sync()
    x = float((m.field("lam", n).cpu().numpy() > 0).mean())
    m.close()
    ms_md = b.elapsed_time(c)
    return {"workload": "vacancy2k", "atoms": n, "precision": "fp64", "x_ace": x,
            "energy_forces_ms": a.elapsed_time(b), "md_100_steps_ms": ms_md,
            "atom_steps_per_s": n * 100 / (ms_md * 1e-3)}


def extra_void_fp64(torch, W, apip, flush, steps=10, drift_steps=1000):
    """C2 in float64: the same void crystal and step, every pair in float64."""
    s = W.config(WORKLOAD, apip.apip_ace_basis_size)
    n = len(s["pos"])
    m, t, box = setup(torch, s["prm"], s, "paper", precision="fp64")
    timed_steps(torch, m, t, box, 3, flush)
    per = timed_steps(torch, m, t, box, steps, flush)
    x = float((m.field("lam", n).cpu().numpy() > 0).mean())
    drift, window = nve_drift(torch, m, t, box, n, drift_steps)
    m.close()
    return {"workload": WORKLOAD, "atoms": n, "precision": "fp64", "steps": steps, "ms_per_step": sum(per) / steps,
            "atom_steps_per_s": n * steps / (sum(per) * 1e-3), "x_ace": x,
            "nve_drift_ev_per_atom_ps": drift, "nve_drift_window": window}


def extra_crack2m(torch, W, apip, flush, steps=3):
    """C3: the 2.0 M-atom cracked slab, ACE n_max 8 / l_max 4 / nu <= 4, float32."""
    s = W.config("crack2m", apip.apip_ace_basis_size)
    n = len(s["pos"])
    m = apip.Apip(s["prm"], n, precision="fp32", lam_mode="paper", max_nb=80, cell_cap=48)
    t = device_arrays(torch, s)
    box = [float(x) for x in s["box"]]
    lam_fixed = torch.tensor(s["lam_fixed"], dtype=torch.float64, device="cuda")
    m.set_lam_fixed(lam_fixed)
    m.init_csp_pairs(t["pos"], box, t["ids"])
    m.energy_forces(t["pos"], box, t["types"], t["ids"], t["F"])
    m.sync()
    timed_steps(torch, m, t, box, 1, flush)
    per = timed_steps(torch, m, t, box, steps, flush)
    x = float((m.field("lam", n).cpu().numpy() > 0).mean())
    info = apip.apip_ace_info(m.ctx)
    m.close()
    return {"workload": "crack2m", "atoms": n, "precision": "fp32", "ace": "n_max 8, l_max 4, nu<=4",
            "basis_functions": int(s["prm"]["ace"]["c1"].shape[0]), "steps": steps,
            "ms_per_step": sum(per) / steps, "atom_steps_per_s": n * steps / (sum(per) * 1e-3), "x_ace": x,
            "ace_group": info["group"]}


def extra_training(torch, W, apip, configs=4000, epochs=20, batch=65536):
    """C4 on a subsample: labels + descriptors of ``configs`` 2000-site defect
    crystals, then Adam epochs; returns the trained weights for the indentation line."""
    from paper_2512_07693_gb300 import train
    prm = W.config("vacancy2k", apip.apip_ace_basis_size)["prm"]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G, y, ref = train.make_dataset(prm, configs)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    params, hist = train.train(G, y, epochs=epochs, batch=min(batch, len(y)), lr=1e-3, prm=prm)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    na = int(len(y))
    del G, y
    # the training step alone (loss and gradient, then Adam), device-timed on a
    # synthetic batch of the same size: its roofline is the bf16 tensor pipe
    us, tf = train.step_time(batch, steps=50, warmup=5)
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops", FALLBACK_BF16)
    line = {"workload": f"learned-indicator training, {configs} of the 50 000 configurations", "atoms": na,
            "epochs": epochs, "label_and_descriptor_s": t1 - t0, "label_atoms_per_s": na / (t1 - t0),
            "training_s": t2 - t1, "training_atom_epochs_per_s": na * epochs / (t2 - t1),
            "loss_first_last": [hist[0], hist[-1]],
            "step": {"batch": batch, "us_per_step": us, "samples_per_s": batch / (us * 1e-6),
                     "flop_per_sample": train.FLOP_PER_SAMPLE,
                     "roofline": {"kernel": "k_train_tc (+ k_train_reduce, k_adam)", "bound": "tensor",
                                  "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                  "frac": tf / peak if peak else None, "traffic": None,
                                  "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured, burst)"
                                  if "bf16_tflops" in peaks else "fallback"}}}
    return line, params


def extra_indent4m(torch, W, apip, flush, params, steps=20, ace_steps=3):
    """C5: the 3 993 600-atom indentation slab, three arms on the same GPU: the
    paper's switch, the learned switch (window placed at the paper's x on the
    starting configuration, the rule of the full-size indentation run), all-ACE.
    The network here is trained on 4 000 of the 50 000 configurations; its x rises
    while the slab heats up from its start-up state (x_ace_start, x_ace at the end
    of the timed steps)."""
    import numpy as np
    from paper_2512_07693_gb300 import indent
    s = W.config("indent4m", apip.apip_ace_basis_size)
    n = len(s["pos"])
    arms = {}
    x_paper_start = None
    for arm in ("paper", "learned", "ace"):
        t = indent._device(torch, s)
        prm = s["prm"]
        if arm == "learned":
            free = ~np.isfinite(s["lam_fixed"])
            lo, hi = indent.learned_window(torch, s, t, params, x_paper_start * n / free.sum())
            prm = dict(s["prm"], switch=dict(s["prm"]["switch"], d_lo=lo, d_hi=hi))
        m, box = indent.model(torch, s, arm, t, prm=prm, mlp_flat=params)
        x_start = float((m.field("lam", n).cpu().numpy() > 0).mean())
        if arm == "paper":
            x_paper_start = x_start
        k = steps if arm != "ace" else ace_steps
        timed_steps(torch, m, t, box, 2, flush)
        per = timed_steps(torch, m, t, box, k, flush)
        lam = m.field("lam", n).cpu().numpy()
        x = float((lam > 0).mean())
        m.close()
        arms[arm] = {"steps": k, "ms_per_step": sum(per) / k, "atom_steps_per_s": n * k / (sum(per) * 1e-3),
                     "x_ace_start": x_start, "x_ace": x}
    for a in arms.values():
        a["speedup_vs_all_ace"] = a["atom_steps_per_s"] / arms["ace"]["atom_steps_per_s"]
    return {"workload": "indent4m", "atoms": n, "precision": "fp32", "arms": arms}


def run_extras(torch, W, apip, flush):
    """One line per other workload; a workload that fails records its error
    instead of ending the run."""
    out = {}

    def guarded(name, fn):
        try:
            r = fn()
        except Exception as e:    # recorded in the output line, not raised
            r = {"error": f"{type(e).__name__}: {e}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return r

    out["vacancy2k_fp64"] = guarded("vacancy2k", lambda: extra_vacancy2k(torch, W, apip))
    out["void250k_fp64"] = guarded("void250k_fp64", lambda: extra_void_fp64(torch, W, apip, flush))
    out["crack2m"] = guarded("crack2m", lambda: extra_crack2m(torch, W, apip, flush))
    params = {}

    def train_line():
        line, p = extra_training(torch, W, apip)
        params["p"] = p
        return line
    out["training"] = guarded("training", train_line)
    if "p" in params:
        out["indent4m"] = guarded("indent4m", lambda: extra_indent4m(torch, W, apip, flush, params["p"]))
    return out


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

    fp32_peak, fp64_peak = apip.apip_measure_peaks()
    s = W.config(WORKLOAD, apip.apip_ace_basis_size, scale=args.cells)
    n = len(s["pos"])
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    # --- adaptive run (the metric); the clock sampler runs from the set-up through
    # the timed steps, since the timed region alone is shorter than its period
    clk = clocks_start()
    m, t, box = setup(torch, s["prm"], s, "paper")
    timed_steps(torch, m, t, box, args.warmup, flush)
    n_log = args.steps // THERMO_EVERY
    thermo = torch.zeros((max(1, n_log), 5), dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    per = timed_steps(torch, m, t, box, args.steps, flush, thermo)
    clocks = clocks_stop(clk, local)
    total_ms = job_ms(torch, sum(per), world, "cuda")
    value = job_value(world, n, args.steps, total_ms)
    th = thermo.cpu().numpy()[:n_log]
    H = (th[:, 0] + th[:, 1]) / n
    tps = (np.arange(n_log) + 1) * THERMO_EVERY * 0.001
    drift_timed = float(np.polyfit(tps, H, 1)[0]) if n_log > 2 else None
    pmom = th[-1, 2:] - th[0, 2:] if n_log > 1 else np.zeros(3)
    # energy drift: least-squares slope of H/N over a 10 ps NVE continuation (untimed),
    # after the timed steps let the start-up transient decay
    drift, drift_window = None, None
    if args.drift_steps >= 100:
        drift, drift_window = nve_drift(torch, m, t, box, n, args.drift_steps)
        drift_window["start_ps"] = (args.warmup + args.steps) * 0.001
    lam = m.field("lam", n).cpu().numpy()
    x_ace = float((lam > 0).mean())

    # --- per-phase device time (profiled pass, same workload)
    apip.apip_profile(m.ctx, 1)
    apip.apip_profile_read(m.ctx)
    prof_steps = min(args.steps, 50)
    timed_steps(torch, m, t, box, prof_steps, flush)
    prof = apip.apip_profile_read(m.ctx)
    apip.apip_profile(m.ctx, 0)
    launches_per_step = sum(v[1] for v in prof.values()) / prof_steps
    nnb = m.field("nnb", n).cpu().numpy()
    lam = m.field("lam", n).cpu().numpy()
    P = m.field("ace_list", n).cpu().numpy()[: int((lam > 0).sum())]
    ace_info = apip.apip_ace_info(m.ctx)
    rc = s["prm"]["ace"]["rc"]
    nb_rc_ace = neighbours_within(torch, m, t, box, P, rc, n)
    m.close()

    # --- all-ACE run on the same GPU (lam = 1 everywhere)
    ma, ta, boxa = setup(torch, s["prm"], s, "const1")
    timed_steps(torch, ma, ta, boxa, 1, flush)
    per_a = timed_steps(torch, ma, ta, boxa, args.ace_steps, flush)
    all_ace = n * args.ace_steps / (sum(per_a) * 1e-3)
    apip.apip_profile(ma.ctx, 1)
    timed_steps(torch, ma, ta, boxa, 2, flush)
    prof_a = apip.apip_profile_read(ma.ctx)
    nb_rc_all = neighbours_within(torch, ma, ta, boxa, np.arange(0, n, 97), rc, n)
    ace_info_a = apip.apip_ace_info(ma.ctx)
    ma.close()

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
    me.close()
    e2e = dict(value=world * n * e2e_steps / e2e_dt, unit="atom-steps/s", h2d_bytes_per_step=2 * 24 * n,
               d2h_bytes_per_step=2 * 24 * n + 40)

    # --- rooflines: the dominant kernel of the step, and the ACE kernel (adaptive
    # and all-ACE) against the measured float32 multiply-add peak
    peaks = json.load(open(PEAKS)) if os.path.exists(PEAKS) else {}
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM)
    peak_src = "apip_measure_peaks: float32 multiply-add loop on every SM (measured in this run)"
    dom = max((k for k in prof if k != "reduce"), key=lambda k: prof[k][0])
    dom_ms = prof[dom][0] / max(1, prof[dom][1] if dom != "neighbor" else prof_steps)
    ace_ms = prof["ace"][0] / max(1, prof["ace"][1])
    ace_ms_a = prof_a["ace"][0] / max(1, prof_a["ace"][1])
    roof_ace = ace_roofline(s, nb_rc_ace, ace_info, len(P), ace_ms, fp32_peak, peak_src)
    roof_ace_all = ace_roofline(s, nb_rc_all, ace_info_a, n, ace_ms_a, fp32_peak, peak_src)
    if dom in ("pass1", "pass2", "prep", "neighbor"):
        # algorithmic bytes per atom: neighbour indices 4 B each + nnb + own position
        # (hi/lo 32 B) + per-atom inputs/outputs (pass1: 8 partner ids 32 B + 4 outputs 16 B;
        # pass2: g, xi' 8 B + lam, dlam, wbar, d 16 B + force 24 B)
        extra = {"pass1": 32 + 16, "pass2": 8 + 16 + 24, "prep": 0, "neighbor": 0}[dom]
        per_atom = 4 * float(nnb.mean()) + 4 + 32 + extra
        if dom == "prep":
            per_atom = 2 * 48 + 24 + 24 + 32 + 8      # Verlet: pos, vel r/w, F, ref, hi/lo, inv_mass
        traffic_alg = per_atom * n
        achieved = traffic_alg / (dom_ms * 1e-3) / 1e9
        cap = NCU_TRAFFIC_CURRENT.get(dom) if args.cells is None else None
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": cap[0] if cap else None,
                "traffic_source": cap[1] if cap else "no ncu capture of the current kernel",
                "algorithmic_bytes_per_launch": traffic_alg,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if peaks else "fallback"}
    else:
        roof = dict(roof_ace)

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
        "roofline_ace": {"adaptive": roof_ace, "all_ace": roof_ace_all},
        "peaks_measured": {"fp32_tflops": fp32_peak, "fp64_tflops": fp64_peak, "hbm_gbs": hbm},
        "clocks": clocks,
        "thermo_every": THERMO_EVERY,
        "e2e": e2e,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "ace_tables": ace_info,
    }
    if rank == 0 and not args.no_extra and args.cells is None:
        out["workloads"] = run_extras(torch, W, apip, flush)
    if rank == 0 and not args.no_cpu_baseline:
        cb = oracle_sample(12.0)
        out["cpu_baseline"] = {"value": cb["value"], "unit": "atom-steps/s", "cores": cb["workers"], "kind": "oracle",
                               "sample": f"{cb['reps']} FP64 numpy energy/force calls on the {WORKLOAD} recipe at "
                                         f"{cb['cells']}^3 cells ({cb['n']} atoms, x = {cb['x']:.3f}) in "
                                         f"{cb['workers']} independent processes, one per host core, "
                                         f"{cb['seconds']:.1f} s; atom-steps/s summed"}
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
