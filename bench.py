"""Throughput benchmark of the GB300 PIC step.

Workload (default): the large uniform thermal plasma, 2048 x 2048 cells,
dx = dy = 0.1, dt = 0.07, periodic, electrons + positrons at 8x8 particles
per cell each (536,870,912 particles), u_th = 0.1, FP32 (--precision fp64
for the all-FP64 form).  One step = push+deposit, Yee, tile migration and
end-of-step bookkeeping for every particle and cell.

Printed (rank 0, one JSON line): particle-steps/s of the whole job (inputs
resident in HBM, CUDA events on the library's stream), the e2e figure
through the C ABI with host buffers (particles uploaded from pinned host
memory, stepped, energies and particles read back, all inside the timed
region), the roofline of the dominant kernel (push_deposit) against the
measured HBM copy bandwidth, and the FP64 CPU oracle timed on a bounded
sample on this host as a baseline.

--impl reference times the oracle itself as the reference arm.
Multi-GPU (torchrun): every rank advances its own independent replica
(different generator stream); value = all ranks' particle-steps / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.txt")
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--ppc", type=int, default=8, help="particles per cell "
                    "per side and species")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the FP64 form, the batched-vs-per-sim "
                    "comparison and the precision errors against the oracle")
    ap.add_argument("--cpu-sample", type=int, default=512,
                    help="cells per side of the oracle sample")
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "clouds", "lwfa", "lwfa_paper",
                             "weibel", "batch", "precision", "tiles"],
                    help="uniform (default): the large uniform plasma; the "
                    "others print one line for that workload")
    return ap.parse_args()


# --------------------------------------------------------------- dist ----

def dist_init(n):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def all_max(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def all_sum(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(local_units, local_ms, world):
    """Whole-job rate of N ranks: the units all ranks processed over the
    slowest rank's time.  Returns (value per second, max ms, total units)."""
    ms_max = all_max(local_ms, world)
    total = all_sum(float(local_units), world)
    return total / (ms_max / 1e3), ms_max, total


# ------------------------------------------------------------- clocks ----

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                mhz.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not mhz:
            return None
        return {"sm_mhz": float(np.median(mhz)), "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# ------------------------------------------------------------ helpers ----

def hbm_peak():
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def push_kernel_hash():
    src = os.path.join(ROOT, "paper_2106_12485_gb300", "csrc", "k_push.cu")
    with open(src, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def measured_traffic(precision, n_particles, n_cells):
    """DRAM bytes per push_deposit launch from the committed ncu summary,
    scaled to this launch by particles (null if the kernel changed)."""
    try:
        with open(TRAFFIC_PATH) as f:
            for ln in f:
                if not ln.startswith("push_deposit "):
                    continue
                kv = dict(t.split("=", 1) for t in ln.split()[1:])
                if kv.get("sha") != push_kernel_hash():
                    return None
                if kv.get("precision") != precision:
                    continue
                bpp = float(kv["dram_bytes_per_particle"])
                return bpp * n_particles
    except Exception:
        return None
    return None


def algorithmic_bytes(n_particles, n_cells, real_bytes):
    # one read + one write of the SoA record (16-bit cell within the tile +
    # x, y, ux, uy, uz) per particle, plus E, B read and J written once per
    # cell
    rec = 2 + 5 * real_bytes
    return 2 * rec * n_particles + (6 + 3) * real_bytes * n_cells


# ---------------------------------------------------------- CPU oracle ----

def oracle_sample(cells, ppc, steps, nthreads, keep=False):
    """Times the FP64 oracle on a cells x cells periodic box of the same
    plasma (both species, same ppc and u_th).  Returns (ps/s, n_particles,
    seconds), and with keep=True also the oracle (advanced `steps` steps
    from step 0; an untimed warm-up runs on a copy) and its loads."""
    from oracle import oracle as O
    from synthetic import plasma as P

    def make():
        lds, sps = [], []
        for s, qm in enumerate((-1.0, 1.0)):
            ld = P.plasma_load(cells, cells, ppc, ppc, species=s,
                               u_th=(0.1, 0.1, 0.1), dtype=np.float32)
            lds.append(ld)
            f = {k: np.asarray(ld[k], np.float64)
                 for k in ("x", "y", "ux", "uy", "uz", "w")}
            sps.append(O.Species(qm, (1 if qm > 0 else -1) / ppc ** 2,
                                 ld["ix"], ld["iy"], f["x"], f["y"], f["ux"],
                                 f["uy"], f["uz"], w=f["w"], ids=ld["id"]))
        return O.Sim(cells, cells, 0.1, 0.1, 0.07, species=sps), lds, \
            sum(s.n for s in sps)

    sim, lds, n = make()
    if keep:
        warm, _, _ = make()
        warm.step(1, nthreads=nthreads)   # warm-up (page faults, threads)
        del warm
    else:
        sim.step(1, nthreads=nthreads)
    t0 = time.perf_counter()
    sim.step(steps, nthreads=nthreads)
    dt = time.perf_counter() - t0
    if keep:
        return n * steps / dt, n, dt, sim, lds
    return n * steps / dt, n, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return
    nthreads = os.cpu_count() or 1
    cells = args.cpu_sample // 2
    from oracle import oracle as O
    from synthetic import plasma as P
    sps = []
    for s, qm in enumerate((-1.0, 1.0)):
        ld = P.plasma_load(cells, cells, args.ppc, args.ppc, species=s,
                           u_th=(0.1, 0.1, 0.1), dtype=np.float64)
        sps.append(O.Species(qm, (1 if qm > 0 else -1) / args.ppc ** 2,
                             ld["ix"], ld["iy"], ld["x"], ld["y"], ld["ux"],
                             ld["uy"], ld["uz"], w=ld["w"], ids=ld["id"]))
    sim = O.Sim(cells, cells, 0.1, 0.1, 0.07, species=sps)
    n = sum(s.n for s in sps)
    for _ in range(args.warmup):
        sim.step(1, nthreads=nthreads)
    t0 = time.perf_counter()
    sim.step(args.steps, nthreads=nthreads)
    dt = time.perf_counter() - t0
    v = n * args.steps / dt
    sample = ("%dx%d periodic box of the same plasma (%d particles), %d "
              "oracle steps" % (cells, cells, n, args.steps))
    # the config is the box the oracle ran: a sample of the GPU workload
    # (same plasma, cell size, time step and particles per cell), not the
    # full grid
    config = sampled_config(args, cells, n)
    print(json.dumps({
        "impl": "reference", "metric": "particle-steps/s", "value": v,
        "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": v, "unit": "particle-steps/s",
                         "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "particle-steps/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def workload_config(args):
    ppc = args.ppc
    return {"workload": "uniform thermal plasma %dx%d, e-/e+ %dx%d ppc each, "
                        "u_th 0.1, dx=dy=0.1, dt=0.07, periodic" %
                        (args.nx, args.ny, ppc, ppc),
            "nx": args.nx, "ny": args.ny, "species": 2,
            "ppc_per_species": ppc * ppc,
            "particles": 2 * args.nx * args.ny * ppc * ppc,
            "precision": args.precision,
            "l2": "inputs larger than L2 (particle store >> 129 MB)"}


def sampled_config(args, cells, n):
    """Config of a timed sample of the workload: a cells x cells periodic
    box of the same plasma."""
    full = workload_config(args)
    return {"workload": "uniform thermal plasma %dx%d, e-/e+ %dx%d ppc "
                        "each, u_th 0.1, dx=dy=0.1, dt=0.07, periodic "
                        "(sample of the %dx%d workload)" %
                        (cells, cells, args.ppc, args.ppc, args.nx, args.ny),
            "nx": cells, "ny": cells, "species": 2,
            "ppc_per_species": args.ppc * args.ppc, "particles": int(n),
            "precision": "fp64", "sampled": True,
            "sampled_from": full["workload"]}


# ------------------------------------------------- secondary figures ----

def fp32_over_fp64(args, stream, torch, fp32_value, steps=5):
    """The all-FP64 GPU form on the same workload and time step: its
    particle-steps/s over `steps` CUDA-event-timed steps (after 2 warm-up
    steps) and the ratio FP32 / FP64.  Both forms share dt, so their
    energy-conservation error is the scheme's (equal drift, measured by
    --workload precision)."""
    from paper_2106_12485_gb300 import workloads as W
    from paper_2106_12485_gb300 import zpic as Z
    cfg = W.precision_study(args.nx, args.ny, ppc=(args.ppc, args.ppc),
                            precision=Z.FP64, energy_every=1)
    sim = Z.Sim(cfg)
    sim.set_stream(stream.cuda_stream)
    inf = sim.info()
    n = int(sum(inf.n_particles[:2]))
    sim.step(2)
    sim.sync()
    ms = timed_steps(sim, stream, steps, torch)
    e = sim.energy()
    tot = [r[1] + r[2] + sum(r[3]) for r in e]
    drift = max(abs(t - tot[0]) for t in tot) / tot[0]
    del sim
    v64 = n * steps / (ms / 1e3)
    # the same with the fixed-point (bitwise reproducible) FP64 current
    cfg_d = W.precision_study(args.nx, args.ny, ppc=(args.ppc, args.ppc),
                              precision=Z.FP64, deterministic=True)
    sim = Z.Sim(cfg_d)
    sim.set_stream(stream.cuda_stream)
    sim.step(2)
    sim.sync()
    ms_d = timed_steps(sim, stream, steps, torch)
    del sim
    return {"fp64_value": v64, "fp64_ms_per_step": ms / steps,
            "fp64_steps": steps, "fp64_energy_drift": drift,
            "fp64_deterministic_value": n * steps / (ms_d / 1e3),
            "ratio": fp32_value / v64}


def tune_batch_and_sims(cfgs, Z, steps=10):
    """The autotuner's settings for both forms of a sweep: the batch as a
    whole (zpic_batch_autotune; Batch(cfgs) then uses them) and each
    simulation's class for the per-simulation launches (zpic_autotune; Sim
    uses its tile).  Returns a summary of the choices."""
    out = {}
    if len(cfgs) >= 2:
        t, _ = Z.batch_autotune(cfgs, steps=steps)
        out["batch"] = {"tile": [t.tile_x, t.tile_y],
                        "ctas_per_sm": t.push_ctas_per_sm,
                        "sort_every": t.sort_every}
    tiles = {}
    for c in cfgs:
        tx, ty, _ = Z.autotune(c, steps=4)
        key = "%dx%d" % (tx, ty)
        tiles[key] = tiles.get(key, 0) + 1
    out["per_sim_tiles"] = tiles
    return out


def batched_over_per_sim(args, stream, torch, steps=10):
    """The batched sweep (256 independent simulations, one persistent
    launch per stage, captured in a CUDA graph) against the same simulations
    stepped one by one: aggregate particle-steps/s of both and the ratio."""
    from paper_2106_12485_gb300 import workloads as W
    from paper_2106_12485_gb300 import zpic as Z
    from synthetic import plasma as P
    cfgs = W.batch_sweep(P.batch_specs(256))
    tuning = tune_batch_and_sims(cfgs, Z, steps)
    batch = Z.Batch(cfgs)
    batch.set_stream(stream.cuda_stream)
    batch.step(3)
    batch.sync()
    n = 0
    for i in range(len(cfgs)):
        inf = batch.sim(i).info()
        n += sum(inf.n_particles[:inf.n_species])
    ms_b = timed_steps(batch, stream, steps, torch)
    del batch
    sims = [Z.Sim(c) for c in cfgs]
    for sm in sims:
        sm.set_stream(stream.cuda_stream)
        sm.step(3)
    for sm in sims:
        sm.sync()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for sm in sims:
            sm.step(1)
    for sm in sims:
        sm.sync()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    del sims
    return {"sims": len(cfgs), "particles": int(n), "steps": steps,
            "batched_value": n * steps / (ms_b / 1e3),
            "per_sim_value": n * steps / (ms_s / 1e3),
            "ratio": ms_s / ms_b, "tuning": tuning}


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def precision_vs_oracle(orc, loads, cells, steps, stream):
    """Error of the FP32 and the all-FP64 GPU forms against the FP64 oracle
    `orc` (already advanced `steps` steps from `loads`, a cells x cells box
    of the workload's plasma): relative L2 of each field, of the particle
    displacements and momenta (particles paired by id), and of the total
    energy at every step."""
    from paper_2106_12485_gb300 import zpic as Z
    FIELDS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")
    x0 = []
    for ld in loads:
        o = np.argsort(ld["id"], kind="stable")
        x0.append((ld["ix"][o] + ld["x"][o].astype(np.float64),
                   ld["iy"][o] + ld["y"][o].astype(np.float64)))
    tot_o = np.array([h[1] + h[2] + float(np.sum(h[3])) for h in orc.history])
    out = {}
    for name, prec, dt in (("fp32", Z.FP32, np.float32),
                           ("fp64", Z.FP64, np.float64)):
        ppc = int(round(np.sqrt(len(loads[0]["ix"]) / cells ** 2)))
        sps = [Z.species(qm, (ppc, ppc), profile=Z.PROFILE_NONE)
               for qm in (-1.0, 1.0)]
        cfg = Z.config(cells, cells, (cells * 0.1, cells * 0.1), 0.07, sps,
                       precision=prec, track_ids=True, energy_every=1)
        sim = Z.Sim(cfg)
        sim.set_stream(stream.cuda_stream)
        for s, ld in enumerate(loads):
            sim.set_particles(s, {k: (v.astype(dt) if v.dtype.kind == "f"
                                      else v) for k, v in ld.items()})
        sim.step(steps)
        f = {k: rel_l2(sim.field(k), orc.f[k]) for k in FIELDS}
        pos, mom = 0.0, 0.0
        for s in range(2):
            st = sim.particles(s)
            og = np.argsort(st["id"], kind="stable")
            ost = orc.species[s].state()
            oo = np.argsort(ost["id"], kind="stable")
            if not np.array_equal(st["id"][og], ost["id"][oo]):
                pos = mom = float("inf")
                break
            rx, ry = x0[s]
            gx = st["ix"][og] + st["x"][og].astype(np.float64)
            gy = st["iy"][og] + st["y"][og].astype(np.float64)
            ox = ost["ix"][oo] + ost["x"][oo]
            oy = ost["iy"][oo] + ost["y"][oo]
            wrap = lambda d: (d + cells / 2) % cells - cells / 2  # noqa: E731
            num = np.hypot(wrap(gx - ox), wrap(gy - oy))
            den = np.hypot(wrap(ox - rx), wrap(oy - ry))
            pos = max(pos, float(np.linalg.norm(num) / np.linalg.norm(den)))
            gu = np.stack([st[k][og] for k in ("ux", "uy", "uz")])
            ou = np.stack([ost[k][oo] for k in ("ux", "uy", "uz")])
            mom = max(mom, rel_l2(gu, ou))
        e = sim.energy()
        tot_g = np.array([r[1] + r[2] + sum(r[3]) for r in e])
        del sim
        out[name] = {"fields_rel_l2_max": max(f.values()),
                     "fields_rel_l2": f,
                     "displacement_rel_l2": pos, "momentum_rel_l2": mom,
                     "total_energy_rel_err_max":
                         float(np.max(np.abs(tot_g - tot_o) / tot_o)),
                     "energy_drift": float(np.max(np.abs(tot_g - tot_g[0]))
                                           / tot_g[0])}
    out["oracle_energy_drift"] = float(np.max(np.abs(tot_o - tot_o[0]))
                                       / tot_o[0])
    out["steps"] = steps
    out["box"] = "%dx%d periodic, same plasma as the workload" % (cells,
                                                                  cells)
    return out


# --------------------------------------------------------------- main ----

def timed_steps(sim, stream, steps, torch):
    """CUDA-event time (ms) of `steps` steps, any re-sort included."""
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    sim.sync()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def stage_split(sim, steps):
    """CUDA-event time per stage and step over `steps` further steps run
    with per-stage events (outside the timed region)."""
    sim.profile_enable(True)
    sim.profile_read(reset=True)
    sim.step(steps)
    sim.sync()
    prof = sim.profile_read(reset=True)
    sim.profile_enable(False)
    return {k: v[0] / max(v[1], 1) for k, v in prof.items()}


def base_line(metric_value, ms, args, dtype, config, **extra):
    out = {"metric": "particle-steps/s", "value": metric_value,
           "unit": "particle-steps/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype, "data": "synthetic", "config": config}
    out.update(extra)
    return out


def batch_workload(args, rank, world):
    """The batched sweep (256 independent simulations).  With N ranks the
    simulations are split by longest-processing-time-first on their
    algorithmic bytes per step (every rank computes the same partition, so
    nothing is exchanged on the data path); each rank advances its share as
    one batch (one persistent launch per kernel and step, captured in a CUDA
    graph), then as per-simulation launches for comparison.  The line gives
    the whole job: particles of all ranks x steps / the slowest rank's
    time."""
    import torch
    from paper_2106_12485_gb300 import workloads as W
    from paper_2106_12485_gb300 import zpic as Z
    from synthetic import plasma as P

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    stream = torch.cuda.Stream()
    specs = P.batch_specs(256)
    parts = W.lpt_partition(W.batch_costs(specs), world)
    mine = set(parts[rank])
    cfgs = [c for i, c in enumerate(W.batch_sweep(specs)) if i in mine]
    tuning = tune_batch_and_sims(cfgs, Z)
    batch = Z.Batch(cfgs)
    batch.set_stream(stream.cuda_stream)
    batch.step(args.warmup)
    batch.sync()
    n = 0
    for i in range(len(cfgs)):
        inf = batch.sim(i).info()
        n += sum(inf.n_particles[:inf.n_species])
    barrier(world)
    ms_b = timed_steps(batch, stream, args.steps, torch)
    split = stage_split(batch, args.steps)
    del batch
    sims = [Z.Sim(c) for c in cfgs]
    for sm in sims:
        sm.set_stream(stream.cuda_stream)
        sm.step(args.warmup)
    for sm in sims:
        sm.sync()
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        for sm in sims:
            sm.step(1)
    for sm in sims:
        sm.sync()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    value, ms_b_max, total = aggregate(float(n) * args.steps, ms_b, world)
    value_s, ms_s_max, _ = aggregate(float(n) * args.steps, ms_s, world)
    if rank == 0:
        print(json.dumps(base_line(
            value, ms_b_max, args, "f32",
            {"workload": "batched sweep: 256 independent sims 32-256 cells "
                         "per side, 4-64 ppc, half thermal, half clouds",
             "sims": len(specs), "particles": int(all_sum(float(n), world)),
             "sharding": "LPT over %d ranks on bytes per step" % world},
            n_gpus=world, scaling="strong",
            per_sim_launches={"value": value_s,
                              "ms_per_step": ms_s_max / args.steps},
            batched_over_per_sim=ms_s_max / ms_b_max,
            kernels_ms_next_steps=split, tuning=tuning)))
    else:
        all_sum(float(n), world)


def other_workload(args):
    """Lines for the workloads other than the large uniform plasma."""
    import torch
    from paper_2106_12485_gb300 import workloads as W
    from paper_2106_12485_gb300 import zpic as Z
    from synthetic import plasma as P

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    if args.workload in ("clouds", "lwfa", "lwfa_paper", "weibel"):
        if args.workload == "clouds":
            cfg = W.clouds(energy_every=10)
            warm = args.warmup
            desc = ("collision of plasma clouds 1024x1024, e-/e+ 4x4 ppc in "
                    "two clouds drifting +-0.2, u_th 0.05, FP32")
        elif args.workload == "lwfa_paper":
            cfg = W.lwfa_paper(energy_every=10)
            warm = max(args.warmup, 2000)   # let the plasma fill the window
            desc = ("laser wakefield, the paper's form: 2000x512, 16 ppc "
                    "(4x4 lattice) behind a ramp, compensated binomial "
                    "current filter, moving window, FP32")
        elif args.workload == "weibel":
            cfg = W.weibel(energy_every=10)
            warm = args.warmup
            desc = ("Weibel: e-/e+ 16x16 ppc each over 512x512 cells, "
                    "counter-drifting +-0.6 along z, u_th 0.1, FP32")
        else:
            cfg = W.lwfa(energy_every=10)
            warm = max(args.warmup, 2000)   # let the plasma fill the window
            desc = ("laser wakefield 4096x512, a0=2 w0=10 laser, moving "
                    "window, cold e- 2x2 ppc behind a ramp, FP32")
        sim = Z.Sim(cfg)
        sim.set_stream(stream.cuda_stream)
        sim.step(warm)
        sim.sync()
        info = sim.info()
        n0 = sum(info.n_particles[:info.n_species])
        r0 = info.resorts
        ms = timed_steps(sim, stream, args.steps, torch)
        info = sim.info()
        n1 = sum(info.n_particles[:info.n_species])
        r1 = info.resorts
        ps = 0.5 * (n0 + n1) * args.steps
        print(json.dumps(base_line(
            ps / (ms / 1e3), ms, args, "f32",
            {"workload": desc, "nx": cfg.nx, "ny": cfg.ny,
             "particles_start": int(n0), "particles_end": int(n1),
             "steps_before_timing": warm},
            resorts_in_timed_region=r1 - r0,
            step_after=int(info.step),
            kernels_ms_next_steps=stage_split(sim, args.steps))))
        return
    if args.workload == "tiles":
        # the autotuner for the workload classes (each on its copy reduced
        # to at most 1024 x 1024 cells): tile size, then resident push CTAs
        # per SM, then the cell-order re-sort interval
        out = {}
        for name, cfg in (("uniform_2048", W.precision_study()),
                          ("clouds_1024", W.clouds()),
                          ("lwfa_4096x512", W.lwfa()),
                          ("weibel_512", W.weibel())):
            t, times = Z.autotune_all(cfg, steps=args.steps)
            stages = {}
            for stage, cand, ms in times:
                key = "%dx%d" % cand if stage == "tile" else str(cand)
                stages.setdefault(stage, {})[key] = round(ms, 4)
            out[name] = {"best": {"tile": [t.tile_x, t.tile_y],
                                  "ctas_per_sm": t.push_ctas_per_sm,
                                  "sort_every": t.sort_every,
                                  "ms_per_step": round(t.ms_per_step, 4)},
                         "ms_per_step": stages}
        print(json.dumps({"workload": "autotuner: tile size, CTAs per SM, "
                          "re-sort interval", "steps": args.steps,
                          "classes": out}))
        return
    if args.workload == "precision":
        # FP32 vs FP64 at equal energy-conservation error: for each form the
        # largest dt of the sweep whose total-energy drift over 100 steps
        # stays within DRIFT_MAX, compared in simulated time per second
        DRIFT_MAX, NSTEPS = 1e-3, 100
        res = {}
        for name, prec in (("fp32", Z.FP32), ("fp64", Z.FP64)):
            runs = []
            for dt in (0.07, 0.05, 0.035):
                cfg = W.precision_study(args.nx, args.ny,
                                        ppc=(args.ppc, args.ppc), dt=dt,
                                        precision=prec, energy_every=1)
                sim = Z.Sim(cfg)
                sim.set_stream(stream.cuda_stream)
                inf = sim.info()
                n = sum(inf.n_particles[:2])
                sim.step(args.warmup)
                ms = timed_steps(sim, stream, NSTEPS, torch)
                e = sim.energy()
                tot = [r[1] + r[2] + sum(r[3]) for r in e]
                drift = max(abs(t - tot[0]) for t in tot) / tot[0]
                runs.append({"dt": dt, "ms_per_step": ms / NSTEPS,
                             "particle_steps_per_s": n * NSTEPS / (ms / 1e3),
                             "energy_drift": drift,
                             "steps": NSTEPS + args.warmup})
                del sim
            ok = [r for r in runs if r["energy_drift"] <= DRIFT_MAX]
            best = max(ok, key=lambda r: r["dt"]) if ok else None
            res[name] = {"runs": runs,
                         "dt_at_drift_max": best["dt"] if best else None,
                         "simulated_time_per_s":
                             best["dt"] / (best["ms_per_step"] / 1e3)
                             if best else None}
        a, b = (res["fp32"]["simulated_time_per_s"],
                res["fp64"]["simulated_time_per_s"])
        head = res["fp32"]["runs"][0]
        print(json.dumps(base_line(
            head["particle_steps_per_s"], head["ms_per_step"] * NSTEPS,
            args, "f32",
            {"workload": "precision study, uniform plasma %dx%d, e-/e+ %dx%d "
                         "ppc, u_th 0.1, dt 0.07/0.05/0.035, %d steps each"
                         % (args.nx, args.ny, args.ppc, args.ppc, NSTEPS),
             "energy_drift_max": DRIFT_MAX},
            fp32=res["fp32"], fp64=res["fp64"],
            fp32_over_fp64_at_equal_drift=(a / b) if a and b else None)))
        return


def main():
    args = parse_args()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "batch":
        batch_workload(args, rank, world)
        return
    if args.workload != "uniform":
        if rank == 0:
            other_workload(args)
        return
    import torch
    from paper_2106_12485_gb300 import workloads as W
    from paper_2106_12485_gb300 import zpic as Z

    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    prec = Z.FP64 if args.precision == "fp64" else Z.FP32
    rb = 8 if prec == Z.FP64 else 4
    cfg = W.precision_study(args.nx, args.ny, ppc=(args.ppc, args.ppc),
                            precision=prec, energy_every=1,
                            tile=(args.tile, args.tile), sim_index=rank)
    stream = torch.cuda.Stream()
    sim = Z.Sim(cfg)
    sim.set_stream(stream.cuda_stream)
    info = sim.info()
    n_p = int(sum(info.n_particles[:2]))
    n_cells = args.nx * args.ny

    # warm-up (untimed)
    sim.step(args.warmup)
    sim.sync()

    # ---- device-resident timed region --------------------------------
    sim.profile_enable(True)
    sim.profile_read(reset=True)
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    resorts0 = sim.info().resorts
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    sim.sync()          # a capacity re-sort, if any, is inside the region
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    resorts_timed = sim.info().resorts - resorts0
    prof = sim.profile_read(reset=True)
    sim.profile_enable(False)
    value, ms_max, total_ps = aggregate(float(n_p) * args.steps, ms, world)
    # kernels per profiled stage: the migration stage launches the scatter
    # of the outboxes and the fold of the arrival counts
    per_stage = {"migrate": 2}
    launches = sum(v[1] * per_stage.get(k, 1) for k, v in prof.items())

    push_ms, push_n = prof.get("push_deposit", (0.0, 0))
    push_avg_s = push_ms / max(push_n, 1) / 1e3
    alg = algorithmic_bytes(n_p, n_cells, rb)
    peak, peak_kind = hbm_peak()
    achieved = alg / push_avg_s / 1e9 if push_avg_s > 0 else 0.0
    traffic = measured_traffic(args.precision, n_p, n_cells)

    # ---- e2e through the C ABI with host buffers ----------------------
    e2e = None
    if not args.no_e2e:
        pinned = []
        host = []
        for s in range(2):
            n_s = int(info.n_particles[s])
            real = torch.float64 if prec == Z.FP64 else torch.float32
            buf = {k: torch.empty(n_s, dtype=torch.int32, pin_memory=True)
                   for k in ("ix", "iy")}
            for k in ("x", "y", "ux", "uy", "uz"):
                buf[k] = torch.empty(n_s, dtype=real, pin_memory=True)
            pinned.append(buf)
            host.append({k: v.numpy() for k, v in buf.items()})
            sim.particles(s, with_w=False, with_id=False, out=host[s])
        h2d = sum(v.nbytes for h in host for v in h.values())
        # one untimed pass of the same calls (the first upload and download
        # after the steps run 10-20 ms slower than later ones)
        for s in range(2):
            sim.set_particles(s, host[s])
        sim.step(args.warmup)
        sim.energy()
        for s in range(2):
            sim.particles(s, with_w=False, with_id=False, out=host[s])
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(2):
            sim.set_particles(s, host[s])
        sim.step(args.steps)
        recs = sim.energy()
        for s in range(2):
            sim.particles(s, with_w=False, with_id=False, out=host[s])
        t1 = time.perf_counter()
        barrier(world)
        d2h = h2d + 88 * len(recs)
        e2e_s = all_max(t1 - t0, world)
        e2e = {"value": total_ps / e2e_s, "unit": "particle-steps/s",
               "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps,
               "what": "set_particles from pinned host arrays + steps + "
                       "energy history + get_particles to host, timed "
                       "on the host clock"}
        del pinned

    # ---- secondary figures: FP32 vs FP64, batched vs per-sim ----------
    second = {}
    if world == 1 and not args.no_secondary:
        del sim
        torch.cuda.synchronize()
        if prec == Z.FP32:
            second["fp32_over_fp64"] = fp32_over_fp64(args, stream, torch,
                                                      value)
        second["batched_over_per_sim"] = batched_over_per_sim(args, stream,
                                                              torch)

    # ---- CPU oracle baseline (rank 0 only) ----------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # all host threads (the particle-decomposed mode of Sec. 3.1) on a
        # box of cpu_sample^2 cells, and one thread on a quarter of it.  The
        # timed oracle run (20 steps from the seeded load) is also the
        # reference of the precision errors of both GPU forms at step 20.
        nthreads = os.cpu_count() or 1
        steps_mt = 20
        v, n, secs, orc, lds = oracle_sample(args.cpu_sample, args.ppc,
                                             steps_mt, nthreads, keep=True)
        if prec == Z.FP32 and not args.no_secondary:
            second["precision_vs_oracle"] = precision_vs_oracle(
                orc, lds, args.cpu_sample, steps_mt, stream)
        del orc, lds
        c1 = max(args.cpu_sample // 2, 8)
        v1, n1, secs1 = oracle_sample(c1, args.ppc, 2, 1)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": nthreads,
               "kind": "oracle",
               "sample": "%dx%d periodic box of the same plasma (%d "
                         "particles), %d steps, FP64, %d threads, %.1f s" %
                         (args.cpu_sample, args.cpu_sample, n, steps_mt,
                          nthreads, secs),
               "single_thread": {
                   "value": v1, "unit": "particle-steps/s", "cores": 1,
                   "sample": "%dx%d box (%d particles), 2 steps, %.1f s" %
                             (c1, c1, n1, secs1)}}

    if rank == 0:
        out = {
            "metric": "particle-steps/s", "value": value,
            "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == Z.FP64 else "f32",
            "data": "synthetic", "config": workload_config(args),
            "roofline": {"bound": "hbm", "kernel": "push_deposit",
                         "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": traffic,
                         "algorithmic_bytes_per_launch": alg,
                         "avg_launch_ms": push_avg_s * 1e3},
            "kernels_ms": {k: v[0] / max(v[1], 1) for k, v in prof.items()},
            "resorts_in_timed_region": resorts_timed,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
        }
        out.update(second)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
