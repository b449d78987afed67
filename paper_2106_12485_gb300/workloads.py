"""Configurations of the benchmark workloads (plain data).

Each builder returns a zpic_config (see zpic.config); `scale` shrinks the
grid for parity tests while keeping cell size, time step, particles per cell
and momenta.  The workloads:

* uniform_thermal: uniform thermal electron plasma, 64x64 cells, dx=dy=0.1,
  dt=0.07, 4x4 random particles per cell, u_th=0.1, periodic.
* clouds: collision of plasma clouds, 1024x1024 cells, dx=dy=0.1, dt=0.07;
  two clouds each 25% of the box wide separated by 25% gaps, electrons and
  positrons at 4x4 per cell, drift +-0.2 in x, u_th=0.05 (four species:
  e- left, e+ left, e- right, e+ right).
* lwfa: 4096x512 cells, box 81.92 x 102.4, dt=0.019, moving window along x,
  periodic y, Gaussian laser a0=2, omega0=10, waist 4, FWHM 2 centred
  3 FWHM inside the right edge; cold electrons on a 2x2 lattice behind a
  linear density ramp of length 5 that starts at the box edge.
* lwfa_paper: the paper's own LWFA shape (Sec. 4.1): 2000x512 cells,
  16 particles per cell (4x4 lattice), compensated binomial current
  filter; cell size, time step and laser as in lwfa.
* precision_study: 2048x2048 cells, dx=dy=0.1, dt=0.07, electrons and
  positrons 8x8 per cell each, u_th=0.1 (FP32 or FP64).
* weibel: the paper's cloud-collision (Weibel) case, 512x512 cells,
  electrons and positrons 16x16 per cell each, uniform over the box,
  drifting in opposite directions along z (perpendicular to the plane);
  drift 0.6, u_th=0.1, dx=dy=0.1, dt=0.07 (the paper gives grid and ppc
  only).
* batch_sweep: independent small simulations (see synthetic.plasma.
  batch_specs for how sizes, ppc and u_th are drawn).
"""
from __future__ import annotations

from . import zpic as Z

SEED = 2106012485


def uniform_thermal(nx=64, ny=64, ppc=(4, 4), u_th=0.1, dt=0.07, d=0.1,
                    precision=Z.FP32, **kw):
    sp = Z.species(-1.0, ppc, u_th=(u_th,) * 3)
    return Z.config(nx, ny, (nx * d, ny * d), dt, [sp], precision=precision,
                    seed=kw.pop("seed", SEED), **kw)


def clouds(nx=1024, ny=1024, ppc=(4, 4), drift=0.2, u_th=0.05, dt=0.07,
           d=0.1, precision=Z.FP32, sim_index=0, **kw):
    Lx = nx * d
    left = (0.125 * Lx, 0.375 * Lx)
    right = (0.625 * Lx, 0.875 * Lx)
    sps = []
    for (a, b), dr in ((left, drift), (left, drift), (right, -drift),
                       (right, -drift)):
        qm = -1.0 if len(sps) % 2 == 0 else 1.0
        sps.append(Z.species(qm, ppc, u_th=(u_th,) * 3, u_fl=(dr, 0.0, 0.0),
                             profile=Z.PROFILE_SLAB, x0=a, x1=b))
    return Z.config(nx, ny, (Lx, ny * d), dt, sps, precision=precision,
                    seed=kw.pop("seed", SEED), sim_index=sim_index, **kw)


def lwfa(nx=4096, ny=512, dx=0.02, dy=0.2, dt=0.019, ppc=(2, 2),
         precision=Z.FP32, plasma=True, **kw):
    Lx, Ly = nx * dx, ny * dy
    fwhm = 2.0
    laser = {"a0": 2.0, "omega0": 10.0, "w0": 4.0, "fwhm": fwhm,
             "x0": Lx - 3 * fwhm, "y_center": Ly / 2}
    sps = []
    if plasma:
        sps.append(Z.species(-1.0, ppc, profile=Z.PROFILE_RAMP, x0=Lx,
                             x1=5.0, lattice=True))
    return Z.config(nx, ny, (Lx, Ly), dt, sps, precision=precision,
                    bc_x=Z.BC_OPEN, moving_window=True, laser=laser,
                    seed=kw.pop("seed", SEED), **kw)


def lwfa_paper(nx=2000, ny=512, ppc=(4, 4), **kw):
    return lwfa(nx=nx, ny=ny, ppc=ppc, filter_j=kw.pop("filter_j", True), **kw)


def precision_study(nx=2048, ny=2048, ppc=(8, 8), u_th=0.1, dt=0.07, d=0.1,
                    precision=Z.FP32, **kw):
    sps = [Z.species(-1.0, ppc, u_th=(u_th,) * 3),
           Z.species(1.0, ppc, u_th=(u_th,) * 3)]
    return Z.config(nx, ny, (nx * d, ny * d), dt, sps, precision=precision,
                    seed=kw.pop("seed", SEED), **kw)


def weibel(nx=512, ny=512, ppc=(16, 16), u_fl=0.6, u_th=0.1, dt=0.07,
           d=0.1, precision=Z.FP32, **kw):
    sps = [Z.species(-1.0, ppc, u_th=(u_th,) * 3, u_fl=(0.0, 0.0, u_fl)),
           Z.species(1.0, ppc, u_th=(u_th,) * 3, u_fl=(0.0, 0.0, -u_fl))]
    return Z.config(nx, ny, (nx * d, ny * d), dt, sps, precision=precision,
                    seed=kw.pop("seed", SEED), **kw)


def batch_sweep(specs, dt=0.07, d=0.1, precision=Z.FP32, **kw):
    cfgs = []
    for i, s in enumerate(specs):
        ppc = (s["ppc_side"], s["ppc_side"])
        if s["kind"] == "thermal":
            c = uniform_thermal(s["nx"], s["ny"], ppc=ppc, u_th=s["u_th"],
                                dt=dt, d=d, precision=precision,
                                sim_index=i, **kw)
        else:
            c = clouds(s["nx"], s["ny"], ppc=ppc, drift=s["drift"],
                       u_th=s["u_th"], dt=dt, d=d, precision=precision,
                       sim_index=i, **kw)
        cfgs.append(c)
    return cfgs


# ---- sharding independent simulations over GPUs ---------------------------

def batch_particles(spec):
    """Particles of one batched simulation at creation: the whole box for
    thermal plasma; for the cloud collision two clouds (columns
    [nx/8, 3nx/8) and [5nx/8, 7nx/8)), each with electrons and positrons."""
    k2 = spec["ppc_side"] ** 2
    if spec["kind"] == "thermal":
        return spec["nx"] * spec["ny"] * k2
    nx = spec["nx"]
    width = (3 * nx // 8 - nx // 8) + (7 * nx // 8 - 5 * nx // 8)
    return 2 * width * spec["ny"] * k2


def batch_costs(specs, bytes_per_particle=44, bytes_per_cell=36):
    """Cost of one step of each simulation in algorithmic HBM bytes: the
    particle record read and written once (44 B in FP32) plus E, B read and
    J written once per cell (36 B)."""
    return [bytes_per_particle * batch_particles(s) +
            bytes_per_cell * s["nx"] * s["ny"] for s in specs]


def lpt_partition(costs, n_parts):
    """Longest-processing-time-first assignment of independent jobs to
    n_parts workers: jobs in decreasing cost (ties by index) each go to the
    worker with the least load so far (ties to the lowest worker).  The
    result is deterministic, so every rank computes the same partition
    without exchanging anything; the largest load exceeds the smallest by
    at most the largest job.  Returns one ascending list of job indices per
    worker."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * n_parts
    parts = [[] for _ in range(n_parts)]
    for i in order:
        w = min(range(n_parts), key=lambda p: (load[p], p))
        parts[w].append(i)
        load[w] += costs[i]
    return [sorted(p) for p in parts]
