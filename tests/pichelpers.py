"""Shared helpers of the GPU parity tests: run the same seeded inputs
through the CUDA library and through the FP64 oracle and compare.

Inputs come only from synthetic/ (the seeded generator); expected values
come only from oracle/.  Nothing here feeds a GPU result into the oracle.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2106_12485_gb300 import zpic as Z

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")


def q0_of(qm, ppc):
    return (1.0 if qm > 0 else -1.0) / ppc


def oracle_species(ld, qm, ppc, cap=None):
    f = lambda k: np.asarray(ld[k], dtype=np.float64)  # noqa: E731
    return O.Species(qm, q0_of(qm, ppc), ld["ix"], ld["iy"], f("x"), f("y"),
                     f("ux"), f("uy"), f("uz"), w=f("w"), ids=ld["id"],
                     cap=cap)


def oracle_sim(cfg, loads, window=None, cap_extra=0):
    """The oracle on `loads` (one per species of cfg)."""
    species = []
    for s, ld in enumerate(loads):
        sp = cfg.species[s]
        species.append(oracle_species(ld, sp.q_over_m, sp.ppc_x * sp.ppc_y,
                                      cap=len(ld["ix"]) + cap_extra))
    dx, dy = cfg.box_x / cfg.nx, cfg.box_y / cfg.ny
    return O.Sim(cfg.nx, cfg.ny, dx, dy, cfg.dt, open_x=bool(cfg.bc_x),
                 species=species, window=window,
                 filter_j=bool(cfg.flags & Z.FILTER_J))


def make_pair(cfg, loads, fields=None, window=None, cap_extra=0):
    """GPU sim (cfg, particles from `loads`) and oracle sim on the same
    inputs.  cfg's species give q/m and ppc; their profile should be NONE so
    that `loads` (one per species) is the whole initial state."""
    gpu = Z.Sim(cfg)
    for s, ld in enumerate(loads):
        gpu.set_particles(s, ld)
    species = []
    for s, ld in enumerate(loads):
        sp = cfg.species[s]
        species.append(oracle_species(ld, sp.q_over_m, sp.ppc_x * sp.ppc_y,
                                      cap=len(ld["ix"]) + cap_extra))
    dx, dy = cfg.box_x / cfg.nx, cfg.box_y / cfg.ny
    orc = O.Sim(cfg.nx, cfg.ny, dx, dy, cfg.dt, open_x=bool(cfg.bc_x),
                species=species, window=window,
                filter_j=bool(cfg.flags & Z.FILTER_J))
    if fields:
        for k, v in fields.items():
            gpu.set_field(k, v)
            orc.set_field(k, np.asarray(v, dtype=np.float64))
    return gpu, orc


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.linalg.norm(a)
    return np.linalg.norm(a - b) / nb


def compare_fields(gpu, orc, tol, names=FIELDS):
    errs = {}
    for k in names:
        g = gpu.field(k)
        o = orc.f[k]
        errs[k] = rel_l2(g, o)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "field rel L2 above %g: %s" % (tol, bad)
    return errs


def by_id(st):
    order = np.argsort(st["id"], kind="stable")
    return {k: v[order] for k, v in st.items()}


def compare_particles(gpu, orc, s, nx, ny, tol, x_ref=None):
    """Counts exact, ids equal, u rel L2 <= tol, positions: rel L2 of the
    displacement from x_ref (by id) <= tol, or of the absolute cell
    coordinate when x_ref is None."""
    g = by_id(gpu.particles(s))
    o = by_id(orc.species[s].state())
    assert len(g["id"]) == len(o["id"]), "particle count differs"
    np.testing.assert_array_equal(g["id"], o["id"])
    gx = g["ix"] + g["x"].astype(np.float64)
    gy = g["iy"] + g["y"].astype(np.float64)
    ox = o["ix"] + o["x"]
    oy = o["iy"] + o["y"]
    # periodic unwrap of the difference
    ddx = (gx - ox + nx / 2) % nx - nx / 2
    ddy = (gy - oy + ny / 2) % ny - ny / 2
    errs = {}
    if x_ref is not None:
        rx, ry = x_ref
        mx = (ox - rx + nx / 2) % nx - nx / 2
        my = (oy - ry + ny / 2) % ny - ny / 2
        den = np.sqrt(np.sum(mx ** 2 + my ** 2))
    else:
        den = np.sqrt(np.sum(ox ** 2 + oy ** 2))
    errs["pos"] = np.sqrt(np.sum(ddx ** 2 + ddy ** 2)) / max(den, 1e-300)
    gu = np.stack([g["ux"], g["uy"], g["uz"]]).astype(np.float64)
    ou = np.stack([o["ux"], o["uy"], o["uz"]])
    errs["u"] = rel_l2(gu, ou)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, "particle rel L2 above %g: %s" % (tol, bad)
    return errs


def positions_by_id(sp_state):
    st = by_id(sp_state)
    return st["ix"] + np.asarray(st["x"], np.float64), \
        st["iy"] + np.asarray(st["y"], np.float64)


def cic_rho(nx, ny, st, q0, open_x=False):
    """Charge density at nodes from CIC weights (FP64, numpy)."""
    ix = np.asarray(st["ix"], np.int64)
    iy = np.asarray(st["iy"], np.int64)
    x = np.asarray(st["x"], np.float64)
    y = np.asarray(st["y"], np.float64)
    w = np.asarray(st.get("w", np.ones_like(x)), np.float64) * q0
    rho = np.zeros(nx * ny)
    for di, wx in ((0, 1 - x), (1, x)):
        for dj, wy in ((0, 1 - y), (1, y)):
            i = ix + di
            j = (iy + dj) % ny
            keep = np.ones_like(i, dtype=bool)
            if open_x:
                keep = (i >= 0) & (i < nx)
            i = i % nx
            np.add.at(rho, (j * nx + i)[keep], (w * wx * wy)[keep])
    return rho.reshape(ny, nx)


def continuity_residual(jx, jy, rho0, rho1, dx, dy, dt):
    div = (jx - np.roll(jx, 1, axis=1)) / dx + (jy - np.roll(jy, 1, axis=0)) / dy
    drho = (rho1 - rho0) / dt
    return np.linalg.norm(drho + div) / np.linalg.norm(drho)


def strip_layout(ld):
    """The load without weight and id planes: uploaded to a simulation
    without ZPIC_TRACK_IDS it gives the plain particle layout (the one the
    16x16 FP32 kernel is specialised for); every weight of these loads is 1,
    so the particles are the same."""
    assert np.all(np.asarray(ld["w"]) == 1)
    return {k: v for k, v in ld.items() if k not in ("w", "id")}


def tile_counts_of(st, tx, ty, ntx, nty):
    """Particles per tile (index ty * ntx + tx) of a particle set."""
    t = (np.asarray(st["iy"]) // ty) * ntx + np.asarray(st["ix"]) // tx
    return np.bincount(t, minlength=ntx * nty)


def cic_map(nx, ny, st, weight, open_x=False):
    """Sum of `weight` per particle spread to the nodes with CIC weights
    (FP64, numpy); weight = the particle's charge gives the charge density,
    charge x u_k a momentum density."""
    ix = np.asarray(st["ix"], np.int64)
    iy = np.asarray(st["iy"], np.int64)
    x = np.asarray(st["x"], np.float64)
    y = np.asarray(st["y"], np.float64)
    w = np.asarray(weight, np.float64)
    out = np.zeros(nx * ny)
    for di, wx in ((0, 1 - x), (1, x)):
        for dj, wy in ((0, 1 - y), (1, y)):
            i = ix + di
            j = (iy + dj) % ny
            keep = (i >= 0) & (i < nx) if open_x else np.ones(i.shape, bool)
            i = i % nx
            np.add.at(out, (j * nx + i)[keep], (w * wx * wy)[keep])
    return out.reshape(ny, nx)


def fluct_rel_l2(a, b):
    """Relative L2 of a - b against the fluctuation of b about its mean (a
    uniform plasma's density is dominated by its mean, which hides errors in
    the positions)."""
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(np.asarray(a, np.float64) - b)
    return d / max(np.linalg.norm(b - b.mean()), 1e-300)


def match_particles(g, o, scale_u=1.0):
    """Pairs the particles of two sets without ids: each particle of g with
    its nearest neighbour of o in (global x, global y, u / scale_u).  Returns
    (index into o for every particle of g, distance); the caller checks that
    the pairing is one-to-one and the distances are small."""
    from scipy.spatial import cKDTree
    def pts(s):
        return np.stack([np.asarray(s["ix"], np.float64) + s["x"],
                         np.asarray(s["iy"], np.float64) + s["y"],
                         np.asarray(s["ux"], np.float64) / scale_u,
                         np.asarray(s["uy"], np.float64) / scale_u,
                         np.asarray(s["uz"], np.float64) / scale_u], axis=1)
    d, k = cKDTree(pts(o)).query(pts(g))
    return k, d
