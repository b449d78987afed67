"""GPU parity of the particle layout the benchmark runs: species that store
neither weights nor ids.  The 16x16-tile FP32 particle kernel is compiled
separately for that layout (periodic and open x boundary), so these tests
compare exactly that form with the FP64 oracle on the same seeded inputs
(validation against the sequential code, Sec. 4.2), and check through
zpic_info.push_variants, which the kernel itself records, that it ran.

Without ids the particles are compared through what does not need them:
counts per species and per tile, the nine fields, the energy history,
charge and momentum densities of the particles, the continuity residual,
and, at full size, a nearest-neighbour pairing of the particles of a region.
"""
import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu

TOL32 = 1e-4


def plain_pair(nx, ny, steps_energy=1, open_x=False, ppc=(8, 8)):
    """Electrons and positrons, uniform thermal, both sides from the same
    seeded loads; the GPU copy gets them without weight and id planes."""
    sps = [Z.species(qm, ppc, profile=Z.PROFILE_NONE) for qm in (-1.0, 1.0)]
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07, sps, tile=(16, 16),
                   energy_every=steps_energy,
                   bc_x=Z.BC_OPEN if open_x else Z.BC_PERIODIC)
    loads = [P.plasma_load(nx, ny, ppc[0], ppc[1], species=s,
                           u_th=(0.1, 0.1, 0.1)) for s in range(2)]
    gpu = Z.Sim(cfg)
    for s, ld in enumerate(loads):
        gpu.set_particles(s, H.strip_layout(ld))
    orc = H.oracle_sim(cfg, loads)
    return cfg, gpu, orc


def q0(s, ppc=64):
    return (-1.0 if s == 0 else 1.0) / ppc


def check_plain(cfg, gpu, orc, steps, open_x):
    nx, ny = cfg.nx, cfg.ny
    form = Z.PUSH_PLAIN_OPEN if open_x else Z.PUSH_PLAIN_PERIODIC
    info = gpu.info()
    assert list(info.push_variants[:2]) == [form, form]
    ntx, nty = info.ntiles_x, info.ntiles_y
    for s in range(2):
        g = gpu.particles(s, with_w=False, with_id=False)
        o = orc.species[s].state()
        # counts: exact per species
        assert len(g["ix"]) == len(o["ix"]) == orc.species[s].n
        # per tile: exact up to particles within rounding of a tile face
        ox = o["ix"] + o["x"]
        oy = o["iy"] + o["y"]
        near = np.sum((np.abs(ox - np.round(ox / 16) * 16) < 1e-5) |
                      (np.abs(oy - np.round(oy / 16) * 16) < 1e-5))
        dt = np.abs(gpu.tile_counts(s) - H.tile_counts_of(o, 16, 16, ntx, nty))
        assert dt.sum() <= 2 * near, (s, dt.sum(), near)
        np.testing.assert_array_equal(
            gpu.tile_counts(s), H.tile_counts_of(g, 16, 16, ntx, nty))
        # charge and momentum densities of the particles
        qg = np.full(len(g["ix"]), q0(s))
        qo = np.full(len(o["ix"]), q0(s))
        e = H.fluct_rel_l2(H.cic_map(nx, ny, g, qg, open_x),
                           H.cic_map(nx, ny, o, qo, open_x))
        assert e <= TOL32, ("rho", s, e)
        for k in ("ux", "uy", "uz"):
            e = H.fluct_rel_l2(
                H.cic_map(nx, ny, g, qg * g[k].astype(np.float64), open_x),
                H.cic_map(nx, ny, o, qo * o[k], open_x))
            assert e <= TOL32, (k, s, e)
    H.compare_fields(gpu, orc, TOL32)
    ge = gpu.energy()
    assert len(ge) == steps
    for (st, wE, wB, kin), (ost, owE, owB, okin) in zip(ge, orc.history):
        assert st == ost
        tot_o = owE + owB + okin[:2].sum()
        assert abs(wE + wB + sum(kin[:2]) - tot_o) <= 1e-3 * tot_o
        for s in range(2):
            assert abs(kin[s] - okin[s]) <= 1e-3 * okin[s]


def test_plain_layout_periodic_matches_oracle():
    cfg, gpu, orc = plain_pair(64, 48)
    gpu.step(10)
    orc.step(10, nthreads=4)
    check_plain(cfg, gpu, orc, 10, open_x=False)


def test_plain_layout_open_x_matches_oracle():
    # open x boundary: the plasma streams out through both x edges (the
    # removed particles leave the counts), fields read zero beyond them
    cfg, gpu, orc = plain_pair(64, 48, open_x=True)
    gpu.step(10)
    orc.step(10, nthreads=4)
    n0 = 64 * 48 * 64
    for s in range(2):
        assert orc.species[s].n < n0   # something left
    check_plain(cfg, gpu, orc, 10, open_x=True)


def test_plain_layout_continuity_residual():
    cfg, gpu, orc = plain_pair(64, 48)
    del orc
    gpu.step(3)
    g0 = [gpu.particles(s, with_w=False, with_id=False) for s in range(2)]
    rho0 = sum(H.cic_map(64, 48, g0[s], np.full(len(g0[s]["ix"]), q0(s)))
               for s in range(2))
    gpu.step(1)
    g1 = [gpu.particles(s, with_w=False, with_id=False) for s in range(2)]
    rho1 = sum(H.cic_map(64, 48, g1[s], np.full(len(g1[s]["ix"]), q0(s)))
               for s in range(2))
    res = H.continuity_residual(gpu.field("jx"), gpu.field("jy"), rho0, rho1,
                                0.1, 0.1, 0.07)
    assert res <= 1e-6, res


def test_plain_layout_full_size_sampled_parity():
    """The benchmark's own configuration (2048^2 cells, e-/e+ 8x8 per cell,
    no ids): one step, then the particles and fields of a 32x32-cell region
    against the oracle run on the regenerated initial load of that region
    plus a 4-cell margin.  Particles are paired by nearest neighbour in
    position and momentum."""
    nx = ny = 2048
    cfg = W.precision_study()
    assert not cfg.flags & Z.TRACK_IDS
    gpu = Z.Sim(cfg)
    n_each = nx * ny * 64
    gpu.step(1)
    assert gpu.num_particles(0) == n_each and gpu.num_particles(1) == n_each
    info = gpu.info()
    assert info.tile_x == info.tile_y == 16
    assert list(info.push_variants[:2]) == [Z.PUSH_PLAIN_PERIODIC] * 2
    t_lo = 1024 // 16
    lo, hi = 1020, 1060
    cx, cy = np.meshgrid(np.arange(lo, hi), np.arange(lo, hi))
    cells = (cy * nx + cx).ravel()
    loads = []
    for s in range(2):
        ld = P.plasma_load(nx, ny, 8, 8, species=s, u_th=(0.1, 0.1, 0.1),
                           cells=cells)
        ld["ix"] = ld["ix"] - lo
        ld["iy"] = ld["iy"] - lo
        loads.append(ld)
    from tests.test_gpu_workloads import oracle_from_load
    orc = oracle_from_load(W.precision_study(hi - lo, hi - lo), loads)
    orc.step(1)
    for s in range(2):
        got = []
        for ty in (t_lo, t_lo + 1):
            t0 = ty * info.ntiles_x + t_lo
            got.append(gpu.particles(s, tiles=(t0, t0 + 2), with_w=False,
                                     with_id=False))
        g = {k: np.concatenate([d[k] for d in got]) for k in got[0]}
        o = orc.species[s].state()
        o = {k: v for k, v in o.items()}
        o["ix"] = o["ix"] + lo
        o["iy"] = o["iy"] + lo
        inside = ((o["ix"] >= 1024) & (o["ix"] < 1056) &
                  (o["iy"] >= 1024) & (o["iy"] < 1056))
        o = {k: v[inside] for k, v in o.items()}
        # the region's count: exact up to particles within rounding of its
        # faces (FP32 and FP64 may put them on either side)
        assert abs(len(g["ix"]) - len(o["ix"])) <= 4
        k, d = H.match_particles(g, o)
        ok = d <= 4e-6
        assert np.unique(k[ok]).size == ok.sum()        # one-to-one
        gx = g["ix"] + g["x"].astype(np.float64)
        gy = g["iy"] + g["y"].astype(np.float64)
        edge = ((np.abs(gx - 1024) < 1e-5) | (np.abs(gx - 1056) < 1e-5) |
                (np.abs(gy - 1024) < 1e-5) | (np.abs(gy - 1056) < 1e-5))
        assert np.all(ok | edge), np.sort(d)[-5:]
        assert ok.sum() >= len(g["ix"]) - 4
        for c, f in (("ix", "x"), ("iy", "y")):
            np.testing.assert_allclose(
                (g[c] + g[f].astype(np.float64))[ok],
                (o[c] + o[f])[k[ok]], rtol=0, atol=2e-6)
        for q in ("ux", "uy", "uz"):
            np.testing.assert_allclose(g[q][ok], o[q][k[ok]], rtol=0,
                                       atol=2e-6)
    a, b = 1024 - lo, 1056 - lo
    for name in H.FIELDS:
        gf = gpu.field(name)[1024:1056, 1024:1056]
        of = orc.f[name][a:b, a:b]
        assert H.rel_l2(gf, of) <= 1e-4, name
