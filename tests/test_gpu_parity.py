"""GPU parity: the CUDA library against the FP64 oracle on the same seeded
inputs (through the C ABI).  Tolerances: counts and ids exact; fields and
particle state relative L2 <= 1e-4 after 10 steps in FP32 (1e-10 in FP64);
energy history <= 1e-3 relative; continuity residual <= 1e-6.
"""
import numpy as np
import pytest

from paper_2106_12485_gb300 import zpic as Z
from paper_2106_12485_gb300 import workloads as W
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
TOL64 = 1e-10


def cfg_for_loads(nx, ny, d, dt, qms_ppc, **kw):
    sps = [Z.species(qm, ppc, profile=Z.PROFILE_NONE) for qm, ppc in qms_ppc]
    return Z.config(nx, ny, (nx * d[0], ny * d[1]), dt, sps, track_ids=True,
                    **kw)


def test_library_init_matches_generator():
    cfg = W.uniform_thermal(track_ids=True)
    sim = Z.Sim(cfg)
    g = H.by_id(sim.particles(0))
    ref = H.by_id(P.plasma_load(64, 64, 4, 4, u_th=(0.1, 0.1, 0.1)))
    for k in ("ix", "iy", "id", "x", "y"):
        np.testing.assert_array_equal(g[k], ref[k])
    for k in ("ux", "uy", "uz"):
        np.testing.assert_allclose(g[k], ref[k], rtol=3e-7, atol=1e-9)


def test_parity_uniform_thermal_10_steps():
    nx = ny = 64
    ld = P.plasma_load(nx, ny, 4, 4, u_th=(0.1, 0.1, 0.1))
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (4, 4))])
    gpu, orc = H.make_pair(cfg, [ld])
    x0 = H.positions_by_id(orc.species[0].state())
    gpu.step(10)
    orc.step(10)
    H.compare_fields(gpu, orc, TOL32)
    H.compare_particles(gpu, orc, 0, nx, ny, TOL32, x_ref=x0)


@pytest.mark.parametrize("tile", [(16, 16), (8, 4), (32, 32)])
def test_parity_ragged_tiles_fast_particles_random_fields(tile):
    nx, ny = 72, 40
    ld = P.random_particles(nx, ny, 20000, seed=5, umax=3.0,
                            dtype=np.float32)
    ld["w"] = np.ones(len(ld["ix"]), np.float32)
    fields = P.random_fields(nx, ny, seed=9, scale=0.2)
    fields = {k: v.astype(np.float32).astype(np.float64)
              for k, v in fields.items()}
    cfg = cfg_for_loads(nx, ny, (0.1, 0.13), 0.06, [(-1.0, (2, 2))],
                        tile=tile)
    gpu, orc = H.make_pair(cfg, [ld], fields=fields)
    x0 = H.positions_by_id(orc.species[0].state())
    for _ in range(3):
        gpu.step(1)
        orc.step(1)
    H.compare_fields(gpu, orc, TOL32)
    H.compare_particles(gpu, orc, 0, nx, ny, TOL32, x_ref=x0)


def test_energy_history_50_steps():
    nx = ny = 64
    ld = P.plasma_load(nx, ny, 4, 4, u_th=(0.1, 0.1, 0.1))
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (4, 4))],
                        energy_every=1)
    gpu, orc = H.make_pair(cfg, [ld])
    gpu.step(50)
    orc.step(50)
    ge = gpu.energy()
    assert len(ge) == 50
    for (st, wE, wB, kin), (ost, owE, owB, okin) in zip(ge, orc.history):
        assert st == ost
        tot_o = owE + owB + okin.sum()
        tot_g = wE + wB + sum(kin)
        assert abs(tot_g - tot_o) <= 1e-3 * tot_o
        assert abs(kin[0] - okin[0]) <= 1e-3 * okin[0]
        assert abs(wE - owE) <= 1e-3 * max(owE, 1e-3 * tot_o)


def test_continuity_residual():
    nx = ny = 64
    dx = dy = 0.1
    dt = 0.07
    ld = P.plasma_load(nx, ny, 4, 4, u_th=(0.1, 0.1, 0.1))
    cfg = cfg_for_loads(nx, ny, (dx, dy), dt, [(-1.0, (4, 4))])
    gpu = Z.Sim(cfg)
    gpu.set_particles(0, ld)
    gpu.step(3)
    q0 = -1.0 / 16
    rho0 = H.cic_rho(nx, ny, gpu.particles(0), q0)
    gpu.step(1)
    rho1 = H.cic_rho(nx, ny, gpu.particles(0), q0)
    res = H.continuity_residual(gpu.field("jx"), gpu.field("jy"), rho0, rho1,
                                dx, dy, dt)
    assert res <= 1e-6, res


def test_migration_invariants():
    nx, ny = 96, 80
    ld = P.random_particles(nx, ny, 50000, seed=2, umax=2.0,
                            dtype=np.float32)
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (4, 4))],
                        tile=(16, 16))
    gpu = Z.Sim(cfg)
    gpu.set_particles(0, ld)
    for _ in range(5):
        gpu.step(2)
        st = gpu.particles(0)
        # count conserved, ids a permutation
        assert len(st["id"]) == 50000
        np.testing.assert_array_equal(np.sort(st["id"]), np.arange(50000))
        # every particle lies in its tile (get_particles is in tile order)
        cnt = gpu.tile_counts(0)
        tiles = np.repeat(np.arange(cnt.size), cnt)
        info = gpu.info()
        t = (st["iy"] // info.tile_y) * info.ntiles_x + st["ix"] // info.tile_x
        np.testing.assert_array_equal(t, tiles)
        assert (st["x"] >= 0).all() and (st["x"] < 1).all()
        assert (st["y"] >= 0).all() and (st["y"] < 1).all()


def test_overflow_recovery_matches_oracle():
    # a beam at four times the configured density (8x8 particles per cell
    # against 4x4) drifts into empty tiles, whose capacity is the configured
    # full density plus 1 %: they overflow and the host re-sorts
    nx, ny = 64, 32
    ld = P.plasma_load(nx, ny, 8, 8, u_th=(0.05, 0.05, 0.05),
                       u_fl=(0.9, 0.0, 0.0), x_range=(0, 8))
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (4, 4))],
                        tile=(8, 8), capacity_slack=0.01)
    gpu, orc = H.make_pair(cfg, [ld])
    x0 = H.positions_by_id(orc.species[0].state())
    gpu.step(12)
    orc.step(12)
    assert gpu.info().resorts >= 1
    assert gpu.info().step == 12
    H.compare_fields(gpu, orc, TOL32)
    H.compare_particles(gpu, orc, 0, nx, ny, TOL32, x_ref=x0)


def test_parity_fp64_mode():
    nx, ny = 48, 40
    ld = P.plasma_load(nx, ny, 3, 3, u_th=(0.2, 0.2, 0.2), dtype=np.float64)
    fields = P.random_fields(nx, ny, seed=4, scale=0.1)
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (3, 3))],
                        precision=Z.FP64, tile=(8, 8))
    gpu, orc = H.make_pair(cfg, [ld], fields=fields)
    x0 = H.positions_by_id(orc.species[0].state())
    gpu.step(10)
    orc.step(10)
    H.compare_fields(gpu, orc, TOL64)
    H.compare_particles(gpu, orc, 0, nx, ny, TOL64, x_ref=x0)


def test_parity_two_clouds_four_species():
    nx, ny = 128, 64
    loads = P.two_clouds(nx, ny, 2, 2, drift=0.2, u_th=0.05)
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07,
                        [(-1.0, (2, 2)), (1.0, (2, 2)), (-1.0, (2, 2)),
                         (1.0, (2, 2))], energy_every=5)
    gpu, orc = H.make_pair(cfg, loads)
    refs = [H.positions_by_id(sp.state()) for sp in orc.species]
    gpu.step(10)
    orc.step(10)
    H.compare_fields(gpu, orc, TOL32)
    for s in range(4):
        H.compare_particles(gpu, orc, s, nx, ny, TOL32, x_ref=refs[s])


def test_vacuum_yee_only():
    nx, ny = 100, 36
    fields = P.random_fields(nx, ny, seed=8, scale=1.0)
    fields = {k: v.astype(np.float32).astype(np.float64)
              for k, v in fields.items()}
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.15), 0.06, [])
    gpu = Z.Sim(cfg)
    from oracle import oracle as O
    orc = O.Sim(nx, ny, 0.1, 0.15, 0.06)
    for k, v in fields.items():
        gpu.set_field(k, v)
        orc.set_field(k, v)
    gpu.step(20)
    orc.step(20)
    H.compare_fields(gpu, orc, 1e-5, names=H.FIELDS[:6])


def test_library_init_clouds_matches_generator():
    nx, ny = 128, 32
    cfg = W.clouds(nx, ny, ppc=(2, 2), track_ids=True)
    sim = Z.Sim(cfg)
    ref = P.two_clouds(nx, ny, 2, 2, drift=0.2, u_th=0.05)
    for s in range(4):
        g = H.by_id(sim.particles(s))
        r = H.by_id(ref[s])
        for k in ("ix", "iy", "id", "x", "y"):
            np.testing.assert_array_equal(g[k], r[k])
        for k in ("ux", "uy", "uz"):
            np.testing.assert_allclose(g[k], r[k], rtol=3e-7, atol=1e-9)


def test_error_paths():
    cfg = cfg_for_loads(32, 32, (0.1, 0.1), 0.07, [(-1.0, (2, 2))])
    sim = Z.Sim(cfg)
    bad = P.random_particles(32, 32, 10, seed=1, dtype=np.float32)
    bad["ix"][3] = 32
    with pytest.raises(Z.ZpicError) as e:
        sim.set_particles(0, bad)
    assert e.value.code == Z.EINVAL
    out = np.empty(10)
    code = Z.lib().zpic_get_fields_f64(sim.h, Z.EX, out.ctypes.data, 10)
    assert code == Z.ECAP
    assert Z.lib().zpic_step(sim.h, -1) == Z.EINVAL
    # empty simulation steps fine
    sim.step(3)
    assert sim.info().step == 3
    assert sim.num_particles(0) == 0


def test_field_energy_matches_oracle():
    nx, ny = 80, 60
    fields = P.random_fields(nx, ny, seed=21, scale=0.7)
    fields = {k: v.astype(np.float32).astype(np.float64)
              for k, v in fields.items()}
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.2), 0.06, [])
    gpu = Z.Sim(cfg)
    from oracle import oracle as O
    orc = O.Sim(nx, ny, 0.1, 0.2, 0.06)
    for k, v in fields.items():
        gpu.set_field(k, v)
        orc.set_field(k, v)
    wE, wB = gpu.field_energy()
    oE, oB = orc.field_energy()
    assert wE == pytest.approx(oE, rel=1e-6)
    assert wB == pytest.approx(oB, rel=1e-6)
    assert gpu.field_energy() == (wE, wB)    # fixed summation order


@pytest.mark.parametrize("precision,tol", [(Z.FP32, 1e-4), (Z.FP64, 1e-10)])
def test_current_filter_matches_oracle(precision, tol):
    # filtered J (what the getters return and the field update uses), the
    # fields it drives and the particles, with a ragged grid (40 x 36 cells:
    # partial Yee blocks in both directions)
    nx, ny = 40, 36
    dt = np.float64 if precision == Z.FP64 else np.float32
    cfg = W.uniform_thermal(nx, ny, ppc=(3, 3), u_th=0.2, precision=precision,
                            track_ids=True, filter_j=True)
    ld = P.plasma_load(nx, ny, 3, 3, u_th=(0.2,) * 3, dtype=dt)
    fields = P.random_fields(nx, ny, seed=5, scale=0.3)
    gpu, orc = H.make_pair(cfg, [ld], fields=fields)
    x0 = H.positions_by_id(orc.species[0].state())
    for _ in range(2):
        gpu.step(4)
        orc.step(4)
        H.compare_fields(gpu, orc, tol)
        H.compare_particles(gpu, orc, 0, nx, ny, tol, x_ref=x0)
    # the filter removes the grid-scale noise of the deposit: the filtered
    # current is smoother than an unfiltered run of the same state
    raw = Z.Sim(W.uniform_thermal(nx, ny, ppc=(3, 3), u_th=0.2,
                                  precision=precision, track_ids=True))
    raw.set_particles(0, ld)
    for k, v in fields.items():
        raw.set_field(k, v)
    raw.step(1)
    filt = Z.Sim(cfg)
    filt.set_particles(0, ld)
    for k, v in fields.items():
        filt.set_field(k, v)
    filt.step(1)
    for k in ("jx", "jy", "jz"):
        a, b = raw.field(k), filt.field(k)
        assert np.sum(np.diff(b, axis=1) ** 2) < 0.5 * np.sum(np.diff(a, axis=1) ** 2)



@pytest.mark.parametrize("precision", [Z.FP32, Z.FP64])
def test_field_energy_sum_is_compensated(precision):
    # one cell of E_x = 1e9 (square 1e18, ulp 128) among 262,143 cells of
    # E_x = 1: a plain FP64 sum drops every +1 added to the huge partial
    # (255 of them in the first row's first thread alone, two ulps); the
    # compensated sum returns the exactly rounded total.  dx dy / 2 = 1/8
    # keeps the final scaling exact.
    nx, ny = 65536, 4
    ex = np.ones((ny, nx))
    ex[0, 0] = 1e9
    cfg = Z.config(nx, ny, (nx * 0.5, ny * 0.5), 0.3, [], precision=precision)
    gpu = Z.Sim(cfg)
    gpu.set_field("ex", ex)
    wE, wB = gpu.field_energy()
    exact = 10 ** 18 + (nx * ny - 1)
    assert wB == 0.0
    assert wE / 0.125 == float(exact)


@pytest.mark.parametrize("precision", [Z.FP32, Z.FP64])
def test_particle_round_trip_through_host(precision):
    # host transfers of the particle store: the download in tile ranges
    # (any split, empty ranges included) equals the whole download, in the
    # store's own precision and converted; an upload of what was downloaded
    # gives back the same particles; weights and ids travel with them
    nx, ny = 72, 40                      # ragged 16 x 16 tiles (5 x 3)
    real = np.float64 if precision == Z.FP64 else np.float32
    other = np.float32 if precision == Z.FP64 else np.float64
    ld = P.random_particles(nx, ny, 30000, seed=9, umax=1.0, dtype=real)
    ld["w"] = (0.5 + (np.arange(30000) % 7) / 7).astype(real)
    cfg = cfg_for_loads(nx, ny, (0.1, 0.1), 0.07, [(-1.0, (4, 4))],
                        precision=precision, tile=(16, 16))
    gpu = Z.Sim(cfg)
    gpu.set_particles(0, ld)
    gpu.step(3)
    a = gpu.particles(0)
    assert len(a["id"]) == 30000
    nt = gpu.info().ntiles_x * gpu.info().ntiles_y
    for cuts in ((0, nt), (0, 1, 1, 7, nt), (0, 3, 4, nt - 1, nt)):
        parts = [gpu.particles(0, tiles=(cuts[i], cuts[i + 1]))
                 for i in range(len(cuts) - 1)]
        for k in a:
            np.testing.assert_array_equal(
                np.concatenate([p_[k] for p_ in parts]), a[k])
    b = gpu.particles(0, dtype=other)
    for k in a:
        np.testing.assert_array_equal(b[k], a[k].astype(b[k].dtype))
    gpu.set_particles(0, a)
    c = H.by_id(gpu.particles(0))
    a = H.by_id(a)
    for k in a:
        np.testing.assert_array_equal(c[k], a[k])
