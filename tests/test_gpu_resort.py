"""The cell-order re-sort (zpic_config.sort_every) and the settings the full
autotuner chooses, through the C ABI.

Every sort_every steps the particles of each tile are rewritten in
cell-interleaved order (the first particle of every cell in row-major cell
order, then the second of every cell that has one, ...), and the particle
kernel keeps the store order from step to step.  The order of the particles
in the store is not part of the method: the FP32 current is an exact
integer sum, so a run with re-sorts must agree bit for bit with one
without, and the FP64 form must still match the oracle (validation against
the sequential code, Sec. 4.2)."""
import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu


def same_run(a, b, n_species):
    for k in H.FIELDS:
        np.testing.assert_array_equal(a.field(k, np.float32),
                                      b.field(k, np.float32), err_msg=k)
    for s in range(n_species):
        pa, pb = H.by_id(a.particles(s)), H.by_id(b.particles(s))
        for k in ("id", "ix", "iy", "x", "y", "ux", "uy", "uz"):
            np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)
    for ra, rb in zip(a.energy(), b.energy()):
        assert ra[0] == rb[0] and ra[1] == rb[1] and ra[2] == rb[2]


def test_resort_is_bitwise_neutral_fp32():
    cfg0 = W.clouds(96, 80, ppc=(3, 3), track_ids=True, energy_every=5,
                    sort_every=-1)
    cfg1 = W.clouds(96, 80, ppc=(3, 3), track_ids=True, energy_every=5,
                    sort_every=3)
    a, b = Z.Sim(cfg0), Z.Sim(cfg1)
    a.step(25)
    b.step(25)
    assert a.info().sorts == 0
    assert b.info().sorts == 25 // 3 and b.info().sort_every == 3
    same_run(a, b, cfg0.n_species)


def test_resort_gives_the_cell_interleaved_order():
    nx = ny = 64
    cfg = W.uniform_thermal(nx, ny, ppc=(4, 4), tile=(16, 16),
                            track_ids=True, sort_every=2)
    sim = Z.Sim(cfg)
    sim.step(2)                                   # re-sorted after step 2
    assert sim.info().sorts == 1
    cnt = sim.tile_counts(0)
    t = 5
    st = sim.particles(0, tiles=(t, t + 1))
    tx0, ty0 = (t % 4) * 16, (t // 4) * 16
    lc = (st["iy"] - ty0) * 16 + (st["ix"] - tx0)
    assert len(lc) == cnt[t]
    counts = np.bincount(lc, minlength=256)
    # expected: rank 0 of every non-empty cell in cell order, then rank 1 ...
    want = np.concatenate([np.nonzero(counts > r)[0]
                           for r in range(counts.max())])
    np.testing.assert_array_equal(lc, want)


@pytest.mark.parametrize("sort_every", [1, 3])
def test_resort_fp64_matches_oracle(sort_every):
    nx, ny = 48, 40
    ld = P.plasma_load(nx, ny, 3, 3, u_th=(0.2, 0.2, 0.2), dtype=np.float64)
    sps = [Z.species(-1.0, (3, 3), profile=Z.PROFILE_NONE)]
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07, sps,
                   precision=Z.FP64, tile=(8, 8), track_ids=True,
                   sort_every=sort_every)
    gpu, orc = H.make_pair(cfg, [ld])
    x0 = H.positions_by_id(orc.species[0].state())
    gpu.step(10)
    orc.step(10)
    assert gpu.info().sorts == 10 // sort_every
    H.compare_fields(gpu, orc, 1e-10)
    H.compare_particles(gpu, orc, 0, nx, ny, 1e-10, x_ref=x0)


def test_resort_with_overflow_recovery_matches_oracle():
    # the overflow re-sort on the host reads the current copy of the store,
    # which the cell-order re-sort switches on the device
    nx, ny = 64, 32
    ld = P.plasma_load(nx, ny, 8, 8, u_th=(0.05, 0.05, 0.05),
                       u_fl=(0.9, 0.0, 0.0), x_range=(0, 8))
    sps = [Z.species(-1.0, (4, 4), profile=Z.PROFILE_NONE)]
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07, sps, tile=(8, 8),
                   capacity_slack=0.01, track_ids=True, sort_every=3)
    gpu, orc = H.make_pair(cfg, [ld])
    x0 = H.positions_by_id(orc.species[0].state())
    gpu.step(12)
    orc.step(12)
    assert gpu.info().resorts >= 1 and gpu.info().sorts >= 1
    H.compare_fields(gpu, orc, 1e-4)
    H.compare_particles(gpu, orc, 0, nx, ny, 1e-4, x_ref=x0)


def test_batch_members_with_and_without_resort_match_single_runs():
    cfgs = [W.uniform_thermal(48, 40, ppc=(2, 2), sim_index=0,
                              track_ids=True, sort_every=2),
            W.clouds(64, 32, ppc=(2, 2), sim_index=1, track_ids=True,
                     sort_every=-1)]
    batch = Z.Batch(cfgs)
    singles = [Z.Sim(c) for c in cfgs]
    batch.step(9)
    for s in singles:
        s.step(9)
    for i, c in enumerate(cfgs):
        same_run(batch.sim(i), singles[i], c.n_species)
    assert batch.sim(0).info().sorts == 4 and batch.sim(1).info().sorts == 0


def test_autotune_all_chooses_and_create_uses_it():
    cfg = W.uniform_thermal(256, 256, ppc=(4, 4), track_ids=True)
    t, times = Z.autotune_all(cfg, steps=4)
    stages = {}
    for stage, cand, ms in times:
        stages.setdefault(stage, {})[cand] = ms
    assert set(stages) == {"tile", "ctas_per_sm", "sort_every"}
    ok = {k: v for k, v in stages["tile"].items() if v > 0}
    assert ok[(t.tile_x, t.tile_y)] == min(ok.values())
    ok = {k: v for k, v in stages["ctas_per_sm"].items() if v > 0}
    assert ok[t.push_ctas_per_sm] == min(ok.values())
    ok = {k: v for k, v in stages["sort_every"].items() if v > 0}
    assert ok[t.sort_every] == min(ok.values())
    assert t.ms_per_step == pytest.approx(ok[t.sort_every])
    sim = Z.Sim(cfg)                    # settings left at 0 -> the tuning
    i = sim.info()
    assert (i.tile_x, i.tile_y) == (t.tile_x, t.tile_y)
    assert i.sort_every == t.sort_every
    assert i.push_ctas_per_sm == t.push_ctas_per_sm
    # explicit settings win over the tuning
    sim2 = Z.Sim(W.uniform_thermal(256, 256, ppc=(4, 4), sort_every=7,
                                   push_ctas_per_sm=1))
    assert sim2.info().sort_every == 7 and sim2.info().push_ctas_per_sm == 1


@pytest.mark.parametrize("tile,ppc,prec", [
    ((16, 16), (4, 4), Z.FP32),   # through shared memory
    ((32, 32), (5, 5), Z.FP32),   # 25,600 particles a tile: slot by slot
    ((16, 16), (4, 4), Z.FP64),   # through shared memory, two plane buffers
    ((16, 16), (7, 7), Z.FP64),   # 12,544 particles a tile: one plane buffer
    ((16, 16), (8, 8), Z.FP64),   # 16,384 > the FP64 staging room
])
def test_resort_order_and_whole_records(tile, ppc, prec):
    # both ways of moving a tile's particles give the cell-interleaved order
    # and move every record whole (compared by id with a run that does not
    # re-sort; the FP64 deposit is made order-independent for this)
    nx = ny = 64
    det = prec == Z.FP64

    def make(every):
        return Z.Sim(W.uniform_thermal(nx, ny, ppc=ppc, tile=tile,
                                       precision=prec, track_ids=True,
                                       deterministic=det, sort_every=every))
    a, b = make(-1), make(2)
    a.step(2)
    b.step(2)
    assert b.info().sorts == 1 and a.info().sorts == 0
    ntx = nx // tile[0]
    cnt = b.tile_counts(0)
    for t in (0, ntx + 1):
        st = b.particles(0, tiles=(t, t + 1))
        tx0, ty0 = (t % ntx) * tile[0], (t // ntx) * tile[1]
        lc = (st["iy"] - ty0) * tile[0] + (st["ix"] - tx0)
        assert len(lc) == cnt[t]
        counts = np.bincount(lc, minlength=tile[0] * tile[1])
        want = np.concatenate([np.nonzero(counts > r)[0]
                               for r in range(counts.max())])
        np.testing.assert_array_equal(lc, want)
    pa, pb = a.particles(0), b.particles(0)
    oa = np.argsort(pa["id"], kind="stable")
    ob = np.argsort(pb["id"], kind="stable")
    for k in pa:
        np.testing.assert_array_equal(pa[k][oa], pb[k][ob], err_msg=k)
