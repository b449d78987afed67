"""zpic_batch_autotune through the C ABI: the particle kernel's settings for a
batch of independent simulations as a whole.

The batched sweep advances many simulations of uneven size with one launch
per stage; its tile size, resident CTAs per SM and re-sort interval are
chosen by timing the batch itself (the region-count study of Sec. 4.3, for
a batch instead of one box), and a batch created from the same list uses
them for the settings its members leave at 0.  Without a batch tuning the
members run 16 x 16 tiles, not the per-class choices zpic_autotune makes
for a simulation alone on the GPU."""
import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu


def argmin_ok(stage):
    ok = {k: v for k, v in stage.items() if v > 0}
    return min(ok, key=ok.get)


def test_batch_members_do_not_take_single_simulation_tiles():
    cfgs = W.batch_sweep(P.batch_specs(7))
    for c in cfgs:
        Z.autotune(c, steps=2)          # per-class choices for one sim alone
    b = Z.Batch(cfgs)
    for i, c in enumerate(cfgs):
        inf = b.sim(i).info()
        assert (inf.tile_x, inf.tile_y) == (min(16, c.nx), min(16, c.ny))


def test_batch_autotune_chooses_and_batch_uses_it():
    cfgs = W.batch_sweep(P.batch_specs(6))
    t, times = Z.batch_autotune(cfgs, steps=3)
    stages = {}
    for stage, cand, ms in times:
        stages.setdefault(stage, {})[cand] = ms
    assert set(stages) == {"tile", "ctas_per_sm", "sort_every"}
    assert argmin_ok(stages["tile"]) == (t.tile_x, t.tile_y)
    assert argmin_ok(stages["ctas_per_sm"]) == t.push_ctas_per_sm
    assert argmin_ok(stages["sort_every"]) == t.sort_every
    assert t.ms_per_step == pytest.approx(stages["sort_every"][t.sort_every])

    b = Z.Batch(cfgs)
    for i, c in enumerate(cfgs):
        inf = b.sim(i).info()
        assert (inf.tile_x, inf.tile_y) == (min(t.tile_x, c.nx),
                                            min(t.tile_y, c.ny))
        assert inf.sort_every == t.sort_every
        assert 1 <= inf.push_ctas_per_sm <= t.push_ctas_per_sm

    # a member of the tuned batch still gives the same fields, bit for bit,
    # as the simulation alone at its default settings (the FP32 current is
    # an exact sum, so neither the tile size nor the order of the tiles
    # changes a bit)
    b.step(6)
    for i in (0, 1):
        single = Z.Sim(cfgs[i])
        single.step(6)
        for k in H.FIELDS:
            np.testing.assert_array_equal(b.sim(i).field(k, np.float32),
                                          single.field(k, np.float32),
                                          err_msg="sim %d %s" % (i, k))


def test_batch_autotune_rejects_bad_arguments():
    cfgs = W.batch_sweep(P.batch_specs(2))
    with pytest.raises(Z.ZpicError):
        Z.batch_autotune(cfgs[:1], steps=2)
    with pytest.raises(Z.ZpicError):
        Z.batch_autotune(cfgs, steps=0)
