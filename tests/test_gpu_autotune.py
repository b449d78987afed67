"""The host tile-size autotuner through the C ABI: every candidate is timed
on the reduced configuration, the fastest is returned and cached for the
configuration's class, and a configuration that asks for tile size 0 gets
it; the tuned run still matches an untuned one step for step."""
import ctypes as C

import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z

pytestmark = pytest.mark.gpu


def test_autotune_picks_the_fastest_candidate_and_create_uses_it():
    cfg = W.uniform_thermal(96, 80, ppc=(3, 3), track_ids=True)
    bx, by, times = Z.autotune(cfg, steps=4)
    assert (bx, by) in times
    ok = {k: v for k, v in times.items() if v > 0}
    assert len(ok) >= 5                      # all tile sizes fit this case
    assert ok[(bx, by)] == min(ok.values())
    # cached for the class: no timing the second time
    bx2, by2, t2 = Z.autotune(cfg, retune=False)
    assert (bx2, by2) == (bx, by) and t2 == {}
    sim = Z.Sim(cfg)                          # tile 0 -> the tuned size
    i = sim.info()
    assert (i.tile_x, i.tile_y) == (min(bx, 96), min(by, 80))
    # results do not depend on the tile size (exact fixed-point current)
    ref = Z.Sim(W.uniform_thermal(96, 80, ppc=(3, 3), track_ids=True,
                                  tile=(16, 16)))
    sim.step(5)
    ref.step(5)
    for k in ("ex", "by", "jz"):
        np.testing.assert_array_equal(sim.field(k, np.float32),
                                      ref.field(k, np.float32))


def test_autotune_reduces_large_and_window_configurations():
    # a 4096 x 512 laser-wakefield class is tuned on a 1024 x 512 copy with
    # the laser and the plasma ramp at the same distance from the edge
    bx, by, times = Z.autotune(W.lwfa(), steps=3)
    assert (bx, by) in times and times[(bx, by)] > 0


def test_autotune_errors():
    bx, by = C.c_int(), C.c_int()
    cfg = W.uniform_thermal(32, 32)
    assert Z.lib().zpic_autotune(C.byref(cfg), 0, C.byref(bx), C.byref(by),
                                 None, 0, None) == Z.EINVAL
    assert Z.lib().zpic_autotune(None, 3, C.byref(bx), C.byref(by), None, 0,
                                 None) == Z.EINVAL
