"""Failure handling, with failures injected on the host (ZPIC_FAULT): no
test here faults, traps or hangs the GPU.  A failed allocation, a failed
launch and a bounded wait that gives up each come back as the documented
status code; the handle stays usable after a launch failure and stays
failed after a timeout."""
import ctypes as C
import os

import numpy as np
import pytest

from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z

pytestmark = pytest.mark.gpu


@pytest.fixture
def fault():
    def set_(kind):
        if kind is None:
            os.environ.pop("ZPIC_FAULT", None)
        else:
            os.environ["ZPIC_FAULT"] = kind
    yield set_
    os.environ.pop("ZPIC_FAULT", None)


def test_allocation_failure(fault):
    cfg = W.uniform_thermal(32, 32)
    h = C.c_void_p()
    fault("alloc")
    assert Z.lib().zpic_create(C.byref(cfg), C.byref(h)) == Z.ENOMEM
    assert b"" != Z.lib().zpic_last_error()
    fault(None)
    sim = Z.Sim(cfg)
    sim.step(2)
    sim.sync()


def test_launch_failure_then_recovery(fault):
    cfg = W.uniform_thermal(32, 32, track_ids=True)
    ref = Z.Sim(cfg)
    ref.step(3)
    sim = Z.Sim(cfg)
    fault("launch")
    assert Z.lib().zpic_step(sim.h, 1) == Z.ECUDA
    assert b"launch" in Z.lib().zpic_last_error().lower()
    fault(None)
    sim.step(3)
    assert sim.info().step == 3
    np.testing.assert_array_equal(sim.field("ex", np.float32),
                                  ref.field("ex", np.float32))
    # the graph path too: a captured graph whose launch is refused
    sim.step(1)
    fault("launch")
    assert Z.lib().zpic_step(sim.h, 2) == Z.ECUDA
    fault(None)
    sim.step(1)
    ref.step(2)
    assert sim.info().step == ref.info().step == 5
    np.testing.assert_array_equal(sim.field("bz", np.float32),
                                  ref.field("bz", np.float32))


def test_timeout_is_sticky(fault):
    sim = Z.Sim(W.uniform_thermal(32, 32))
    sim.step(2)
    fault("timeout")
    assert Z.lib().zpic_sync(sim.h) == Z.ETIMEOUT
    fault(None)
    assert Z.lib().zpic_sync(sim.h) == Z.ETIMEOUT
    assert Z.lib().zpic_step(sim.h, 1) == Z.ETIMEOUT
    assert Z.lib().zpic_strerror(Z.ETIMEOUT)
