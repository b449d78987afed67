"""GPU checks (through the C ABI) of the phase-space report against the
oracle's definition, and of checkpoint / restart: a run interrupted, saved,
restored into a new handle and continued matches the uninterrupted run."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2106_12485_gb300 import workloads as W
from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu


def clouds_pair(precision):
    """GPU sim and oracle on the same seeded cloud-collision load (four
    species, 3 x 3 per cell), every input from the generator."""
    real = np.float64 if precision == Z.FP64 else np.float32
    loads = P.two_clouds(96, 64, 3, 3, drift=0.2, u_th=0.05, dtype=real)
    sps = [Z.species(qm, (3, 3), profile=Z.PROFILE_NONE)
           for qm in (-1.0, 1.0, -1.0, 1.0)]
    cfg = Z.config(96, 64, (9.6, 6.4), 0.07, sps, track_ids=True,
                   precision=precision)
    return H.make_pair(cfg, loads)


CASES = (("x", "ux", (0, 96, -0.6, 0.6), (48, 40)),
         ("x", "y", (0, 96, 0, 64), (96, 64)),
         ("uy", "uz", (-0.2, 0.25, -0.3, 0.3), (17, 9)))


@pytest.mark.parametrize("precision", [Z.FP32, Z.FP64])
def test_phasespace_matches_oracle(precision):
    # the GPU's report of its particles against the oracle's definition on
    # the oracle's particles, both advanced from the same seeded load
    gpu, orc = clouds_pair(precision)
    q0 = 1.0 / 9
    for steps in (0, 7):
        gpu.step(steps)
        orc.step(steps)
        for s in range(4):
            st = orc.species[s].state()
            for qx, qy, rg, bins in CASES:
                got = gpu.phasespace(s, qx, qy, rg, bins)
                want = O.phasespace(st, q0, qx, qy, rg, bins)
                if steps == 0 or precision == Z.FP64:
                    # the same particles (FP64: to 1e-14): every particle
                    # adds exactly 1/9 to the same bin on both sides
                    np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
                    assert np.count_nonzero(got) == np.count_nonzero(want)
                else:
                    # FP32 particles differ from the oracle's by rounding:
                    # at most a few may sit on the other side of a bin edge
                    assert abs(got.sum() - want.sum()) <= 4 * q0 + 1e-9
                    assert np.abs(got - want).sum() <= 8 * q0 + 1e-9
    # charge inside a range that covers everything = particles x |q0|
    n = gpu.num_particles(0)
    tot = gpu.phasespace(0, "x", "y", (0, 96, 0, 64), (1, 1))
    assert tot[0, 0] == pytest.approx(n / 9.0, rel=1e-11)  # n adds of 1/9


def test_phasespace_weighted_window_plasma():
    # the LWFA ramp gives weights < 1 to the injected particles; FP64, so
    # that the GPU's and the oracle's particles agree to rounding
    from tests.test_gpu_workloads import lwfa_pair
    gpu, orc = lwfa_pair(256, 16, 300, Z.FP64)
    gpu.step(300)
    orc.step(300)
    st = orc.species[0].state()
    assert np.any(st["w"] < 1)
    assert gpu.num_particles(0) == orc.species[0].n
    q0 = 1.0 / 4
    for qx, qy, rg, bins in (("x", "ux", (0, 256, -0.5, 0.5), (64, 32)),
                             ("x", "uy", (100, 256, -1, 1), (39, 7))):
        got = gpu.phasespace(0, qx, qy, rg, bins)
        want = O.phasespace(st, q0, qx, qy, rg, bins)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)


def test_phasespace_argument_errors():
    sim = Z.Sim(W.uniform_thermal(32, 32))
    import ctypes as C
    out = np.zeros(16)
    rg = np.array([0.0, 1.0, 0.0, 1.0])
    L = Z.lib()
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    assert L.zpic_phasespace(sim.h, 0, 9, 0, ptr(rg), 4, 4, ptr(out), 16) == Z.EINVAL
    assert L.zpic_phasespace(sim.h, 3, 0, 1, ptr(rg), 4, 4, ptr(out), 16) == Z.EINVAL
    assert L.zpic_phasespace(sim.h, 0, 0, 1, ptr(rg), 0, 4, ptr(out), 16) == Z.EINVAL
    assert L.zpic_phasespace(sim.h, 0, 0, 1, ptr(rg), 4, 4, ptr(out), 15) == Z.ECAP
    bad = np.array([1.0, 1.0, 0.0, 1.0])
    assert L.zpic_phasespace(sim.h, 0, 0, 1, ptr(bad), 4, 4, ptr(out), 16) == Z.EINVAL


def restart_pair(cfg, n_before, n_after, tmp_path):
    ref = Z.Sim(cfg)
    ref.step(n_before + n_after)
    run = Z.Sim(cfg)
    run.step(n_before)
    path = str(tmp_path / "ckpt.npz")
    run.save_checkpoint(path)
    st = run.state()
    del run
    back = Z.load_checkpoint(cfg, path)
    st2 = back.state()
    assert (st2.step, st2.n_shift) == (st.step, st.n_shift)
    assert list(st2.removed) == list(st.removed)
    back.step(n_after)
    return ref, back


@pytest.mark.parametrize("n_before", [12, 13])   # even and odd step parity
def test_restart_continues_the_run(n_before, tmp_path):
    cfg = W.uniform_thermal(64, 48, ppc=(3, 3), track_ids=True, energy_every=4)
    ref, back = restart_pair(cfg, n_before, 9, tmp_path)
    assert back.info().step == ref.info().step == n_before + 9
    # FP32 sums the current exactly (fixed point), so the restored run, whose
    # particles sit in a different order, reproduces the uninterrupted one
    # bit for bit
    for k in H.FIELDS:
        np.testing.assert_array_equal(back.field(k, np.float32),
                                      ref.field(k, np.float32), err_msg=k)
    a, b = H.by_id(back.particles(0)), H.by_id(ref.particles(0))
    for k in ("id", "ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    # the energy history restarts with the restored run
    recs = back.energy()
    assert recs and recs[0][0] > n_before


def test_restart_moving_window_fp64(tmp_path):
    # window shifts, injection and removal counts carry over exactly
    cfg = W.lwfa(nx=256, ny=16, precision=Z.FP64, track_ids=True)
    ref, back = restart_pair(cfg, 151, 60, tmp_path)
    assert back.info().n_shift == ref.info().n_shift > 190
    assert back.num_particles(0) == ref.num_particles(0)
    assert list(back.state().removed) == list(ref.state().removed)
    for k in H.FIELDS:
        assert H.rel_l2(back.field(k), ref.field(k)) < 1e-12, k


def test_set_state_errors():
    import ctypes as C
    sim = Z.Sim(W.uniform_thermal(32, 32))
    st = Z.zpic_state()
    st.step = -1
    assert Z.lib().zpic_set_state(sim.h, C.byref(st)) == Z.EINVAL
    st.step, st.n_shift = 4, -2
    assert Z.lib().zpic_set_state(sim.h, C.byref(st)) == Z.EINVAL
    batch = Z.Batch([W.uniform_thermal(32, 32), W.uniform_thermal(32, 32)])
    st.n_shift = 0
    assert Z.lib().zpic_set_state(batch.sim(0).h, C.byref(st)) == Z.EINVAL
    assert Z.lib().zpic_get_state(sim.h, None) == Z.EINVAL


def test_fp32_runs_are_bitwise_reproducible():
    # the tile currents and their sum over tiles are exact integer sums, so
    # neither the warps' order inside a tile nor the tiles' order changes a
    # bit of the fields or of any particle; a batch member equals the same
    # simulation run alone
    cfg = W.clouds(96, 80, ppc=(3, 3), track_ids=True, energy_every=5)
    runs = [Z.Sim(cfg) for _ in range(2)]
    batch = Z.Batch([W.uniform_thermal(40, 40, sim_index=5), cfg])
    for r in runs:
        r.step(25)
    batch.step(25)
    views = runs + [batch.sim(1)]
    for k in H.FIELDS:
        f0 = views[0].field(k, np.float32)
        for v in views[1:]:
            np.testing.assert_array_equal(v.field(k, np.float32), f0,
                                          err_msg=k)
    for s in range(cfg.n_species):
        p0 = H.by_id(views[0].particles(s))
        for v in views[1:]:
            p = H.by_id(v.particles(s))
            for k in ("id", "ix", "iy", "x", "y", "ux", "uy", "uz"):
                np.testing.assert_array_equal(p[k], p0[k], err_msg=k)
    # field energies come from fixed-order block sums of identical fields
    e0 = views[0].energy()
    for v in views[1:]:
        for a, b in zip(v.energy(), e0):
            assert a[0] == b[0] and a[1] == b[1] and a[2] == b[2]

