"""The allocation-free field-energy entry point (for callers that cannot
allocate device memory when they need the diagnostic, e.g. while a stream
is being captured into a CUDA graph) must give the same energies as the
allocating entry point zpic_field_energy.  This file is named to be
collected last, so a stop-at-first-failure run has run everything else."""
import numpy as np
import pytest

from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P

pytestmark = pytest.mark.gpu

NAMES = ("ex", "ey", "ez", "bx", "by", "bz")


def test_noalloc_energy_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    nx, ny, dx, dy = 96, 70, 0.1, 0.2
    fields = P.random_fields(nx, ny, seed=31, scale=0.8)
    f32 = {k: fields[k].astype(np.float32) for k in NAMES}
    sim = Z.Sim(Z.config(nx, ny, (nx * dx, ny * dy), 0.06, []))
    for k in NAMES:
        sim.set_field(k, f32[k].astype(np.float64))
    ref = np.array(sim.field_energy())
    dev = {k: torch.from_numpy(f32[k]).cuda() for k in NAMES}
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for _ in range(2):          # two calls in a row share the static scratch
        out = np.zeros(2)
        rc = Z.lib().zpic_field_energy_noalloc_f32(
            *[dev[k].data_ptr() for k in NAMES], nx, ny, nx, dx, dy,
            out.ctypes.data, stream)
        assert rc == Z.OK, Z.lib().zpic_last_error()
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0)
    assert ref.min() > 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    a = torch.zeros(4, device="cuda")
    out = np.zeros(2)
    rc = Z.lib().zpic_field_energy_noalloc_f32(
        *([a.data_ptr()] * 6), 2, 65537, 2, 0.1, 0.1, out.ctypes.data, None)
    assert rc == Z.EINVAL
    assert b"65536" in Z.lib().zpic_last_error()
