"""The allocation-free field-energy entry point (for callers that cannot
allocate device memory when they need the diagnostic: real-time loops that
must not wait on an allocator, hosts with a fixed memory budget) must give
the same energies as the allocating entry point zpic_field_energy.  This
file is named to be collected last, so a stop-at-first-failure run has run
everything else."""
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


def field_energy_fp64(f32, nx, ny, dx, dy):
    """1/2 sum E^2 dx dy, 1/2 sum B^2 dx dy of the nx x ny interior, FP64."""
    e = sum(np.sum(f32[k][:, :nx].astype(np.float64) ** 2)
            for k in NAMES[:3])
    b = sum(np.sum(f32[k][:, :nx].astype(np.float64) ** 2)
            for k in NAMES[3:])
    return np.array([0.5 * e * dx * dy, 0.5 * b * dx * dy])


def call_noalloc(dev, nx, ny, ld, dx, dy, stream):
    out = np.zeros(2)
    rc = Z.lib().zpic_field_energy_noalloc_f32(
        *[dev[k].data_ptr() for k in NAMES], nx, ny, ld, dx, dy,
        out.ctypes.data, stream)
    assert rc == Z.OK, Z.lib().zpic_last_error()
    return out


def test_noalloc_padded_rows_ignore_the_padding():
    # ld > nx: the padding columns hold large values that must not count
    torch = pytest.importorskip("torch")
    nx, ny, ld, dx, dy = 37, 50, 48, 0.1, 0.15
    rng = np.random.default_rng(4)
    f32 = {k: rng.standard_normal((ny, ld)).astype(np.float32)
           for k in NAMES}
    for k in NAMES:
        f32[k][:, nx:] = 1e6
    dev = {k: torch.from_numpy(f32[k]).cuda() for k in NAMES}
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    ref = field_energy_fp64(f32, nx, ny, dx, dy)
    for _ in range(2):
        np.testing.assert_allclose(call_noalloc(dev, nx, ny, ld, dx, dy,
                                                stream), ref, rtol=1e-12)


def test_noalloc_at_the_largest_row_count():
    # ny = 65536 fills the built-in scratch exactly (the results sit at its
    # last two values); compared with the allocating entry point and FP64
    torch = pytest.importorskip("torch")
    nx, ny, dx, dy = 4, 65536, 0.1, 0.1
    rng = np.random.default_rng(5)
    f32 = {k: rng.standard_normal((ny, nx)).astype(np.float32)
           for k in NAMES}
    sim = Z.Sim(Z.config(nx, ny, (nx * dx, ny * dy), 0.05, []))
    for k in NAMES:
        sim.set_field(k, f32[k].astype(np.float64))
    ref = np.array(sim.field_energy())
    np.testing.assert_allclose(ref, field_energy_fp64(f32, nx, ny, dx, dy),
                               rtol=1e-12)
    dev = {k: torch.from_numpy(f32[k]).cuda() for k in NAMES}
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for _ in range(2):
        np.testing.assert_allclose(call_noalloc(dev, nx, ny, nx, dx, dy,
                                                stream), ref, rtol=1e-12)
