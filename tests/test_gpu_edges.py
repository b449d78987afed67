"""Edge cases on the GPU against the oracle (through the C ABI): particles
placed on cell faces, at the largest offset below 1, at rest, crossing a
cell corner exactly, crossing the periodic seam, moving near c; an empty
species next to a full one; the smallest grid (4 x 4); the largest
particles per cell the library accepts."""
import numpy as np
import pytest

from paper_2106_12485_gb300 import zpic as Z
from synthetic import plasma as P
from tests import pichelpers as H

pytestmark = pytest.mark.gpu

ONE_M = float(np.nextafter(np.float32(1), np.float32(0)))   # 1 - 2^-24


def crafted(nx, ny, dtype):
    # (ix, iy, x, y, ux, uy, uz)
    rows = [
        (3, 4, 0.0, 0.0, 0.0, 0.0, 0.0),              # at rest on a node
        (5, 5, 0.5, 0.5, 0.0, 0.0, 0.3),              # at rest in x, y
        (6, 2, ONE_M, ONE_M, 0.0, 0.0, 0.0),          # largest offsets
        (7, 7, ONE_M, 0.5, 1e-6, 0.0, 0.0),           # creeps over a face
        (8, 8, 1e-9, 0.5, -1e-7, 0.0, 0.0),           # backward, rounds to 1
        (9, 9, 0.9, 0.9, 0.5, 0.5, 0.0),              # exact corner tie
        (10, 3, 0.1, 0.1, -0.5, -0.5, 0.1),           # corner, backward
        (11, 6, 0.95, 0.05, 0.4, -0.4, 0.0),          # corner, mixed
        (nx - 1, ny - 1, 0.97, 0.97, 0.8, 0.8, 0.0),  # over the seam
        (0, 0, 0.02, 0.03, -0.8, -0.6, 0.0),          # over the seam, back
        (12, 12, 0.5, 0.5, 5.0, 3.0, 2.0),            # gamma ~ 6
        (13, 1, 0.999, 0.001, 7.0, -7.0, 0.0),        # near c, diagonal
        (2, 10, 0.5, 0.0, 0.0, -0.3, 0.0),            # on a face, leaving
        (1, 11, 0.0, 0.5, -0.3, 0.0, 0.0),            # on a face, leaving
    ]
    a = np.array(rows, dtype=np.float64)
    n = len(rows)
    return {"ix": a[:, 0].astype(np.int32), "iy": a[:, 1].astype(np.int32),
            "x": a[:, 2].astype(dtype), "y": a[:, 3].astype(dtype),
            "ux": a[:, 4].astype(dtype), "uy": a[:, 5].astype(dtype),
            "uz": a[:, 6].astype(dtype), "w": np.ones(n, dtype),
            "id": np.arange(n, dtype=np.int32)}


@pytest.mark.parametrize("precision,tol", [(Z.FP32, 1e-4), (Z.FP64, 1e-10)])
def test_crafted_edge_particles_match_oracle(precision, tol):
    nx, ny = 32, 24
    dt = np.float64 if precision == Z.FP64 else np.float32
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07,
                   [Z.species(-1.0, (1, 1), profile=Z.PROFILE_NONE)],
                   precision=precision, track_ids=True)
    ld = crafted(nx, ny, dt)
    fields = P.random_fields(nx, ny, seed=13, scale=0.05)
    gpu, orc = H.make_pair(cfg, [ld], fields=fields)
    for _ in range(3):
        gpu.step(1)
        orc.step(1)
        assert gpu.num_particles(0) == orc.species[0].n == len(ld["ix"])
        H.compare_fields(gpu, orc, tol)
        H.compare_particles(gpu, orc, 0, nx, ny, tol)
    # every stored offset is in [0, 1) and every cell inside the grid
    g = gpu.particles(0)
    assert np.all((g["x"] >= 0) & (g["x"] < 1) & (g["y"] >= 0) & (g["y"] < 1))
    assert np.all((g["ix"] >= 0) & (g["ix"] < nx) & (g["iy"] >= 0) &
                  (g["iy"] < ny))


def face_landings(nx, ny, dtype, d=0.1, dt=0.07,
                  speeds=(0.13, 0.17, 0.21, 0.25, 0.3, 0.34, 0.38, 0.42,
                          0.47, 0.51, 0.55, 0.6)):
    """Particles whose straight path ends within a few units of the last
    place of a cell face, crossing only that face: along y forward (end at
    1 - k ulp .. 1 + k ulp), along y backward (end at -k ulp .. +k ulp), and
    the same along x, for several speeds (so that the quotients of the path
    split round both ways).  u is exact and the fields are zero, so the end
    is start + dt u / (gamma d), which the sweep of start offsets walks
    across the face one unit at a time."""
    one = dtype(1)
    rows = []
    k = 0
    for u0 in speeds:
        c = dtype(dt * u0 / np.sqrt(1.0 + u0 * u0) / d)  # cells per step
        for axis in (0, 1):
            for sign in (1, -1):
                v = dtype(one - c if sign > 0 else c)
                for _ in range(8):               # walk back 8 units
                    v = np.nextafter(v, dtype(0))
                for _ in range(20):
                    ix, iy = k % nx, (k // nx) % ny
                    off = (v, dtype(0.5)) if axis == 0 else (dtype(0.5), v)
                    u = (sign * u0, 0.0) if axis == 0 else (0.0, sign * u0)
                    rows.append((ix, iy, off[0], off[1], u[0], u[1]))
                    v = np.nextafter(v, one)
                    k += 1
    n = len(rows)
    return {"ix": np.array([r[0] for r in rows], np.int32),
            "iy": np.array([r[1] for r in rows], np.int32),
            "x": np.array([r[2] for r in rows], dtype),
            "y": np.array([r[3] for r in rows], dtype),
            "ux": np.array([r[4] for r in rows], dtype),
            "uy": np.array([r[5] for r in rows], dtype),
            "uz": np.zeros(n, dtype), "w": np.ones(n, dtype),
            "id": np.arange(n, dtype=np.int32)}


@pytest.mark.parametrize("precision,tol", [(Z.FP32, 1e-4), (Z.FP64, 1e-10)])
def test_face_landings_within_rounding(precision, tol):
    # a path that crosses one face and ends within rounding of it is split
    # at that face only (the crossing order matters only when both faces
    # are crossed); the current of every particle must match the oracle's
    nx, ny = 48, 40
    dt = np.float64 if precision == Z.FP64 else np.float32
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07,
                   [Z.species(-1.0, (1, 1), profile=Z.PROFILE_NONE)],
                   precision=precision, track_ids=True)
    ld = face_landings(nx, ny, dt)
    gpu, orc = H.make_pair(cfg, [ld])
    gpu.step(1)
    orc.step(1)
    assert gpu.num_particles(0) == orc.species[0].n == len(ld["ix"])
    H.compare_fields(gpu, orc, tol, names=("jx", "jy", "jz"))
    H.compare_particles(gpu, orc, 0, nx, ny, tol)
    g = gpu.particles(0)
    assert np.all((g["x"] >= 0) & (g["x"] < 1) & (g["y"] >= 0) & (g["y"] < 1))


def test_empty_species_next_to_a_full_one():
    nx, ny = 48, 32
    cfg = Z.config(nx, ny, (nx * 0.1, ny * 0.1), 0.07,
                   [Z.species(-1.0, (2, 2), profile=Z.PROFILE_NONE),
                    Z.species(1.0, (2, 2), profile=Z.PROFILE_NONE)],
                   track_ids=True, energy_every=2)
    full = P.plasma_load(nx, ny, 2, 2, u_th=(0.1,) * 3)
    empty = {k: v[:0] for k, v in full.items()}
    gpu, orc = H.make_pair(cfg, [full, empty])
    gpu.step(6)
    orc.step(6)
    assert gpu.num_particles(1) == 0
    H.compare_fields(gpu, orc, 1e-4)
    H.compare_particles(gpu, orc, 0, nx, ny, 1e-4)
    for rec in gpu.energy():
        assert rec[3][1] == 0.0          # no kinetic energy in species 1


def test_smallest_grid_single_particle():
    # 4 x 4 cells (the smallest accepted), one tile of 4 x 4
    nx = ny = 4
    cfg = Z.config(nx, ny, (0.4, 0.4), 0.05,
                   [Z.species(-1.0, (1, 1), profile=Z.PROFILE_NONE)],
                   track_ids=True)
    ld = {"ix": np.array([1], np.int32), "iy": np.array([2], np.int32),
          "x": np.array([0.7], np.float32), "y": np.array([0.95], np.float32),
          "ux": np.array([0.6], np.float32), "uy": np.array([0.9], np.float32),
          "uz": np.array([0.1], np.float32), "w": np.ones(1, np.float32),
          "id": np.zeros(1, np.int32)}
    gpu, orc = H.make_pair(cfg, [ld])
    assert gpu.info().tile_x == 4
    gpu.step(10)
    orc.step(10)
    H.compare_fields(gpu, orc, 1e-4)
    H.compare_particles(gpu, orc, 0, nx, ny, 1e-4)


def test_largest_particles_per_cell():
    # 64 x 64 = 4096 particles per cell (the library's limit) in a 4 x 4
    # box: 65,536 particles in one tile, every current word takes tens of
    # thousands of fixed-point adds per step
    nx = ny = 4
    cfg = Z.config(nx, ny, (0.4, 0.4), 0.07,
                   [Z.species(-1.0, (64, 64), profile=Z.PROFILE_NONE)],
                   track_ids=True)
    ld = P.plasma_load(nx, ny, 64, 64, u_th=(0.2,) * 3)
    gpu, orc = H.make_pair(cfg, [ld])
    gpu.step(4)
    orc.step(4, nthreads=4)
    assert gpu.num_particles(0) == 65536
    H.compare_fields(gpu, orc, 1e-4)
    H.compare_particles(gpu, orc, 0, nx, ny, 1e-4)
    bad = Z.config(nx, ny, (0.4, 0.4), 0.07, [Z.species(-1.0, (65, 64))])
    import ctypes as C
    h = C.c_void_p()
    assert Z.lib().zpic_create(C.byref(bad), C.byref(h)) == Z.EINVAL
