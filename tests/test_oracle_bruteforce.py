"""Pin of the whole oracle step against the 50-digit brute force
(tests/bruteforce_pic.py), which restates every stage in a different form.

Two particles on an 8x8 grid with random initial fields, chosen to cross x
faces, y faces, a corner (both in one step), and the periodic seam; five
steps.  Positions and every field must agree to 1e-13 (relative to the
largest value of each field).  A second case uses the open-x boundary.
"""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import oracle as O  # noqa: E402
from synthetic import plasma as P  # noqa: E402
from tests.bruteforce_pic import BruteSim  # noqa: E402

NAMES = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")


def run_case(open_x, parts, nsteps=5, nx=8, ny=8, dx=0.1, dy=0.12, dt=0.06):
    fields = P.random_fields(nx, ny, seed=11, scale=0.3)
    bs = BruteSim(nx, ny, dx, dy, dt, open_x=open_x)
    for k, v in fields.items():
        bs.f[k] = [[mp.mpf(float(v[j, i])) for i in range(nx)]
                   for j in range(ny)]
    species = []
    for (ix, iy, x, y, u, qm, q0) in parts:
        species.append(O.Species(qm, q0, [ix], [iy], [x], [y], [u[0]], [u[1]],
                                 [u[2]]))
        bs.p.append({"X": (ix + mp.mpf(x)) * bs.dx, "Y": (iy + mp.mpf(y)) * bs.dy,
                     "u": [mp.mpf(c) for c in u], "q": mp.mpf(q0),
                     "qm": mp.mpf(qm)})
    sim = O.Sim(nx, ny, dx, dy, dt, open_x=open_x, species=species)
    for k, v in fields.items():
        sim.set_field(k, v)
    for _ in range(nsteps):
        sim.step()
        bs.step()
        for k in NAMES:
            ref = np.array([[float(c) for c in row] for row in bs.f[k]])
            scale = max(np.abs(ref).max(), 1e-300)
            np.testing.assert_allclose(sim.f[k], ref, rtol=0,
                                       atol=1e-13 * scale, err_msg=k)
        alive = [p for p in species if p.n > 0]
        assert len(alive) == len(bs.p)
        for sp, bp in zip(alive, bs.p):
            st = sp.state()
            X = (st["ix"][0] + st["x"][0]) * dx
            Y = (st["iy"][0] + st["y"][0]) * dy
            assert X == pytest.approx(float(bp["X"]), abs=1e-13)
            assert Y == pytest.approx(float(bp["Y"]), abs=1e-13)
            np.testing.assert_allclose([st["ux"][0], st["uy"][0], st["uz"][0]],
                                       [float(c) for c in bp["u"]],
                                       rtol=0, atol=1e-13)


def test_bruteforce_two_particles_periodic():
    parts = [
        # fast diagonal mover near a corner: corner crossing in step 1,
        # periodic seam in x and y
        (7, 7, 0.9, 0.85, (2.5, 2.0, 0.4), -1.0, -0.5),
        # slower positron crossing x faces backwards
        (2, 4, 0.1, 0.5, (-0.8, 0.15, -0.3), 1.0, 0.5),
    ]
    run_case(False, parts)


def test_bruteforce_open_x_particle_leaves():
    parts = [
        (0, 3, 0.3, 0.4, (-1.5, 0.3, 0.2), -1.0, -0.5),   # leaves at x = 0
        (4, 3, 0.5, 0.5, (0.6, -0.9, 0.0), -1.0, -0.5),
    ]
    run_case(True, parts)
