"""Pins of the oracle's phase-space report (a diagnostic of Sec. 4.1):
hand-placed particles with bins worked out by hand, the bin edges (low edge
in, high edge out), a lattice load whose per-cell counts are known exactly,
and conservation of the total charge inside the range."""
import numpy as np

from oracle import oracle as O


def state(ix, iy, x, y, ux, uy=None, uz=None, w=None):
    n = len(ix)
    z = np.zeros(n)
    d = {"ix": np.asarray(ix), "iy": np.asarray(iy), "x": np.asarray(x, float),
         "y": np.asarray(y, float), "ux": np.asarray(ux, float),
         "uy": z if uy is None else np.asarray(uy, float),
         "uz": z if uz is None else np.asarray(uz, float)}
    if w is not None:
        d["w"] = np.asarray(w, float)
    return d


def test_hand_placed_particles():
    # x in cells over [0, 8) with 4 bins (2 cells each); ux over [-1, 1)
    # with 2 bins
    st = state(ix=[0, 3, 5, 7], iy=[0, 0, 0, 0], x=[0.5, 0.25, 0.9, 0.999],
               y=[0, 0, 0, 0], ux=[-0.5, 0.2, 0.99, -1.0], w=[1, 2, 1, 3])
    h = O.phasespace(st, -0.25, "x", "ux", (0, 8, -1, 1), (4, 2))
    want = np.zeros((2, 4))
    want[0, 0] += 0.25 * 1   # x 0.5,   ux -0.5
    want[1, 1] += 0.25 * 2   # x 3.25,  ux 0.2
    want[1, 2] += 0.25 * 1   # x 5.9,   ux 0.99
    want[0, 3] += 0.25 * 3   # x 7.999, ux -1.0 (low edge is inside)
    np.testing.assert_array_equal(h, want)


def test_edges_low_in_high_out():
    st = state(ix=[2, 4, 1], iy=[0, 0, 0], x=[0.0, 0.0, 0.0], y=[0, 0, 0],
               ux=[0, 0, 0])
    h = O.phasespace(st, 1.0, "x", "y", (2, 4, 0, 1), (2, 1))
    # x = 2 -> bin 0; x = 4 is the high edge (out); x = 1 is below (out)
    np.testing.assert_array_equal(h, [[1.0, 0.0]])


def test_lattice_load_counts_per_cell():
    nx, ny, px, py = 6, 5, 2, 3
    ix, iy, x, y = [], [], [], []
    for j in range(ny):
        for i in range(nx):
            for a in range(px):
                for b in range(py):
                    ix.append(i)
                    iy.append(j)
                    x.append((a + 0.5) / px)
                    y.append((b + 0.5) / py)
    st = state(ix, iy, x, y, ux=np.zeros(len(ix)))
    q0 = -1.0 / (px * py)
    h = O.phasespace(st, q0, "x", "y", (0, nx, 0, ny), (nx, ny))
    np.testing.assert_allclose(h, np.ones((ny, nx)), rtol=1e-15)
    # half-cell bins split each cell's lattice columns evenly
    h2 = O.phasespace(st, q0, "x", "y", (0, nx, 0, ny), (2 * nx, ny))
    np.testing.assert_allclose(h2, 0.5 * np.ones((ny, 2 * nx)), rtol=1e-15)


def test_total_inside_range_is_conserved():
    rng = np.random.default_rng(3)
    n = 5000
    st = state(ix=rng.integers(0, 10, n), iy=rng.integers(0, 10, n),
               x=rng.random(n), y=rng.random(n), ux=rng.normal(0, 0.3, n),
               uz=rng.normal(0, 0.3, n), w=rng.random(n))
    h = O.phasespace(st, 0.5, "ux", "uz", (-5, 5, -5, 5), (37, 23))
    assert abs(h.sum() - 0.5 * st["w"].sum()) < 1e-10
