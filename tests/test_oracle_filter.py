"""Pins of the oracle's current filter (the digital filter on J of Sec. 2.2,
compensated binomial as in the LWFA runs of Sec. 4.1): one binomial pass
(1, 2, 1)/4 and one compensation pass (-1, 6, -1)/4 per axis.

Pinned against closed forms that do not restate the implementation:
Fourier modes are eigenvectors with eigenvalue (1 - sin^4(k/2)) per axis;
a unit impulse spreads into the outer product of the 5-point kernel
(-1, 4, 10, 4, -1)/16 (the convolution of the two passes, worked out by
hand); the total is conserved on a periodic grid; at an open x edge each
pass drops what falls outside, which gives (11, 4, -1)/16 for an impulse in
the first column (worked out by hand, pass by pass).
"""
import numpy as np
import pytest

from oracle import oracle as O

NAMES = ("jx", "jy", "jz")


def filtered(nx, ny, arrays, open_x=False):
    sim = O.Sim(nx, ny, 0.1, 0.1, 0.05, open_x=open_x, filter_j=True)
    for k, a in zip(NAMES, arrays):
        sim.set_field(k, a)
    sim.filter_current()
    return [sim.f[k].copy() for k in NAMES]


@pytest.mark.parametrize("m,l", [(1, 0), (0, 1), (3, 2), (7, 5), (16, 12),
                                 (5, 11)])
def test_fourier_modes_are_eigenvectors(m, l):
    nx, ny = 32, 24
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    kx, ky = 2 * np.pi * m / nx, 2 * np.pi * l / ny
    modes = [np.cos(kx * i + ky * j + ph) for ph in (0.0, 0.7, -1.9)]
    gain = (1 - np.sin(kx / 2) ** 4) * (1 - np.sin(ky / 2) ** 4)
    for got, want in zip(filtered(nx, ny, modes), modes):
        np.testing.assert_allclose(got, gain * want, rtol=0, atol=1e-14)


def test_nyquist_mode_is_removed_and_long_waves_kept():
    nx, ny = 16, 16
    i = np.arange(nx)[None, :] + 0 * np.arange(ny)[:, None]
    nyq = np.cos(np.pi * i)          # k = pi: sin^4 = 1, gain 0
    flat = np.ones((ny, nx))         # k = 0: gain 1
    out = filtered(nx, ny, [nyq, flat, 2.5 * flat])
    np.testing.assert_allclose(out[0], 0.0, atol=1e-15)
    np.testing.assert_allclose(out[1], 1.0, rtol=1e-15)
    np.testing.assert_allclose(out[2], 2.5, rtol=1e-15)


def test_impulse_response_is_the_5_point_kernel_squared():
    nx, ny = 20, 18
    k5 = np.array([-1.0, 4.0, 10.0, 4.0, -1.0]) / 16.0
    for (i0, j0) in [(9, 8), (0, 0), (19, 1)]:   # interior and wrapped
        d = np.zeros((ny, nx))
        d[j0, i0] = 1.0
        want = np.zeros((ny, nx))
        for a in range(5):
            for b in range(5):
                want[(j0 + b - 2) % ny, (i0 + a - 2) % nx] += k5[b] * k5[a]
        for got in filtered(nx, ny, [d, 3.0 * d, -d]):
            scale = got[j0, i0] / want[j0, i0]
            assert scale in (1.0, 3.0, -1.0)
            np.testing.assert_allclose(got, scale * want, rtol=0, atol=1e-15)


def test_total_is_conserved_on_a_periodic_grid():
    rng = np.random.default_rng(7)
    nx, ny = 24, 40
    arrays = [rng.standard_normal((ny, nx)) for _ in range(3)]
    for got, a in zip(filtered(nx, ny, arrays), arrays):
        assert got.sum() == pytest.approx(a.sum(), abs=1e-12)
        assert np.linalg.norm(got) < np.linalg.norm(a)


def test_open_x_edge_drops_what_falls_outside():
    nx, ny = 12, 8
    d = np.zeros((ny, nx))
    d[3, 0] = 1.0                    # impulse in the first column
    got = filtered(nx, ny, [d, d, d], open_x=True)[0]
    edge = np.array([11.0, 4.0, -1.0]) / 16.0
    k5 = np.array([-1.0, 4.0, 10.0, 4.0, -1.0]) / 16.0
    want = np.zeros((ny, nx))
    for b in range(5):
        want[(3 + b - 2) % ny, 0:3] = k5[b] * edge
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    # the far edge is open too: nothing wraps from column 0 to nx - 1
    assert np.all(got[:, nx - 2:] == 0.0)
