"""Pins of the FP64 oracle against closed forms and invariants.

Each test fixes a part of the oracle against something other than itself,
chosen so that a plausible slip (a dropped term, a wrong sign, a wrong
half-cell shift, a swapped component) fails at least one of them:

* gather ............ exact reproduction of linear fields (stagger offsets)
* Boris, uniform B .. |u| conserved, exact rotation angle 2 atan(..), orbit
                      polygon inscribed in a circle, textbook gyroradius limit
* Boris, uniform E .. u_n = u_0 + n (q/m) E dt, x = sum dt u/gamma,
                      hyperbolic motion to O(dt^2)
* Yee ............... numerical dispersion relation of a standing mode (TM
                      and TE, dx != dy)
* coupling .......... cold plasma oscillation recurrence at w_p
* deposit ........... continuity residual at roundoff (random particles,
                      corner crossings, edge rounding), Jz path average vs
                      quadrature
* laser ............. pulse moves in +x at the group velocity, peak E0
* moving window ..... exact one-cell shift, injected counts
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from synthetic import plasma as P


def make_species(ld, qm, q0, cap=None):
    return O.Species(qm, q0, ld["ix"], ld["iy"], ld["x"], ld["y"], ld["ux"],
                     ld["uy"], ld["uz"], w=ld.get("w"), ids=ld.get("id"),
                     cap=cap)


def one_particle(ix, iy, x, y, u, qm=-1.0, q0=-1.0):
    return O.Species(qm, q0, [ix], [iy], [x], [y], [u[0]], [u[1]], [u[2]])


# ---------------------------------------------------------------- gather --

def test_gather_reproduces_linear_fields():
    nx, ny, dx, dy = 12, 10, 0.3, 0.2
    sim = O.Sim(nx, ny, dx, dy, 0.05)
    stag = {"ex": (0.5, 0), "ey": (0, 0.5), "ez": (0, 0), "bx": (0, 0.5),
            "by": (0.5, 0), "bz": (0.5, 0.5)}
    coef = {}
    rng = np.random.default_rng(1)
    for name, (sx, sy) in stag.items():
        a, b, c = rng.uniform(-2, 2, 3)
        coef[name] = (a, b, c)
        i = np.arange(nx)[None, :]
        j = np.arange(ny)[:, None]
        sim.set_field(name, a + b * (i + sx) * dx + c * (j + sy) * dy)
    # particles away from the periodic seam, offsets on both sides of 1/2
    for _ in range(200):
        ix, iy = rng.integers(2, nx - 3), rng.integers(2, ny - 3)
        x, y = rng.uniform(0, 1, 2)
        E, B = sim.gather(int(ix), int(iy), x, y)
        X, Y = (ix + x) * dx, (iy + y) * dy
        got = dict(zip(("ex", "ey", "ez"), E))
        got.update(zip(("bx", "by", "bz"), B))
        for name, (a, b, c) in coef.items():
            assert got[name] == pytest.approx(a + b * X + c * Y, abs=1e-12)


def test_gather_uniform_field_any_position_periodic():
    sim = O.Sim(6, 5, 0.1, 0.1, 0.05)
    vals = [0.3, -1.2, 2.5, 0.7, -0.4, 1.1]
    for name, v in zip(("ex", "ey", "ez", "bx", "by", "bz"), vals):
        sim.set_field(name, np.full((5, 6), v))
    for ix, iy, x, y in [(0, 0, 0.0, 0.0), (5, 4, 0.999, 0.999),
                         (0, 4, 0.25, 0.75), (5, 0, 0.5, 0.5)]:
        E, B = sim.gather(ix, iy, x, y)
        np.testing.assert_allclose(np.r_[E, B], vals, atol=1e-14)


# ---------------------------------------------------------------- Boris --

@pytest.mark.parametrize("qm", [-1.0, 1.0, -2.5])
def test_boris_uniform_B_rotation_and_orbit(qm):
    nx = ny = 64
    dx = dy = 0.1
    dt = 0.07
    B0 = 0.8
    sim = O.Sim(nx, ny, dx, dy, dt)
    sim.set_field("bz", np.full((ny, nx), B0))
    u0 = np.array([0.3, -0.2, 0.0])
    sp = one_particle(32, 32, 0.5, 0.5, u0, qm=qm, q0=np.sign(qm))
    sim = O.Sim(nx, ny, dx, dy, dt, species=[sp])
    sim.set_field("bz", np.full((ny, nx), B0))
    gam = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(abs(qm) * B0 * dt / (2 * gam))
    sense = -np.sign(qm)        # rotation sense about +z
    pos, us = [], []
    X = np.array([32.5 * dx, 32.5 * dy])
    for n in range(120):
        sim.push_deposit(0, do_deposit=False)
        st = sp.state()
        u = np.array([st["ux"][0], st["uy"][0], st["uz"][0]])
        us.append(u)
        Xn = np.array([(st["ix"][0] + st["x"][0]) * dx,
                       (st["iy"][0] + st["y"][0]) * dy])
        # unwrap across the periodic box
        L = np.array([nx * dx, ny * dy])
        Xn = Xn + L * np.round((X - Xn) / L)
        pos.append(Xn)
        X = Xn
    us = np.array(us)
    pos = np.array(pos)
    # |u| conserved to roundoff
    np.testing.assert_allclose(np.linalg.norm(us, axis=1),
                               np.linalg.norm(u0), rtol=1e-14)
    # exact rotation by theta per step
    ang0 = math.atan2(u0[1], u0[0])
    for n in (0, 7, 59, 119):
        expect = ang0 + sense * theta * (n + 1)
        got = math.atan2(us[n][1], us[n][0])
        d = (got - expect + math.pi) % (2 * math.pi) - math.pi
        assert abs(d) < 1e-12
    # positions on a circle of radius R = (|u|/gamma) dt / (2 sin(theta/2))
    R = (np.linalg.norm(u0) / gam) * dt / (2 * math.sin(theta / 2))
    a, b, c = pos[10], pos[40], pos[70]
    # circumcentre of three vertices
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux_ = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) +
           (c @ c) * (a[1] - b[1])) / d
    uy_ = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) +
           (c @ c) * (b[0] - a[0])) / d
    r = np.linalg.norm(pos - np.array([ux_, uy_]), axis=1)
    np.testing.assert_allclose(r, R, rtol=1e-9)
    # textbook gyroradius |u_perp| / (|q/m| B) is the dt -> 0 limit
    assert R == pytest.approx(np.linalg.norm(u0) / (abs(qm) * B0),
                              rel=dt ** 2)


def test_boris_uniform_E_exact_momentum_and_position():
    qm, dt, d = -1.0, 0.05, 0.1
    E = np.array([0.4, -0.25, 0.1])
    u0 = np.array([0.1, 0.0, -0.3])
    nx = ny = 4000
    sp = one_particle(2000, 2000, 0.5, 0.5, u0, qm=qm, q0=-1.0)
    sim = O.Sim(nx, ny, d, d, dt, species=[sp])
    for k, v in zip(("ex", "ey", "ez"), E):
        sim.set_field(k, np.full((ny, nx), v))
    X = np.array([2000.5 * d, 2000.5 * d])
    for n in range(1, 300):
        sim.push_deposit(0, do_deposit=False)
        st = sp.state()
        u = np.array([st["ux"][0], st["uy"][0], st["uz"][0]])
        # u_n = u_0 + n (q/m) E dt, to roundoff
        np.testing.assert_allclose(u, u0 + n * qm * E * dt, rtol=0,
                                   atol=4e-16 * n)
        # x_n = x_{n-1} + dt u_n / gamma_n
        X = X + dt * u[:2] / math.sqrt(1 + u @ u)
        got = np.array([(st["ix"][0] + st["x"][0]) * d,
                        (st["iy"][0] + st["y"][0]) * d])
        np.testing.assert_allclose(got, X, rtol=0, atol=1e-11)


def _hyperbolic_error(dt, T=4.0):
    """Uniform E along x from rest: x(t) = (gamma(t) - 1)/(|q/m| E),
    u(t) = q/m E t.  Returns |x_num - x_exact| at t = T."""
    qm, E0 = 1.0, 0.5
    nx, ny, d = 400, 4, 0.1
    sp = one_particle(10, 1, 0.0, 0.5, [0.0, 0.0, 0.0], qm=qm, q0=1.0)
    sim = O.Sim(nx, ny, d, d, dt, species=[sp])
    sim.set_field("ex", np.full((ny, nx), E0))
    # leapfrog: u starts at t = -dt/2; from rest at t=0 -> u(-dt/2)
    sp.uy[0] = 0.0
    sp.ux[0] = -qm * E0 * dt / 2
    steps = int(round(T / dt))
    for _ in range(steps):
        sim.push_deposit(0, do_deposit=False)
    st = sp.state()
    X = (st["ix"][0] + st["x"][0]) * d - 10 * d
    g = math.sqrt(1 + (qm * E0 * T) ** 2)
    return abs(X - (g - 1) / (qm * E0))


def test_boris_uniform_E_hyperbolic_motion_second_order():
    e1 = _hyperbolic_error(0.04)
    e2 = _hyperbolic_error(0.02)
    assert e1 < 1e-3
    assert 3.3 < e1 / e2 < 4.7     # O(dt^2)


# ------------------------------------------------------------------ Yee --

@pytest.mark.parametrize("mode", ["TM", "TE"])
def test_yee_vacuum_dispersion(mode):
    nx, ny, dx, dy, dt = 32, 24, 0.1, 0.15, 0.06
    mx, my = 3, 2
    kx, ky = 2 * math.pi * mx / (nx * dx), 2 * math.pi * my / (ny * dy)
    sim = O.Sim(nx, ny, dx, dy, dt)
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    if mode == "TM":   # Ez(i, j) standing wave, B = 0
        f0 = np.cos(kx * i * dx) * np.cos(ky * j * dy)
        sim.set_field("ez", f0)
        name = "ez"
    else:              # Bz(i+1/2, j+1/2) standing wave, E = 0
        f0 = np.cos(kx * (i + 0.5) * dx) * np.cos(ky * (j + 0.5) * dy)
        sim.set_field("bz", f0)
        name = "bz"
    s = math.sqrt((math.sin(kx * dx / 2) / dx) ** 2 +
                  (math.sin(ky * dy / 2) / dy) ** 2)
    theta = 2 * math.asin(s * dt)          # omega dt
    N = 300
    for _ in range(N):
        sim.yee()
    np.testing.assert_allclose(sim.f[name], math.cos(N * theta) * f0,
                               atol=1e-11)
    # the continuum frequency differs: the test is sensitive to the stencil
    omega_c = math.hypot(kx, ky)
    assert abs(math.cos(N * omega_c * dt) - math.cos(N * theta)) > 1e-3


# ----------------------------------------------------- plasma oscillation --

def test_cold_plasma_oscillation_frequency():
    nx = ny = 8
    dx = dy = 0.2
    dt = 0.1
    eps = 1e-4
    ld = P.plasma_load(nx, ny, 2, 2, lattice=True, dtype=np.float64)
    ld["ux"][:] = eps
    sp = make_species(ld, qm=-1.0, q0=-1.0 / 4)
    sim = O.Sim(nx, ny, dx, dy, dt, species=[sp])
    ex = []
    for _ in range(400):
        sim.step()
        ex.append(sim.f["ex"].copy())
    ex = np.array(ex)
    # E_x uniform in space, no Ey
    assert np.ptp(ex, axis=(1, 2)).max() < 1e-12 * np.abs(ex).max()
    assert np.abs(sim.f["ey"]).max() < 1e-15
    e = ex[:, 0, 0]
    # leapfrog oscillator at w_p = 1: E_{n+1} + E_{n-1} = 2 cos(w dt) E_n
    # with sin(w dt / 2) = w_p dt / 2  (relativistic correction ~ eps^2)
    c = 1 - dt ** 2 / 2
    res = e[2:] + e[:-2] - 2 * c * e[1:-1]
    assert np.abs(res).max() < 1e-6 * np.abs(e).max()
    w = 2 * math.asin(dt / 2) / dt
    # the period from the zero crossings matches to < 0.1 %
    zc = np.where(np.sign(e[:-1]) != np.sign(e[1:]))[0]
    frac = zc + e[zc] / (e[zc] - e[zc + 1])
    period = 2 * (frac[-1] - frac[0]) / (len(frac) - 1) * dt
    assert period == pytest.approx(2 * math.pi / w, rel=1e-3)


# ------------------------------------------------------------ deposition --

def cic_density(nx, ny, st, q0, open_x=False):
    """rho at nodes from the tent weights (written here, independently)."""
    rho = np.zeros((ny, nx))
    for ix, iy, x, y, w in zip(st["ix"], st["iy"], st["x"], st["y"], st["w"]):
        for di, wx in ((0, 1 - x), (1, x)):
            for dj, wy in ((0, 1 - y), (1, y)):
                i, j = ix + di, (iy + dj) % ny
                if open_x and not (0 <= i < nx):
                    continue
                rho[j, i % nx] += q0 * w * wx * wy
    return rho


def continuity_residual(sim, nx, ny, dx, dy, dt, rho0, rho1):
    jx, jy = sim.f["jx"], sim.f["jy"]
    div = (jx - np.roll(jx, 1, axis=1)) / dx + (jy - np.roll(jy, 1, axis=0)) / dy
    drho = (rho1 - rho0) / dt
    return np.linalg.norm(drho + div) / np.linalg.norm(drho)


def test_continuity_random_particles():
    nx, ny, dx, dy, dt = 16, 12, 0.1, 0.13, 0.07
    ld = P.random_particles(nx, ny, 3000, seed=7, umax=4.0)
    # hand-made edge cases: corners, faces, backward rounding onto a face
    extra = [
        (3, 3, 0.999, 0.999, 2.0, 2.0), (4, 4, 0.0, 0.0, -2.0, -2.0),
        (5, 5, 0.0, 0.5, -1e-20, 0.0), (6, 6, 0.5, 0.0, 0.0, -1e-20),
        (0, 0, 0.01, 0.01, -3.0, -3.0), (nx - 1, ny - 1, 0.99, 0.99, 3, 3),
        (7, 7, 0.9, 0.1, 3.0, -3.0), (8, 2, 0.5, 0.5, 0.0, 0.0),
    ]
    for k, v in enumerate(("ix", "iy", "x", "y", "ux", "uy")):
        ld[v] = np.concatenate([ld[v], np.array([e[k] for e in extra],
                                                 dtype=ld[v].dtype)])
    for v in ("uz", "w"):
        ld[v] = np.concatenate([ld[v], np.full(len(extra), 0.5 if v == "uz" else 1.0)])
    ld["id"] = np.arange(len(ld["ix"]), dtype=np.int32)
    sp = make_species(ld, qm=-1.0, q0=-0.01)
    sim = O.Sim(nx, ny, dx, dy, dt, species=[sp])
    for k, v in P.random_fields(nx, ny, seed=3, scale=0.5).items():
        sim.set_field(k, v)
    rho0 = cic_density(nx, ny, sp.state(), sp.q0)
    for k in ("jx", "jy", "jz"):
        sim.f[k][...] = 0
    sim.push_deposit(0)
    rho1 = cic_density(nx, ny, sp.state(), sp.q0)
    assert continuity_residual(sim, nx, ny, dx, dy, dt, rho0, rho1) < 1e-13
    st = sp.state()
    assert (st["x"] >= 0).all() and (st["x"] < 1).all()
    assert (st["y"] >= 0).all() and (st["y"] < 1).all()


def test_backward_rounding_onto_face_stays_in_cell():
    sp = one_particle(5, 5, 0.0, 0.5, [-1e-20, 0.0, 0.0])
    sim = O.Sim(10, 10, 0.1, 0.1, 0.07, species=[sp])
    sim.push_deposit(0)
    st = sp.state()
    assert (st["ix"][0], st["x"][0]) == (5, 0.0)


def test_jz_path_average_matches_quadrature():
    nx = ny = 8
    dx, dy, dt = 0.1, 0.1, 0.07
    u = np.array([0.9, -0.7, 0.6])      # crosses an x and a y face
    sp = one_particle(3, 4, 0.8, 0.15, u, qm=-1, q0=-1)
    sim = O.Sim(nx, ny, dx, dy, dt, species=[sp])
    sim.push_deposit(0)
    g = math.sqrt(1 + u @ u)
    v = u / g
    X0, Y0 = 3.8 * dx, 4.15 * dy
    N = 100000
    t = (np.arange(N) + 0.5) / N * dt
    cx, cy = (X0 + v[0] * t) / dx, (Y0 + v[1] * t) / dy
    jz = np.zeros((ny, nx))
    for i in range(2, 6):
        for j in range(2, 7):
            wx = np.clip(1 - np.abs(cx - i), 0, None)
            wy = np.clip(1 - np.abs(cy - j), 0, None)
            jz[j, i] = -1 * v[2] * np.mean(wx * wy)
    np.testing.assert_allclose(sim.f["jz"], jz, atol=1e-9)
    assert np.abs(jz).max() > 0.05


def test_threaded_deposit_matches_serial():
    nx, ny = 32, 32
    ld = P.plasma_load(nx, ny, 4, 4, u_th=(0.3, 0.3, 0.3), dtype=np.float64)
    res = []
    for nt in (1, 4):
        sp = make_species(ld, qm=-1.0, q0=-1 / 16)
        sim = O.Sim(nx, ny, 0.1, 0.1, 0.07, species=[sp])
        for _ in range(3):
            sim.step(nthreads=nt)
        res.append((sim.f["ez"].copy(), sp.state()["x"]))
    np.testing.assert_allclose(res[0][0], res[1][0], atol=1e-13)
    np.testing.assert_allclose(res[0][1], res[1][1], rtol=0, atol=1e-13)


# ---------------------------------------------------------------- energy --

def test_energy_bounded_thermal_plasma():
    """Energy drift is not pinned (O(dt^2) scheme): record that it stays
    small for the 64x64-class thermal plasma over 50 steps."""
    nx = ny = 32
    ld = P.plasma_load(nx, ny, 4, 4, u_th=(0.1, 0.1, 0.1), dtype=np.float64)
    sp = make_species(ld, qm=-1.0, q0=-1 / 16)
    sim = O.Sim(nx, ny, 0.1, 0.1, 0.07, species=[sp])
    tot = []
    for _ in range(50):
        _, wE, wB, kin = sim.step()
        tot.append(wE + wB + kin.sum())
    tot = np.array(tot)
    kin0 = sim.history[0][3].sum()
    assert np.abs(tot - tot[0]).max() / tot[0] < 2e-2
    assert kin0 == pytest.approx(
        nx * ny * 0.01 * 0.5 * 3 * 0.01, rel=0.05)  # ~ n m u_th^2 * 3/2 * area


def test_field_energy_closed_form():
    """W_E = 1/2 sum E^2 dx dy and W_B = 1/2 sum B^2 dx dy over the cells,
    every component counted: a uniform component, a single cell of another
    and a single negative cell of the third, with dx != dy."""
    nx, ny, dx, dy = 6, 5, 0.3, 0.2
    sim = O.Sim(nx, ny, dx, dy, 0.1)
    z = np.zeros((ny, nx))
    ey, ez, bz = z.copy(), z.copy(), z.copy()
    ey[1, 2] = 2.0
    ez[4, 5] = -3.0
    bz[0, 0] = 4.0
    for k, v in (("ex", np.ones((ny, nx))), ("ey", ey), ("ez", ez),
                 ("bx", np.full((ny, nx), 0.5)), ("by", z), ("bz", bz)):
        sim.set_field(k, v)
    wE, wB = sim.field_energy()
    assert wE == pytest.approx(0.5 * (nx * ny * 1.0 + 4.0 + 9.0) * dx * dy,
                               rel=1e-15)
    assert wB == pytest.approx(0.5 * (nx * ny * 0.25 + 16.0) * dx * dy,
                               rel=1e-15)


def test_kinetic_energy_closed_form():
    """K_s = sum m_p (gamma - 1) dx dy with m_p = q_p / (q/m) and gamma of
    the momentum after the push; with no fields the push leaves u as it
    is, so hand-picked momenta give exact values: u = (3/4, 0, 0) has
    gamma - 1 = 1/4, u = (0, 0.6, 0.8) has gamma = sqrt 2.  Two species with
    different q0, q/m and weights are kept apart."""
    dx, dy = 0.25, 0.5
    a = O.Species(-2.0, -0.5, [1, 3], [2, 0], [0.5, 0.25], [0.5, 0.75],
                  [0.75, 0.0], [0.0, 0.6], [0.0, 0.8], w=[1.0, 2.0])
    b = O.Species(1.0, 0.125, [2], [1], [0.5], [0.5], [0.0], [0.0], [0.75])
    sim = O.Sim(8, 4, dx, dy, 0.05, species=[a, b])
    _, wE, wB, kin = sim.step()
    # m_p: 0.5 * 1 / 2 = 0.25 and 0.5 * 2 / 2 = 0.5; 0.125 / 1
    assert kin[0] == pytest.approx((0.25 * 0.25 + 0.5 * (np.sqrt(2) - 1))
                                   * dx * dy, rel=1e-14)
    assert kin[1] == pytest.approx(0.125 * 0.25 * dx * dy, rel=1e-14)


# ----------------------------------------------------------------- laser --

def test_laser_propagates_forward_at_group_velocity():
    nx, ny = 1200, 32
    dx, dy, dt = 0.02, 0.2, 0.019
    sim = O.Sim(nx, ny, dx, dy, dt, open_x=True)
    a0, w0l, W0, fwhm = 2.0, 10.0, 4.0, 2.0
    x0, yc = 10.0, ny * dy / 2
    sim.laser(a0, w0l, W0, fwhm, x0, yc)
    # peak field a0*omega0 on the axis, at the node x0 = 500 dx
    row = sim.f["ey"][ny // 2 - 1]   # Ey(j+1/2) nearest yc
    yrow = (ny // 2 - 1 + 0.5) * dy
    assert np.abs(row).max() == pytest.approx(
        a0 * w0l * math.exp(-((yrow - yc) / W0) ** 2), rel=1e-12)
    xs = np.arange(nx) * dx

    def centroid():
        e2 = (sim.f["ey"] ** 2).sum(axis=0)
        return (xs * e2).sum() / e2.sum()

    c0 = centroid()
    n = 300
    for _ in range(n):
        sim.yee()
    v = (centroid() - c0) / (n * dt)
    assert 0.97 < v < 1.0


# --------------------------------------------------------- moving window --

def test_window_shift_exact():
    nx, ny, dx, dt = 20, 6, 0.02, 0.019
    ld = P.plasma_load(nx, ny, 2, 2, lattice=True, dtype=np.float64)
    sp = make_species(ld, qm=-1.0, q0=-0.25, cap=len(ld["ix"]) + 1000)
    win = {"species": [{"ppc_x": 2, "ppc_y": 2, "ramp_x0": 0.0,
                        "ramp_len": 0.0, "n0": 1.0, "id_base": 10 ** 6}]}
    sim = O.Sim(nx, ny, dx, 0.2, dt, open_x=True, species=[sp], window=win)
    rng = np.random.default_rng(0)
    for k in ("ex", "ey", "ez", "bx", "by", "bz"):
        sim.set_field(k, rng.normal(size=(ny, nx)))
    before = {k: sim.f[k].copy() for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    st0 = sp.state()
    from oracle.oracle import lib
    import ctypes as C
    # step index 0: (0+1)*0.019 < 1*0.02 -> no shift; step 1 -> shift
    assert lib().orc_window_shift(C.byref(sim.g), C.byref(sim.fc),
                                  C.byref(sim.win), 1, sim.sc, 0) == 0
    assert lib().orc_window_shift(C.byref(sim.g), C.byref(sim.fc),
                                  C.byref(sim.win), 1, sim.sc, 1) == 1
    for k, v in before.items():
        np.testing.assert_array_equal(sim.f[k][:, :-1], v[:, 1:])
        np.testing.assert_array_equal(sim.f[k][:, -1], 0.0)
    st1 = sp.state()
    kept = st0["ix"] >= 1
    assert sp.n == kept.sum() + ny * 4
    np.testing.assert_array_equal(st1["ix"][:kept.sum()], st0["ix"][kept] - 1)
    inj = st1["ix"][kept.sum():]
    assert (inj == nx - 1).all()
    assert sorted(st1["id"][kept.sum():]) == list(range(10 ** 6, 10 ** 6 + ny * 4))
