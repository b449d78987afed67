"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the PIC method (no interpolation, push,
deposit or field solve).  It only draws initial particle loads and test
fields, with a counter-based generator so that any subset of cells can be
regenerated on its own:

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): output k >= 1 of a generator seeded with s is
  mix64(s + k * 0x9E3779B97F4A7C15) (mod 2**64), with the mix64 finaliser
  of that paper's reference code.
* key(seed, sim, species) = out_{species+1}(out_{sim+1}(seed)); the d-th draw
  (d = 0..5) of particle k in cell c (c = iy*nx + ix, k < ppc) is
  out_{(c*ppc + k)*8 + d + 1}(key).
* offsets: (z >> 40) * 2**-24, exact in float32 and in [0, 1).
* normals: Box-Muller in float64 on u1 = ((z >> 11) + 1) * 2**-53 and
  u2 = (z >> 11) * 2**-53 (draws 2,3 give n_x, n_y; draws 4,5 give n_z).
* particle id = c*ppc + k (ids are unique per species).
* order: k-major (all cells for k = 0, then k = 1, ...) so that neighbouring
  particles in memory sit in different cells.

The CUDA library implements the same generator for its own initial loads;
a GPU test checks that its loads equal these arrays.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
DEFAULT_SEED = 2106012485


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
    return z ^ (z >> np.uint64(31))


def splitmix_out(state, k):
    """k-th output (k >= 1) of SplitMix64 seeded with `state`."""
    with np.errstate(over="ignore"):
        return mix64(np.asarray(state, np.uint64) +
                     np.asarray(k, np.uint64) * GOLDEN)


def species_key(seed, sim=0, species=0):
    k_sim = splitmix_out(np.uint64(seed), np.uint64(sim + 1))
    return splitmix_out(k_sim, np.uint64(species + 1))


def _offsets(z):
    return ((z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24)


def _normal_pair(za, zb):
    u1 = ((za >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (zb >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    return r * np.cos(th), r * np.sin(th)


def plasma_load(nx, ny, ppc_x, ppc_y, *, seed=DEFAULT_SEED, sim=0, species=0,
                u_th=(0.0, 0.0, 0.0), u_fl=(0.0, 0.0, 0.0), lattice=False,
                x_range=None, dtype=np.float32, cells=None):
    """A uniform load of ppc_x*ppc_y particles per cell.

    x_range = (i0, i1) limits the load to cell columns i0 <= ix < i1 (a slab
    of plasma, e.g. one cloud).  `cells` = array of cell indices c restricts
    the load to those cells (used to regenerate a sample of a large load).
    Offsets are random (draws 0, 1) or on the lattice (k + 1/2)/ppc.
    Momenta are u_fl + u_th * N(0, 1) per axis, rounded to `dtype`.
    Returns a dict of numpy arrays ix, iy, x, y, ux, uy, uz, w, id.
    """
    ppc = ppc_x * ppc_y
    if cells is None:
        i0, i1 = (0, nx) if x_range is None else x_range
        cx = np.arange(i0, i1, dtype=np.int64)
        cy = np.arange(ny, dtype=np.int64)
        cells = (cy[:, None] * nx + cx[None, :]).ravel()
    cells = np.asarray(cells, dtype=np.int64)
    nc = cells.size
    # k-major order
    k = np.repeat(np.arange(ppc, dtype=np.int64), nc)
    c = np.tile(cells, ppc)
    key = species_key(seed, sim, species)
    base = (c * ppc + k).astype(np.uint64) * np.uint64(8)
    one = np.uint64(1)

    def draw(d):
        return splitmix_out(key, base + np.uint64(d) + one)

    if lattice:
        kx, ky = k % ppc_x, k // ppc_x
        x = (kx + 0.5) / ppc_x
        y = (ky + 0.5) / ppc_y
    else:
        x = _offsets(draw(0))
        y = _offsets(draw(1))
    u = np.zeros((3, c.size))
    if any(t != 0.0 for t in u_th):
        nxv, nyv = _normal_pair(draw(2), draw(3))
        nzv, _ = _normal_pair(draw(4), draw(5))
        nrm = (nxv, nyv, nzv)
        for a in range(3):
            u[a] = u_fl[a] + u_th[a] * nrm[a]
    else:
        for a in range(3):
            u[a] = u_fl[a]
    out = {
        "ix": (c % nx).astype(np.int32),
        "iy": (c // nx).astype(np.int32),
        "x": x.astype(dtype), "y": y.astype(dtype),
        "ux": u[0].astype(dtype), "uy": u[1].astype(dtype),
        "uz": u[2].astype(dtype),
        "w": np.ones(c.size, dtype),
        "id": (c * ppc + k).astype(np.int32),
    }
    return out


def concat(*loads):
    return {k: np.concatenate([ld[k] for ld in loads]) for k in loads[0]}


def cloud_ranges(nx):
    """Cell columns of the two clouds: each 25% of the box wide, separated
    by 25% gaps in the periodic box: [nx/8, 3nx/8) and [5nx/8, 7nx/8)."""
    return (nx // 8, 3 * nx // 8), (5 * nx // 8, 7 * nx // 8)


def two_clouds(nx, ny, ppc_x, ppc_y, *, drift, u_th, seed=DEFAULT_SEED,
               sim=0, dtype=np.float32):
    """Collision of plasma clouds: electrons and positrons in each cloud,
    left cloud drifting +drift in x, right cloud -drift.  Returned as four
    loads: (e- left, e+ left, e- right, e+ right), species indices 0..3 of
    the generator key."""
    (a0, a1), (b0, b1) = cloud_ranges(nx)
    th = (u_th, u_th, u_th)
    loads = []
    for s, (rng, d) in enumerate([((a0, a1), drift), ((a0, a1), drift),
                                  ((b0, b1), -drift), ((b0, b1), -drift)]):
        loads.append(plasma_load(nx, ny, ppc_x, ppc_y, seed=seed, sim=sim,
                                 species=s, u_th=th, u_fl=(d, 0.0, 0.0),
                                 x_range=rng, dtype=dtype))
    return loads


def batch_specs(n_sims=256, seed=DEFAULT_SEED):
    """The batched sweep: sim i draws from SplitMix64 stream i:
    nx, ny uniform in [32, 256] rounded to multiples of 8; ppc = k*k with k
    uniform in {2..8}; u_th ~ U(0.01, 0.2); even i uniform thermal plasma,
    odd i two-cloud collision with drift ~ U(0.1, 0.3)."""
    specs = []
    for i in range(n_sims):
        key = splitmix_out(np.uint64(seed), np.uint64(i + 1))
        z = splitmix_out(key, np.arange(1, 7, dtype=np.uint64))
        uni = (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        nx = 32 + 8 * int(uni[0] * 29)        # 32..256 step 8
        ny = 32 + 8 * int(uni[1] * 29)
        k = 2 + int(uni[2] * 7)               # 2..8
        u_th = 0.01 + 0.19 * uni[3]
        drift = 0.1 + 0.2 * uni[4]
        specs.append({"nx": nx, "ny": ny, "ppc_side": k, "u_th": float(u_th),
                      "kind": "thermal" if i % 2 == 0 else "clouds",
                      "drift": float(drift)})
    return specs


def random_fields(nx, ny, seed, scale=1.0):
    """Nine smooth-ish random fields (ex..bz, then zeros for J) for tests."""
    rng = np.random.default_rng(seed)
    out = {}
    for name in ("ex", "ey", "ez", "bx", "by", "bz"):
        out[name] = scale * rng.uniform(-1.0, 1.0, size=(ny, nx))
    return out


def random_particles(nx, ny, n, seed, umax=1.0, dtype=np.float64):
    """n particles anywhere in the box with |u_i| < umax, offsets in [0,1)
    exactly representable in float32."""
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 2 ** 24, n) * 2.0 ** -24
    y = rng.integers(0, 2 ** 24, n) * 2.0 ** -24
    return {
        "ix": rng.integers(0, nx, n).astype(np.int32),
        "iy": rng.integers(0, ny, n).astype(np.int32),
        "x": x.astype(dtype), "y": y.astype(dtype),
        "ux": rng.uniform(-umax, umax, n).astype(dtype),
        "uy": rng.uniform(-umax, umax, n).astype(dtype),
        "uz": rng.uniform(-umax, umax, n).astype(dtype),
        "w": np.ones(n, dtype),
        "id": np.arange(n, dtype=np.int32),
    }
