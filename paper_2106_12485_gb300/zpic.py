"""Thin ctypes binding of the C ABI in include/zpic.h.

Argument marshalling only: every step of the PIC method runs in the CUDA
library (_lib/libzpic.so).  If the library is missing the import of this
module still works, but any call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libzpic.so")

MAX_SPECIES = 8
OK, EINVAL, ECFL, ENOMEM, ECUDA, EOVERFLOW, ENAN, ETIMEOUT, ECAP, ENOTSUP = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9)
FP32, FP64 = 0, 1
BC_PERIODIC, BC_OPEN = 0, 1
EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
EB_NAMES = ("ex", "ey", "ez", "bx", "by", "bz")
FIELD_IDS = {"ex": EX, "ey": EY, "ez": EZ, "bx": BX, "by": BY, "bz": BZ,
             "jx": JX, "jy": JY, "jz": JZ}
PROFILE_NONE, PROFILE_UNIFORM, PROFILE_SLAB, PROFILE_RAMP = 0, 1, 2, 3
TRACK_IDS = 1
FILTER_J = 2
DETERMINISTIC = 4
PUSH_GENERIC, PUSH_PLAIN_PERIODIC, PUSH_PLAIN_OPEN = 1, 2, 4


class zpic_species(C.Structure):
    _fields_ = [("q_over_m", C.c_double), ("ppc_x", C.c_int),
                ("ppc_y", C.c_int), ("lattice", C.c_int),
                ("u_th", C.c_double * 3), ("u_fl", C.c_double * 3),
                ("profile", C.c_int), ("x0", C.c_double), ("x1", C.c_double),
                ("n0", C.c_double)]


class zpic_laser(C.Structure):
    _fields_ = [("enabled", C.c_int), ("a0", C.c_double),
                ("omega0", C.c_double), ("w0", C.c_double),
                ("fwhm", C.c_double), ("x0", C.c_double),
                ("y_center", C.c_double)]


class zpic_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("box_x", C.c_double),
                ("box_y", C.c_double), ("dt", C.c_double),
                ("precision", C.c_int), ("bc_x", C.c_int),
                ("moving_window", C.c_int), ("n_species", C.c_int),
                ("species", zpic_species * MAX_SPECIES),
                ("laser", zpic_laser), ("seed", C.c_uint64),
                ("sim_index", C.c_int), ("energy_every", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("flags", C.c_int),
                ("capacity_slack", C.c_double), ("sort_every", C.c_int),
                ("push_ctas_per_sm", C.c_int)]


class zpic_particles(C.Structure):
    _fields_ = [("precision", C.c_int), ("cap", C.c_size_t),
                ("n", C.c_size_t), ("ix", C.c_void_p), ("iy", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("ux", C.c_void_p),
                ("uy", C.c_void_p), ("uz", C.c_void_p), ("w", C.c_void_p),
                ("id", C.c_void_p)]


class zpic_energy_rec(C.Structure):
    _fields_ = [("step", C.c_int32), ("n_species", C.c_int32),
                ("wE", C.c_double), ("wB", C.c_double),
                ("kin", C.c_double * MAX_SPECIES)]


class zpic_info(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("ld", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
                ("tile_x", C.c_int), ("tile_y", C.c_int),
                ("ntiles_x", C.c_int), ("ntiles_y", C.c_int),
                ("precision", C.c_int), ("step", C.c_int32),
                ("n_shift", C.c_int32), ("n_species", C.c_int),
                ("n_particles", C.c_int64 * MAX_SPECIES),
                ("capacity", C.c_int64 * MAX_SPECIES),
                ("resorts", C.c_int32), ("device_bytes", C.c_size_t),
                ("push_variants", C.c_int32 * MAX_SPECIES),
                ("sort_every", C.c_int32), ("push_ctas_per_sm", C.c_int32),
                ("sorts", C.c_int32)]


class zpic_tuning(C.Structure):
    _fields_ = [("tile_x", C.c_int), ("tile_y", C.c_int),
                ("push_ctas_per_sm", C.c_int), ("sort_every", C.c_int),
                ("ms_per_step", C.c_double)]


class zpic_state(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_shift", C.c_int32),
                ("reserved", C.c_int32),
                ("removed", C.c_int64 * MAX_SPECIES)]


PS_X, PS_Y, PS_UX, PS_UY, PS_UZ = range(5)
PS_IDS = {"x": PS_X, "y": PS_Y, "ux": PS_UX, "uy": PS_UY, "uz": PS_UZ}

_P = C.c_void_p
_PROTOS = {
    "zpic_create": (C.c_int, [C.POINTER(zpic_config), C.POINTER(_P)]),
    "zpic_destroy": (C.c_int, [_P]),
    "zpic_step": (C.c_int, [_P, C.c_int]),
    "zpic_sync": (C.c_int, [_P]),
    "zpic_set_stream": (C.c_int, [_P, _P]),
    "zpic_get_fields_f32": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    "zpic_get_fields_f64": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    "zpic_set_fields_f64": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    "zpic_num_particles": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64)]),
    "zpic_get_particles": (C.c_int, [_P, C.c_int, C.POINTER(zpic_particles),
                                     C.POINTER(C.c_size_t)]),
    "zpic_get_particles_tiles": (C.c_int, [_P, C.c_int, C.c_int, C.c_int,
                                           C.POINTER(zpic_particles),
                                           C.POINTER(C.c_size_t)]),
    "zpic_set_particles": (C.c_int, [_P, C.c_int, C.POINTER(zpic_particles)]),
    "zpic_energy": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "zpic_get_info": (C.c_int, [_P, C.POINTER(zpic_info)]),
    "zpic_field_energy": (C.c_int, [_P, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]),
    "zpic_field_energy_noalloc_f32": (C.c_int, [_P] * 6 + [
        C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, _P, _P]),
    "zpic_get_tile_counts": (C.c_int, [_P, C.c_int, _P, C.c_size_t]),
    "zpic_get_state": (C.c_int, [_P, C.POINTER(zpic_state)]),
    "zpic_set_state": (C.c_int, [_P, C.POINTER(zpic_state)]),
    "zpic_phasespace": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, C.c_int,
                                  C.c_int, _P, C.c_size_t]),
    "zpic_autotune": (C.c_int, [C.POINTER(zpic_config), C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_int), _P,
                                C.c_int, C.POINTER(C.c_int)]),
    "zpic_autotune_candidates": (C.c_int, [_P, C.c_int]),
    "zpic_autotune_all": (C.c_int, [C.POINTER(zpic_config), C.c_int,
                                    C.POINTER(zpic_tuning), _P, C.c_int,
                                    C.POINTER(C.c_int)]),
    "zpic_batch_autotune": (C.c_int, [C.POINTER(zpic_config), C.c_int,
                                      C.c_int, C.POINTER(zpic_tuning), _P,
                                      C.c_int, C.POINTER(C.c_int)]),
    "zpic_profile_enable": (C.c_int, [_P, C.c_int]),
    "zpic_profile_read": (C.c_int, [_P, _P, C.c_size_t, _P, _P, C.c_int,
                                    C.POINTER(C.c_int), C.c_int]),
    "zpic_batch_create": (C.c_int, [C.POINTER(zpic_config), C.c_int,
                                    C.POINTER(_P)]),
    "zpic_batch_step": (C.c_int, [_P, C.c_int]),
    "zpic_batch_sync": (C.c_int, [_P]),
    "zpic_batch_sim": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "zpic_batch_set_stream": (C.c_int, [_P, _P]),
    "zpic_batch_profile_enable": (C.c_int, [_P, C.c_int]),
    "zpic_batch_destroy": (C.c_int, [_P]),
    "zpic_set_allocator": (C.c_int, [_P, _P, _P]),
    "zpic_strerror": (C.c_char_p, [C.c_int]),
    "zpic_last_error": (C.c_char_p, []),
    "zpic_version": (C.c_int, []),
}

_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "libzpic.so is not built (run __graft_entry__.build()); "
                "the library has no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class ZpicError(RuntimeError):
    def __init__(self, code, where):
        L = lib()
        msg = "%s failed: %s (%d): %s" % (
            where, L.zpic_strerror(code).decode(), code,
            L.zpic_last_error().decode())
        super().__init__(msg)
        self.code = code


def check(code, where):
    if code != OK:
        raise ZpicError(code, where)
    return code


def _ptr(a):
    return None if a is None else a.ctypes.data


# --- configuration helpers (plain data, no arithmetic of the method) --------

def species(q_over_m=-1.0, ppc=(4, 4), u_th=(0.0, 0.0, 0.0),
            u_fl=(0.0, 0.0, 0.0), profile=PROFILE_UNIFORM, x0=0.0, x1=0.0,
            n0=1.0, lattice=False):
    s = zpic_species()
    s.q_over_m = q_over_m
    s.ppc_x, s.ppc_y = ppc
    s.lattice = 1 if lattice else 0
    s.u_th[:] = list(u_th)
    s.u_fl[:] = list(u_fl)
    s.profile, s.x0, s.x1, s.n0 = profile, x0, x1, n0
    return s


def config(nx, ny, box, dt, species_list=(), precision=FP32,
           bc_x=BC_PERIODIC, moving_window=False, laser=None,
           seed=2106012485, sim_index=0, energy_every=0, tile=(0, 0),
           track_ids=False, capacity_slack=0.0, filter_j=False,
           sort_every=0, push_ctas_per_sm=0, deterministic=False):
    c = zpic_config()
    c.nx, c.ny = nx, ny
    c.box_x, c.box_y = box
    c.dt = dt
    c.precision = precision
    c.bc_x = bc_x
    c.moving_window = 1 if moving_window else 0
    c.n_species = len(species_list)
    for k, s in enumerate(species_list):
        c.species[k] = s
    if laser is not None:
        c.laser.enabled = 1
        for k in ("a0", "omega0", "w0", "fwhm", "x0", "y_center"):
            setattr(c.laser, k, laser[k])
    c.seed = seed
    c.sim_index = sim_index
    c.energy_every = energy_every
    c.tile_x, c.tile_y = tile
    c.flags = ((TRACK_IDS if track_ids else 0) | (FILTER_J if filter_j else 0)
               | (DETERMINISTIC if deterministic else 0))
    c.capacity_slack = capacity_slack
    c.sort_every = sort_every
    c.push_ctas_per_sm = push_ctas_per_sm
    return c


# --- handle wrappers --------------------------------------------------------

class Sim:
    """A simulation handle (owned, or a view into a Batch)."""

    def __init__(self, cfg=None, _handle=None, _owner=None):
        self._owner = _owner
        if _handle is not None:
            self.h = _handle
            self.owned = False
        else:
            h = _P()
            check(lib().zpic_create(C.byref(cfg), C.byref(h)), "zpic_create")
            self.h = h
            self.owned = True
        self._tracks_ids = cfg is None or bool(cfg.flags & TRACK_IDS)
        self._info_cache = None

    def close(self):
        if self.owned and self.h:
            lib().zpic_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # stepping
    def step(self, n=1):
        check(lib().zpic_step(self.h, n), "zpic_step")

    def sync(self):
        check(lib().zpic_sync(self.h), "zpic_sync")

    def set_stream(self, stream_ptr):
        check(lib().zpic_set_stream(self.h, stream_ptr), "zpic_set_stream")

    # state
    def info(self):
        i = zpic_info()
        check(lib().zpic_get_info(self.h, C.byref(i)), "zpic_get_info")
        return i

    def field(self, name, dtype=np.float64):
        i = self.info()
        out = np.empty((i.ny, i.nx), dtype=dtype)
        fn = (lib().zpic_get_fields_f64 if dtype == np.float64
              else lib().zpic_get_fields_f32)
        check(fn(self.h, FIELD_IDS[name], _ptr(out), out.size),
              "zpic_get_fields")
        return out

    def set_field(self, name, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        check(lib().zpic_set_fields_f64(self.h, FIELD_IDS[name], _ptr(a),
                                        a.size), "zpic_set_fields_f64")

    def num_particles(self, s):
        n = C.c_int64()
        check(lib().zpic_num_particles(self.h, s, C.byref(n)),
              "zpic_num_particles")
        return n.value

    def particles(self, s, dtype=None, with_w=True, with_id=True, out=None,
                  tiles=None):
        """Particles of species s as a dict of numpy arrays (tile order);
        tiles = (begin, end) restricts the copy to those tiles."""
        if dtype is None:
            dtype = np.float64 if self.info().precision == FP64 else np.float32
        if tiles is not None:
            n = int(self.tile_counts(s)[tiles[0]:tiles[1]].sum())
        else:
            n = self.num_particles(s)
        if out is None:
            out = {k: np.empty(n, np.int32) for k in ("ix", "iy")}
            for k in ("x", "y", "ux", "uy", "uz"):
                out[k] = np.empty(n, dtype)
            if with_w:
                out["w"] = np.empty(n, dtype)
            if with_id:
                out["id"] = np.empty(n, np.int32)
        p = zpic_particles()
        p.precision = FP64 if out["x"].dtype == np.float64 else FP32
        p.cap = out["ix"].size
        for k in ("ix", "iy", "x", "y", "ux", "uy", "uz", "w", "id"):
            setattr(p, k, _ptr(out.get(k)))
        nw = C.c_size_t()
        if tiles is not None:
            check(lib().zpic_get_particles_tiles(self.h, s, tiles[0], tiles[1],
                                                 C.byref(p), C.byref(nw)),
                  "zpic_get_particles_tiles")
        else:
            check(lib().zpic_get_particles(self.h, s, C.byref(p), C.byref(nw)),
                  "zpic_get_particles")
        m = nw.value
        return {k: v[:m] for k, v in out.items()}

    def set_particles(self, s, ld):
        """ld: dict with ix, iy, x, y, ux, uy, uz and optional w, id (numpy,
        contiguous; real arrays all float32 or all float64)."""
        dt = ld["x"].dtype
        arrs = {}
        for k in ("ix", "iy", "id"):
            if k in ld and ld[k] is not None:
                arrs[k] = np.ascontiguousarray(ld[k], dtype=np.int32)
        for k in ("x", "y", "ux", "uy", "uz", "w"):
            if k in ld and ld[k] is not None:
                arrs[k] = np.ascontiguousarray(ld[k], dtype=dt)
        p = zpic_particles()
        p.precision = FP64 if dt == np.float64 else FP32
        p.n = p.cap = len(arrs["ix"])
        for k in ("ix", "iy", "x", "y", "ux", "uy", "uz", "w", "id"):
            setattr(p, k, _ptr(arrs.get(k)))
        check(lib().zpic_set_particles(self.h, s, C.byref(p)),
              "zpic_set_particles")

    def energy(self):
        n = C.c_size_t()
        check(lib().zpic_energy(self.h, None, 0, C.byref(n)), "zpic_energy")
        recs = (zpic_energy_rec * max(n.value, 1))()
        check(lib().zpic_energy(self.h, C.cast(recs, _P), n.value,
                                C.byref(n)), "zpic_energy")
        return [(r.step, r.wE, r.wB, list(r.kin[:r.n_species]))
                for r in recs[:n.value]]

    def field_energy(self):
        a, b = C.c_double(), C.c_double()
        check(lib().zpic_field_energy(self.h, C.byref(a), C.byref(b)),
              "zpic_field_energy")
        return a.value, b.value

    def tile_counts(self, s):
        i = self.info()
        out = np.empty(i.ntiles_x * i.ntiles_y, np.int32)
        check(lib().zpic_get_tile_counts(self.h, s, _ptr(out), out.size),
              "zpic_get_tile_counts")
        return out

    # checkpoint / restart
    def state(self):
        st = zpic_state()
        check(lib().zpic_get_state(self.h, C.byref(st)), "zpic_get_state")
        return st

    def set_state(self, st):
        check(lib().zpic_set_state(self.h, C.byref(st)), "zpic_set_state")

    def save_checkpoint(self, path):
        """Writes fields E, B, every species' particles and the run state to
        `path` (numpy .npz); restore with load_checkpoint(cfg, path)."""
        i = self.info()
        arrays = {"f_" + k: self.field(k) for k in EB_NAMES}
        for s in range(i.n_species):
            for k, v in self.particles(s).items():
                # weights only when some differ from 1, ids only when tracked
                if k == "w" and np.all(v == 1):
                    continue
                if k == "id" and not self._tracks_ids:
                    continue
                arrays["p%d_%s" % (s, k)] = v
        st = self.state()
        arrays["state"] = np.array([st.step, st.n_shift] + list(st.removed),
                                   dtype=np.int64)
        arrays["n_species"] = np.array([i.n_species])
        np.savez(path, **arrays)

    # diagnostics
    def phasespace(self, s, qx, qy, range_, bins):
        """Charge density |q0| w per bin of quantities qx, qy ("x", "y", "ux",
        "uy", "uz"; positions in cells) over range_ = (xlo, xhi, ylo, yhi),
        bins = (nbx, nby): an (nby, nbx) array computed on the device."""
        nbx, nby = bins
        out = np.zeros((nby, nbx))
        rg = np.ascontiguousarray(range_, dtype=np.float64)
        check(lib().zpic_phasespace(self.h, s, PS_IDS[qx], PS_IDS[qy],
                                    _ptr(rg), nbx, nby, _ptr(out), out.size),
              "zpic_phasespace")
        return out

    def profile_enable(self, on=True):
        check(lib().zpic_profile_enable(self.h, 1 if on else 0),
              "zpic_profile_enable")

    def profile_read(self, reset=True):
        cap, nl = 16, 64
        names = C.create_string_buffer(cap * nl)
        ms = np.zeros(cap)
        la = np.zeros(cap, np.int32)
        n = C.c_int()
        check(lib().zpic_profile_read(self.h, names, nl, _ptr(ms), _ptr(la),
                                      cap, C.byref(n), 1 if reset else 0),
              "zpic_profile_read")
        out = {}
        for k in range(min(n.value, cap)):
            nm = names.raw[k * nl:(k + 1) * nl].split(b"\0")[0].decode()
            out[nm] = (float(ms[k]), int(la[k]))
        return out


def autotune(cfg, steps=10, retune=True):
    """Best tile size for cfg's class: (tile_x, tile_y, {(tx, ty): ms per
    step}) with every candidate timed (retune=True), or the cached choice
    with an empty dict (retune=False, after an earlier tuning)."""
    n = lib().zpic_autotune_candidates(None, 0)
    xy = np.zeros(2 * n, np.int32)
    lib().zpic_autotune_candidates(_ptr(xy), n)
    ms = np.zeros(n)
    bx, by, nc = C.c_int(), C.c_int(), C.c_int()
    check(lib().zpic_autotune(C.byref(cfg), steps, C.byref(bx), C.byref(by),
                              _ptr(ms) if retune else None, n, C.byref(nc)),
          "zpic_autotune")
    times = {(int(xy[2 * k]), int(xy[2 * k + 1])): float(ms[k])
             for k in range(n)} if retune else {}
    return bx.value, by.value, times


def autotune_all(cfg, steps=10):
    """Tile size, resident CTAs per SM and re-sort interval for cfg's class
    (zpic_autotune_all): (zpic_tuning, list of (stage, candidate, ms per
    step) in the order they were timed)."""
    n = lib().zpic_autotune_candidates(None, 0)
    xy = np.zeros(2 * n, np.int32)
    lib().zpic_autotune_candidates(_ptr(xy), n)
    ms = np.zeros(64)
    t = zpic_tuning()
    nc = C.c_int()
    check(lib().zpic_autotune_all(C.byref(cfg), steps, C.byref(t), _ptr(ms),
                                  ms.size, C.byref(nc)), "zpic_autotune_all")
    n_cta = nc.value - n - 4
    labels = ([("tile", (int(xy[2 * k]), int(xy[2 * k + 1])))
               for k in range(n)] +
              [("ctas_per_sm", k + 1) for k in range(n_cta)] +
              [("sort_every", v) for v in (-1, 10, 20, 40)])
    return t, [(a, b, float(ms[k])) for k, (a, b) in enumerate(labels)]


def load_checkpoint(cfg, path):
    """A Sim created from cfg and restored from save_checkpoint's file."""
    d = np.load(path)
    sim = Sim(cfg)
    st = zpic_state()
    v = d["state"]
    st.step, st.n_shift = int(v[0]), int(v[1])
    for s in range(MAX_SPECIES):
        st.removed[s] = int(v[2 + s])
    sim.set_state(st)
    for k in EB_NAMES:
        sim.set_field(k, d["f_" + k])
    for s in range(int(d["n_species"][0])):
        p = {k: d["p%d_%s" % (s, k)]
             for k in ("ix", "iy", "x", "y", "ux", "uy", "uz", "w", "id")
             if "p%d_%s" % (s, k) in d}
        sim.set_particles(s, p)
    return sim


def _tuning_labels(n_tiles, n_total):
    n = lib().zpic_autotune_candidates(None, 0)
    xy = np.zeros(2 * n, np.int32)
    lib().zpic_autotune_candidates(_ptr(xy), n)
    n_cta = n_total - n - 4
    return ([("tile", (int(xy[2 * k]), int(xy[2 * k + 1]))) for k in range(n)] +
            [("ctas_per_sm", k + 1) for k in range(n_cta)] +
            [("sort_every", v) for v in (-1, 10, 20, 40)])


def batch_autotune(cfgs, steps=10):
    """Tile size, resident CTAs per SM and re-sort interval for the batch of
    cfgs as a whole (zpic_batch_autotune), which Batch(cfgs) then uses for
    settings left at 0: (zpic_tuning, list of (stage, candidate, ms per
    step) in the order they were timed)."""
    arr = (zpic_config * len(cfgs))(*cfgs)
    ms = np.zeros(64)
    t = zpic_tuning()
    nc = C.c_int()
    check(lib().zpic_batch_autotune(arr, len(cfgs), steps, C.byref(t),
                                    _ptr(ms), ms.size, C.byref(nc)),
          "zpic_batch_autotune")
    labels = _tuning_labels(0, nc.value)
    return t, [(a, b, float(ms[k])) for k, (a, b) in enumerate(labels)]


class Batch:
    """Independent simulations advanced together (one launch per stage)."""

    def __init__(self, cfgs):
        arr = (zpic_config * len(cfgs))(*cfgs)
        h = _P()
        check(lib().zpic_batch_create(arr, len(cfgs), C.byref(h)),
              "zpic_batch_create")
        self.h = h
        self.n = len(cfgs)

    def sim(self, i):
        v = _P()
        check(lib().zpic_batch_sim(self.h, i, C.byref(v)), "zpic_batch_sim")
        return Sim(_handle=v, _owner=self)

    def step(self, n=1):
        check(lib().zpic_batch_step(self.h, n), "zpic_batch_step")

    def sync(self):
        check(lib().zpic_batch_sync(self.h), "zpic_batch_sync")

    def set_stream(self, stream_ptr):
        check(lib().zpic_batch_set_stream(self.h, stream_ptr),
              "zpic_batch_set_stream")

    def profile_enable(self, on=True):
        check(lib().zpic_batch_profile_enable(self.h, 1 if on else 0),
              "zpic_batch_profile_enable")

    def profile_read(self, reset=True):
        """Per-stage device time of the batch (read through a member's view,
        which shares the batch's timers)."""
        return self.sim(0).profile_read(reset)

    def close(self):
        if self.h:
            lib().zpic_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
