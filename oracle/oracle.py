"""ctypes front end of the FP64 CPU oracle (zpic_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA path.  State lives in numpy float64 arrays
owned here; the C functions operate on them in place.

Parity pins for every function are in tests/test_oracle_pins.py and
tests/test_oracle_bruteforce.py; what each pin fixes is listed in their
docstrings.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc.so")
_SRC = [os.path.join(_HERE, "zpic_oracle.c")]
_HDR = os.path.join(_HERE, "zpic_oracle.h")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction, so x86
    and Arm hosts give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp] + _SRC + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double),
                ("dy", C.c_double), ("dt", C.c_double), ("open_x", C.c_int),
                ("filter_j", C.c_int)]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


class _Fields(C.Structure):
    _fields_ = [("e", _DP * 3), ("b", _DP * 3), ("j", _DP * 3)]


class _Species(C.Structure):
    _fields_ = [("n", C.c_long), ("cap", C.c_long), ("ix", _IP), ("iy", _IP),
                ("id", _IP), ("x", _DP), ("y", _DP), ("ux", _DP), ("uy", _DP),
                ("uz", _DP), ("w", _DP), ("qm", C.c_double),
                ("q0", C.c_double)]


class _Window(C.Structure):
    _fields_ = [("enabled", C.c_int), ("n_shift", C.c_int),
                ("inject_ppc_x", C.c_int * 8), ("inject_ppc_y", C.c_int * 8),
                ("ramp_x0", C.c_double * 8), ("ramp_len", C.c_double * 8),
                ("dens_n0", C.c_double * 8), ("id_base", C.c_long * 8)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            G, F, S, W = (C.POINTER(_Grid), C.POINTER(_Fields),
                          C.POINTER(_Species), C.POINTER(_Window))
            L.orc_gather.argtypes = [G, F, C.c_int, C.c_int, C.c_double,
                                     C.c_double, _DP, _DP]
            L.orc_boris.argtypes = [C.c_double, C.c_double, _DP, _DP, _DP]
            L.orc_deposit_segment.argtypes = [G, F, C.c_int, C.c_int] + \
                [C.c_double] * 7
            L.orc_move_deposit.argtypes = [G, F, _IP, _IP, _DP, _DP, _DP,
                                           C.c_double]
            L.orc_move_deposit.restype = C.c_int
            L.orc_push_deposit.argtypes = [G, F, S, C.c_int, C.c_int, _DP]
            L.orc_yee_b_half.argtypes = [G, F]
            L.orc_filter_current.argtypes = [G, F]
            L.orc_yee_e.argtypes = [G, F]
            L.orc_field_energy.argtypes = [G, F, _DP, _DP]
            L.orc_laser.argtypes = [G, F] + [C.c_double] * 6
            L.orc_window_shift.argtypes = [G, F, W, C.c_int, S, C.c_int]
            L.orc_window_shift.restype = C.c_int
            L.orc_step.argtypes = [G, F, C.c_int, S, W, C.c_int, C.c_int, _DP]
            L.orc_step.restype = C.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


FIELD_NAMES = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")


class Species:
    """Particle arrays of one species (float64 state, int32 cells)."""

    def __init__(self, qm, q0, ix, iy, x, y, ux, uy, uz, w=None, ids=None,
                 cap=None):
        n = len(ix)
        cap = max(int(cap if cap is not None else n), 1)
        self.qm, self.q0 = float(qm), float(q0)
        self.ix = np.zeros(cap, np.int32)
        self.iy = np.zeros(cap, np.int32)
        self.id = np.zeros(cap, np.int32)
        self.x, self.y, self.ux, self.uy, self.uz, self.w = (
            np.zeros(cap) for _ in range(6))
        self.ix[:n], self.iy[:n] = ix, iy
        self.x[:n], self.y[:n] = x, y
        self.ux[:n], self.uy[:n], self.uz[:n] = ux, uy, uz
        self.w[:n] = 1.0 if w is None else w
        self.id[:n] = np.arange(n) if ids is None else ids
        self.c = _Species(n, cap, _ip(self.ix), _ip(self.iy), _ip(self.id),
                          _dp(self.x), _dp(self.y), _dp(self.ux), _dp(self.uy),
                          _dp(self.uz), _dp(self.w), self.qm, self.q0)

    @property
    def n(self):
        return int(self.c.n)

    def state(self):
        """Dict of the live particle arrays (copies)."""
        n = self.n
        return {k: getattr(self, k)[:n].copy()
                for k in ("ix", "iy", "id", "x", "y", "ux", "uy", "uz", "w")}


class Sim:
    """A grid, its fields and its species, advanced by the oracle."""

    def __init__(self, nx, ny, dx, dy, dt, open_x=False, species=(),
                 window=None, filter_j=False):
        self.g = _Grid(nx, ny, dx, dy, dt, 1 if open_x else 0,
                       1 if filter_j else 0)
        self.f = {k: np.zeros((ny, nx)) for k in FIELD_NAMES}
        self.fc = _Fields((_DP * 3)(*[_dp(self.f[k]) for k in FIELD_NAMES[0:3]]),
                          (_DP * 3)(*[_dp(self.f[k]) for k in FIELD_NAMES[3:6]]),
                          (_DP * 3)(*[_dp(self.f[k]) for k in FIELD_NAMES[6:9]]))
        self.species = list(species)
        self.sc = (_Species * max(len(self.species), 1))(
            *[s.c for s in self.species])
        # the C array holds copies of the structs; keep Species.c pointing
        # at the live copy so counts stay in sync
        for k, s in enumerate(self.species):
            s.c = self.sc[k]
        self.win = _Window()
        if window is not None:
            self.win.enabled = 1
            for s, spec in enumerate(window.get("species", [])):
                self.win.inject_ppc_x[s] = spec.get("ppc_x", 0)
                self.win.inject_ppc_y[s] = spec.get("ppc_y", 0)
                self.win.ramp_x0[s] = spec.get("ramp_x0", 0.0)
                self.win.ramp_len[s] = spec.get("ramp_len", 0.0)
                self.win.dens_n0[s] = spec.get("n0", 1.0)
                self.win.id_base[s] = spec.get("id_base", 0)
        self.step_index = 0
        self.history = []

    @property
    def n_shift(self):
        return int(self.win.n_shift)

    def set_field(self, name, arr):
        self.f[name][...] = arr

    def filter_current(self):
        """Applies the compensated binomial filter to the J arrays."""
        lib().orc_filter_current(C.byref(self.g), C.byref(self.fc))

    def laser(self, a0, omega0, w0, fwhm, x0, yc):
        lib().orc_laser(C.byref(self.g), C.byref(self.fc), a0, omega0, w0,
                        fwhm, x0, yc)

    def step(self, n=1, nthreads=1):
        ns = len(self.species)
        out = np.zeros(2 + max(ns, 1))
        for _ in range(n):
            rc = lib().orc_step(C.byref(self.g), C.byref(self.fc), ns, self.sc,
                                C.byref(self.win), self.step_index, nthreads,
                                _dp(out))
            if rc != 0:
                raise RuntimeError("oracle: species capacity exceeded")
            self.step_index += 1
            self.history.append((self.step_index, out[0], out[1],
                                 out[2:2 + ns].copy()))
        return self.history[-1] if self.history else None

    def push_deposit(self, s, do_deposit=True, nthreads=1):
        kin = C.c_double(0.0)
        lib().orc_push_deposit(C.byref(self.g), C.byref(self.fc),
                               C.byref(self.sc[s]), 1 if do_deposit else 0,
                               nthreads, C.byref(kin))
        return kin.value

    def yee(self):
        L = lib()
        L.orc_yee_b_half(C.byref(self.g), C.byref(self.fc))
        L.orc_yee_e(C.byref(self.g), C.byref(self.fc))
        L.orc_yee_b_half(C.byref(self.g), C.byref(self.fc))

    def gather(self, ix, iy, x, y):
        E = (C.c_double * 3)()
        B = (C.c_double * 3)()
        lib().orc_gather(C.byref(self.g), C.byref(self.fc), ix, iy, x, y, E, B)
        return np.array(E[:]), np.array(B[:])

    def field_energy(self):
        a, b = C.c_double(), C.c_double()
        lib().orc_field_energy(C.byref(self.g), C.byref(self.fc), C.byref(a),
                               C.byref(b))
        return a.value, b.value


def boris(qm, dt, E, B, u):
    """Stage 2 on one momentum vector; returns the new u."""
    Ea = (C.c_double * 3)(*E)
    Ba = (C.c_double * 3)(*B)
    ua = (C.c_double * 3)(*u)
    lib().orc_boris(qm, dt, Ea, Ba, ua)
    return np.array(ua[:])


def phasespace(state, q0, qx, qy, range_, bins):
    """Phase-space density of one species (the field / phase-space reports of
    Sec. 4.1): every particle adds |q0| w to the bin (bx, by) of quantities
    qx, qy ("x", "y": global position ix + x, iy + y in cells; "ux", "uy",
    "uz").  On an axis with bounds lo, hi and nb bins, the bin of v is
    floor((v - lo) * (nb / (hi - lo))) in double precision, and particles
    whose bin falls outside [0, nb) on either axis are not counted.
    Returns an (nby, nbx) array."""
    vals = {"x": state["ix"] + np.asarray(state["x"], np.float64),
            "y": state["iy"] + np.asarray(state["y"], np.float64),
            "ux": np.asarray(state["ux"], np.float64),
            "uy": np.asarray(state["uy"], np.float64),
            "uz": np.asarray(state["uz"], np.float64)}
    nbx, nby = bins
    xlo, xhi, ylo, yhi = (float(v) for v in range_)
    tx = (vals[qx] - xlo) * (nbx / (xhi - xlo))
    ty = (vals[qy] - ylo) * (nby / (yhi - ylo))
    keep = (tx >= 0) & (tx < nbx) & (ty >= 0) & (ty < nby)
    w = state.get("w")
    w = np.ones(len(tx)) if w is None else np.asarray(w, np.float64)
    hist = np.zeros((nby, nbx))
    np.add.at(hist, (np.floor(ty[keep]).astype(np.int64),
                     np.floor(tx[keep]).astype(np.int64)),
              abs(q0) * w[keep])
    return hist

