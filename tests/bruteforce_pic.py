"""Brute-force restatement of one PIC step in 50-digit arithmetic (mpmath).

Used only to pin the FP64 oracle.  Every stage is formulated differently
from the oracle so that a slip in one is not repeated in the other:

* interpolation: sum over all grid samples of F * tent(dX) * tent(dY), with
  tent(s) = max(0, 1 - |s|) in global coordinates (no cell/offset logic,
  no half-cell branch);
* Boris rotation: Rodrigues rotation of u- about t/|t| by -2 atan|t|;
* current: time integral over the step of the charge flux of the moving
  CIC square through each dual face (Jx, Jy) and of q vz times the tent
  weight of each node (Jz), integrated exactly piece by piece between the
  times the path crosses grid lines (2-point Gauss-Legendre is exact for
  the polynomial pieces); no trajectory splitting into segments;
* positions in global coordinates, wrapped at the end.
"""
from __future__ import annotations

import mpmath as mp

mp.mp.dps = 50


def tent(s):
    s = abs(s)
    return 1 - s if s < 1 else mp.mpf(0)


def box(s):
    """1 on the open unit interval (0, 1)."""
    return mp.mpf(1) if 0 < s < 1 else mp.mpf(0)


class BruteSim:
    STAG = {"ex": (0.5, 0), "ey": (0, 0.5), "ez": (0, 0),
            "bx": (0, 0.5), "by": (0.5, 0), "bz": (0.5, 0.5),
            "jx": (0.5, 0), "jy": (0, 0.5), "jz": (0, 0)}

    def __init__(self, nx, ny, dx, dy, dt, open_x=False):
        self.nx, self.ny = nx, ny
        self.dx, self.dy, self.dt = mp.mpf(dx), mp.mpf(dy), mp.mpf(dt)
        self.open_x = open_x
        self.f = {k: [[mp.mpf(0)] * nx for _ in range(ny)]
                  for k in self.STAG}
        self.p = []   # dicts: X, Y (global), u (list of 3), q, qm

    # ---- samples ---------------------------------------------------------
    def get(self, name, i, j):
        j %= self.ny
        if self.open_x:
            if i < 0 or i >= self.nx:
                return mp.mpf(0)
        else:
            i %= self.nx
        return self.f[name][j][i]

    def add(self, name, i, j, v):
        j %= self.ny
        if self.open_x:
            if i < 0 or i >= self.nx:
                return
        else:
            i %= self.nx
        self.f[name][j][i] += v

    # ---- stage 1 ---------------------------------------------------------
    def interp(self, name, X, Y):
        sx, sy = self.STAG[name]
        cx, cy = X / self.dx - sx, Y / self.dy - sy
        tot = mp.mpf(0)
        for i in range(int(mp.floor(cx)) - 1, int(mp.floor(cx)) + 3):
            wx = tent(cx - i)
            if wx == 0:
                continue
            for j in range(int(mp.floor(cy)) - 1, int(mp.floor(cy)) + 3):
                wy = tent(cy - j)
                if wy:
                    tot += self.get(name, i, j) * wx * wy
        return tot

    # ---- stage 2 ---------------------------------------------------------
    @staticmethod
    def boris(qm, dt, E, B, u):
        h = qm * dt / 2
        um = [u[k] + h * E[k] for k in range(3)]
        g = mp.sqrt(1 + sum(c * c for c in um))
        t = [h * B[k] / g for k in range(3)]
        tn = mp.sqrt(sum(c * c for c in t))
        if tn == 0:
            up = um
        else:
            n = [c / tn for c in t]
            phi = -2 * mp.atan(tn)
            cross = [n[1] * um[2] - n[2] * um[1], n[2] * um[0] - n[0] * um[2],
                     n[0] * um[1] - n[1] * um[0]]
            dot = sum(n[k] * um[k] for k in range(3))
            up = [um[k] * mp.cos(phi) + cross[k] * mp.sin(phi) +
                  n[k] * dot * (1 - mp.cos(phi)) for k in range(3)]
        return [up[k] + h * E[k] for k in range(3)]

    # ---- stage 3 ---------------------------------------------------------
    def _pieces(self, X0, Y0, vx, vy):
        """Breakpoints in [0, dt] where X or Y crosses a grid line."""
        ts = {mp.mpf(0), self.dt}
        for X, v, d in ((X0, vx, self.dx), (Y0, vy, self.dy)):
            if v == 0:
                continue
            a, b = X / d, (X + v * self.dt) / d
            lo, hi = (a, b) if a < b else (b, a)
            for k in range(int(mp.floor(lo)) - 1, int(mp.ceil(hi)) + 2):
                t = (k * d - X) / v
                if 0 < t < self.dt:
                    ts.add(t)
        return sorted(ts)

    def deposit(self, X0, Y0, u, q):
        g = mp.sqrt(1 + sum(c * c for c in u))
        vx, vy, vz = u[0] / g, u[1] / g, u[2] / g
        ts = self._pieces(X0, Y0, vx, vy)
        gl = 1 / mp.sqrt(3)
        ci, cj = int(mp.floor(X0 / self.dx)), int(mp.floor(Y0 / self.dy))
        for i in range(ci - 2, ci + 4):
            for j in range(cj - 2, cj + 4):
                jx = jy = jz = mp.mpf(0)
                for a, b in zip(ts[:-1], ts[1:]):
                    m, hw = (a + b) / 2, (b - a) / 2
                    for t in (m - hw * gl, m + hw * gl):
                        cx = (X0 + vx * t) / self.dx
                        cy = (Y0 + vy * t) / self.dy
                        # flux through the dual face x=(i+1/2)dx of node row j
                        jx += hw * q * vx * box(cx - i) * tent(cy - j)
                        jy += hw * q * vy * tent(cx - i) * box(cy - j)
                        jz += hw * q * vz * tent(cx - i) * tent(cy - j)
                if jx:
                    self.add("jx", i, j, jx / self.dt)
                if jy:
                    self.add("jy", i, j, jy / self.dt)
                if jz:
                    self.add("jz", i, j, jz / self.dt)

    # ---- stage 4 ---------------------------------------------------------
    def b_half(self):
        h = self.dt / 2
        nb = {k: [[mp.mpf(0)] * self.nx for _ in range(self.ny)]
              for k in ("bx", "by", "bz")}
        for j in range(self.ny):
            for i in range(self.nx):
                ez_y = (self.get("ez", i, j + 1) - self.get("ez", i, j)) / self.dy
                ez_x = (self.get("ez", i + 1, j) - self.get("ez", i, j)) / self.dx
                ey_x = (self.get("ey", i + 1, j) - self.get("ey", i, j)) / self.dx
                ex_y = (self.get("ex", i, j + 1) - self.get("ex", i, j)) / self.dy
                # curl E = (dEz/dy, -dEz/dx, dEy/dx - dEx/dy); dB/dt = -curl E
                nb["bx"][j][i] = self.f["bx"][j][i] - h * ez_y
                nb["by"][j][i] = self.f["by"][j][i] - h * (-ez_x)
                nb["bz"][j][i] = self.f["bz"][j][i] - h * (ey_x - ex_y)
        self.f.update(nb)

    def e_full(self):
        dt = self.dt
        ne = {k: [[mp.mpf(0)] * self.nx for _ in range(self.ny)]
              for k in ("ex", "ey", "ez")}
        for j in range(self.ny):
            for i in range(self.nx):
                bz_y = (self.get("bz", i, j) - self.get("bz", i, j - 1)) / self.dy
                bz_x = (self.get("bz", i, j) - self.get("bz", i - 1, j)) / self.dx
                by_x = (self.get("by", i, j) - self.get("by", i - 1, j)) / self.dx
                bx_y = (self.get("bx", i, j) - self.get("bx", i, j - 1)) / self.dy
                # curl B = (dBz/dy, -dBz/dx, dBy/dx - dBx/dy); dE/dt = curl B - J
                ne["ex"][j][i] = self.f["ex"][j][i] + dt * (bz_y - self.f["jx"][j][i])
                ne["ey"][j][i] = self.f["ey"][j][i] + dt * (-bz_x - self.f["jy"][j][i])
                ne["ez"][j][i] = self.f["ez"][j][i] + dt * (by_x - bx_y - self.f["jz"][j][i])
        self.f.update(ne)

    # ---- the cycle -------------------------------------------------------
    def step(self):
        for k in ("jx", "jy", "jz"):
            self.f[k] = [[mp.mpf(0)] * self.nx for _ in range(self.ny)]
        kept = []
        for p in self.p:
            E = [self.interp(n, p["X"], p["Y"]) for n in ("ex", "ey", "ez")]
            B = [self.interp(n, p["X"], p["Y"]) for n in ("bx", "by", "bz")]
            u = self.boris(p["qm"], self.dt, E, B, p["u"])
            self.deposit(p["X"], p["Y"], u, p["q"])
            g = mp.sqrt(1 + sum(c * c for c in u))
            X = p["X"] + self.dt * u[0] / g
            Y = p["Y"] + self.dt * u[1] / g
            Lx, Ly = self.nx * self.dx, self.ny * self.dy
            Y = Y % Ly
            if self.open_x:
                if X < 0 or X >= Lx:
                    continue
            else:
                X = X % Lx
            p.update(X=X, Y=Y, u=u)
            kept.append(p)
        self.p = kept
        self.b_half()
        self.e_full()
        self.b_half()
