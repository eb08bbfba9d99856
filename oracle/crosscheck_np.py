"""Independent NumPy restatement of the coupled LB step, D2Q9, periodic.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  This is a second
transcription of Sec. II, written array-wise with ``np.roll`` and with its own
direction order, so that it shares no loop structure or table with
``lbm_oracle.c``.  It implements the same readings (listed in the header of
``lbm_oracle.c``): u^n in the omega-term of P, trace-free Pi in the filter,
phi clamped for rho / tau_mix / omega.  Agreement of the two to ~1e-13 pins
both against transcription slips (a dropped term, a wrong sign or index).
"""
from __future__ import annotations

import numpy as np

T = 1.0 / 3.0
# direction order differs from the C oracle on purpose
C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
REST = 0


def _at(f, cx, cy):
    """f evaluated at x + (cx, cy) on a periodic [ny, nx] grid."""
    return np.roll(f, shift=(-cy, -cx), axis=(0, 1))


def _grad(f):
    gx = np.zeros_like(f)
    gy = np.zeros_like(f)
    for (cx, cy), w in zip(C, WT):
        d = _at(f, cx, cy) - _at(f, -cx, -cy)
        gx += d * cx * w
        gy += d * cy * w
    return gx / (2 * T), gy / (2 * T)


def _lap(f):
    acc = np.zeros_like(f)
    for (cx, cy), w in zip(C, WT):
        acc += (_at(f, cx, cy) - f) * w
    return 2 * acc / T


class CrossCheck2D:
    def __init__(self, params: dict, phi0, P0, ux0, uy0):
        self.p = dict(params)
        self.phi0 = np.array(phi0, dtype=np.float64)
        ny, nx = self.phi0.shape
        self.h = np.zeros((9, ny, nx))
        self.g = np.zeros((9, ny, nx))
        self.P = np.array(P0, dtype=np.float64)
        self.ux = np.array(ux0, dtype=np.float64)
        self.uy = np.array(uy0, dtype=np.float64)
        self.h, self.g = self._collide(self.phi0, self.P, self.ux, self.uy, None, None)

    # material properties
    def _props(self, phi):
        p = self.p
        ph = np.clip(phi, 0.0, 1.0) if p.get("clamp_phi_props", 1) else phi
        rho = p["rho_a"] + ph * (p["rho_w"] - p["rho_a"])
        return ph, rho

    def _collide(self, phi, P, ux, uy, hp, gp):
        p = self.p
        ph, rho = self._props(phi)
        gpx, gpy = _grad(phi)
        lphi = _lap(phi)
        dux = _grad(ux)
        duy = _grad(uy)
        # gu[a][b] = d u_a / d x_b
        gu = [[dux[0], dux[1]], [duy[0], duy[1]]]
        gn = np.sqrt(gpx ** 2 + gpy ** 2)
        nx_, ny_ = gpx / (gn + p["eps"]), gpy / (gn + p["eps"])
        theta = p["M"] / T * (1 - 4 * (phi - 0.5) ** 2) / p["W"]
        s = lphi / (np.abs(lphi) + p["eps"])
        F = lambda v: np.maximum(0.0, np.minimum(1.0, v))
        Y1 = np.minimum(F((phi - p["phi_n"]) / p["D"]), F(-(phi - 1) / p["D"]))
        Y2 = np.minimum(F(phi / p["D"]), F(-(phi - p["phi_m"]) / p["D"]))
        dtheta = p["gamma"] * p["M"] / (T * p["W"]) * gn * ((1 + s) * Y1 + (1 - s) * Y2)
        mu = 48 * p["sigma"] / p["W"] * phi * (phi - 1) * (phi - 0.5) - 1.5 * p["sigma"] * p["W"] * lphi
        gx, gy = p["g_ext"][0], p["g_ext"][1]
        Fx = rho * gx + mu * gpx
        Fy = rho * gy + mu * gpy
        tw = p["nu_w"] / T + 0.5
        ta = p["nu_a"] / T + 0.5
        tau = ta + ph * (tw - ta)
        nu = T * (tau - 0.5)
        B = 2 / 3 * (nu - p["lambda_b"]) + T / 2
        div = gu[0][0] + gu[1][1]
        sig = [[rho * nu * (gu[a][b] + gu[b][a]) + (rho * 2 / 3 * (p["lambda_b"] - nu) * div if a == b else 0.0)
                for b in range(2)] for a in range(2)]
        grx = (p["rho_w"] - p["rho_a"]) * gpx
        gry = (p["rho_w"] - p["rho_a"]) * gpy
        sgx = sig[0][0] * grx + sig[0][1] * gry
        sgy = sig[1][0] * grx + sig[1][1] * gry
        usq = ux ** 2 + uy ** 2
        tau_phi = p["M"] / T + 0.5
        heq = np.zeros((9,) + phi.shape)
        geq = np.zeros((9,) + phi.shape)
        for i, ((cx, cy), w) in enumerate(zip(C, WT)):
            cu = cx * ux + cy * uy
            Gam = w * (1 + cu / T + cu * cu / (2 * T * T) - usq / (2 * T))
            heq[i] = phi * Gam + (theta + dtheta) * w * (cx * nx_ + cy * ny_)
            delta = 1.0 if i == REST else 0.0
            geq[i] = (P / (p["rho_a"] * T) * delta + Gam - w + w * (cx * Fx + cy * Fy) / (rho * T)
                      + B * (w - delta) / T * div + w * (cx * sgx + cy * sgy) / (rho * rho * T))
        if hp is None:
            return heq, geq
        hs = hp - (hp - heq) / tau_phi
        neq = gp - geq
        Pxx = sum(cx * cx * neq[i] for i, (cx, cy) in enumerate(C))
        Pyy = sum(cy * cy * neq[i] for i, (cx, cy) in enumerate(C))
        Pxy = sum(cx * cy * neq[i] for i, (cx, cy) in enumerate(C))
        if not self.p.get("filter_full_trace", 0):
            tr = Pxx + Pyy
            Pxx = Pxx - tr / 2
            Pyy = Pyy - tr / 2
        gs = np.zeros_like(gp)
        for i, ((cx, cy), w) in enumerate(zip(C, WT)):
            contr = (cx * cx - T) * Pxx + (cy * cy - T) * Pyy + 2 * cx * cy * Pxy
            gs[i] = geq[i] + (1 - 1 / tau) * w / (2 * T * T) * contr
        return hs, gs

    def step(self, n=1):
        p = self.p
        for _ in range(n):
            hp = np.stack([_at(self.h[i], -cx, -cy) for i, (cx, cy) in enumerate(C)])
            gp = np.stack([_at(self.g[i], -cx, -cy) for i, (cx, cy) in enumerate(C)])
            phi = hp.sum(axis=0)
            ph, rho = self._props(phi)
            K = np.stack([w / (T * rho) * (_at(self.P, -cx, -cy) - self.P) for (cx, cy), w in zip(C, WT)])
            ux = sum((gp[i] + K[i]) * cx for i, (cx, cy) in enumerate(C))
            uy = sum((gp[i] + K[i]) * cy for i, (cx, cy) in enumerate(C))
            omega = (rho - p["rho_a"]) / (p["rho_w"] - p["rho_a"]) * (p["rho_w"] / p["rho_a"] - 1)
            sgk = sum(gp[i] + (1 + omega) * K[i] for i in range(9))
            swcu = sum(w * (cx * _at(self.ux, -cx, -cy) + cy * _at(self.uy, -cx, -cy))
                       for (cx, cy), w in zip(C, WT))
            P1 = p["rho_a"] * T * sgk + omega * p["rho_a"] * swcu
            self.h, self.g = self._collide(phi, P1, ux, uy, hp, gp)
            self.P, self.ux, self.uy = P1, ux, uy

    def fields(self):
        return self.h.sum(axis=0), self.P, self.ux, self.uy
