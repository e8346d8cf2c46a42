"""Exact solution of the 1D Riemann problem for two stiffened gases.

TEST INFRASTRUCTURE ONLY (a pin for the oracle's whole step on the
gas-liquid shock tube of Sec. 5).  This is the textbook exact solver for the
ideal gas (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
ch. 4) with each side's pressure shifted by its own P_inf, which is exact for
the stiffened-gas EOS of Eq. (eos): rho e = (p + gamma P_inf)/(gamma - 1).
Each side keeps its own (gamma, P_inf); the contact separates the materials.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Side:
    rho: float
    u: float
    p: float
    gamma: float
    pinf: float

    @property
    def pbar(self) -> float:
        return self.p + self.pinf

    @property
    def c(self) -> float:
        return math.sqrt(self.gamma * self.pbar / self.rho)


def _f(p: float, s: Side):
    """Velocity jump across the wave of side s as a function of the star pressure,
    and its derivative (Toro eqs. 4.6-4.7 with p -> p + P_inf)."""
    g = s.gamma
    pb = p + s.pinf
    pk = s.pbar
    if p > s.p:  # shock
        A = 2.0 / ((g + 1.0) * s.rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (pb + B))
        return (pb - pk) * q, q * (1.0 - 0.5 * (pb - pk) / (B + pb))
    # rarefaction
    c = s.c
    r = pb / pk
    val = 2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0)
    der = 1.0 / (s.rho * c) * r ** (-(g + 1.0) / (2.0 * g))
    return val, der


def star_state(L: Side, R: Side):
    """(p*, u*) from f_L(p) + f_R(p) + (u_R - u_L) = 0, by bracketed Newton."""
    du = R.u - L.u
    lo = max(-L.pinf, -R.pinf)
    lo = lo + 1e-12 * max(1.0, abs(lo))
    F = lambda p: _f(p, L)[0] + _f(p, R)[0] + du
    if F(lo) > 0.0:
        raise ValueError("vacuum generated: no star state")
    hi = max(L.p, R.p, 1.0)
    while F(hi) < 0.0:
        hi = hi * 2.0 + abs(lo)
    p = 0.5 * (lo + hi)
    for _ in range(200):
        fl, dl = _f(p, L)
        fr, dr = _f(p, R)
        val = fl + fr + du
        if val > 0.0:
            hi = p
        else:
            lo = p
        pn = p - val / (dl + dr)
        if not (lo < pn < hi):
            pn = 0.5 * (lo + hi)
        if abs(pn - p) <= 1e-15 * max(abs(pn), 1.0):
            p = pn
            break
        p = pn
    u = 0.5 * (L.u + R.u) + 0.5 * (_f(p, R)[0] - _f(p, L)[0])
    return p, u


def sample(L: Side, R: Side, xi: np.ndarray):
    """Solution (rho, u, p, material) at similarity coordinates xi = (x - x0)/t;
    material is 0 on the left material's side of the contact and 1 on the right."""
    ps, us = star_state(L, R)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    mat = np.empty(xi.shape, dtype=np.int8)
    for idx, x in np.ndenumerate(xi):
        if x <= us:
            s, sgn, m = L, 1.0, 0
        else:
            s, sgn, m = R, -1.0, 1
        g, c, pk = s.gamma, s.c, s.pbar
        psb = ps + s.pinf
        # work in the frame where the wave of side s moves in the -sgn direction
        if ps > s.p:  # shock
            S = s.u - sgn * c * math.sqrt((g + 1.0) / (2.0 * g) * psb / pk + (g - 1.0) / (2.0 * g))
            beyond = (x <= S) if sgn > 0 else (x >= S)
            if beyond:
                r, uu, pp = s.rho, s.u, s.p
            else:
                gr = (g - 1.0) / (g + 1.0)
                r = s.rho * (psb / pk + gr) / (gr * psb / pk + 1.0)
                uu, pp = us, ps
        else:  # rarefaction
            cs = c * (psb / pk) ** ((g - 1.0) / (2.0 * g))
            Sh = s.u - sgn * c
            St = us - sgn * cs
            if (x <= Sh) if sgn > 0 else (x >= Sh):
                r, uu, pp = s.rho, s.u, s.p
            elif (x > St) if sgn > 0 else (x < St):
                r, uu, pp = s.rho * (psb / pk) ** (1.0 / g), us, ps
            else:
                a = 2.0 / (g + 1.0) + sgn * (g - 1.0) / ((g + 1.0) * c) * (s.u - x)
                r = s.rho * a ** (2.0 / (g - 1.0))
                uu = 2.0 / (g + 1.0) * (sgn * c + (g - 1.0) / 2.0 * s.u + x)
                pp = pk * a ** (2.0 * g / (g - 1.0)) - s.pinf
        rho[idx], u[idx], p[idx], mat[idx] = r, uu, pp, m
    return rho, u, p, mat


def cell_averages(L: Side, R: Side, x0: float, t: float, edges: np.ndarray, sub: int = 64):
    """Cell averages of rho, u, p over the cells with the given edges (midpoint
    rule with ``sub`` samples per cell)."""
    edges = np.asarray(edges, dtype=np.float64)
    n = edges.size - 1
    w = np.diff(edges)
    frac = (np.arange(sub) + 0.5) / sub
    xs = edges[:-1, None] + w[:, None] * frac[None, :]
    rho, u, p, _ = sample(L, R, (xs - x0) / t)
    return rho.mean(axis=1), u.mean(axis=1), p.mean(axis=1)
