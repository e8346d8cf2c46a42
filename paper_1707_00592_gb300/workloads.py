"""Seeded synthetic initial conditions for the two-phase solver.

This module holds no arithmetic of the numerical method: it only lays out
initial primitive fields ``Q = (rho, u_1..u_ndim, p, Gamma, Pi)`` on the padded
SoA grid (3 ghost layers per side of every active direction; ghosts are left
zero and are filled by the boundary conditions of whichever solver consumes
them).  Material parameters (gamma, P_inf) enter as ``Gamma = 1/(gamma-1)``
and ``Pi = gamma P_inf/(gamma-1)`` (Eq. material-properties of the paper);
smeared interfaces mix rho, Gamma and Pi linearly in the volume fraction,
with p and u uniform across the interface.  Both the CUDA path and the
oracle convert these primitives to conservative variables with their own code.

Workloads (sizes are the defaults; tests pass smaller ones):
  * ``gas_water_tube``   1D gas-water shock tube, 200 cells, x0 = 0.7
  * ``interface_transport`` 1D gas/liquid interface transport (Sec. 5.1)
  * ``shock_bubble_1d``  1D shock/bubble (Sec. 5.3)
  * ``shock_bubble_2d``  2D water shock (Ms = 1.5) on an air bubble, 1024^2
  * ``drop_3d``          3D periodic water drop in air with 1% density noise
  * ``riemann_tubes``    4096 independent 1D Riemann tubes of uneven length
  * ``entropy_wave``     smooth periodic density wave (convergence study)
  * ``random_state``     random smooth / shocked / two-phase fields
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NG = 3
AIR = (1.4, 0.0)
WATER = (4.4, 6.0e8)


def material(gamma: float, pinf: float):
    """(Gamma, Pi) of a stiffened gas with parameters (gamma, P_inf)."""
    return 1.0 / (gamma - 1.0), gamma * pinf / (gamma - 1.0)


@dataclass
class Case:
    """A grid plus its initial primitive state on the padded layout."""
    name: str
    ndim: int
    n: tuple
    dx: tuple
    bc: tuple
    Q: np.ndarray                  # (nv, Pz, Py, Px) primitives, ghosts zero
    t_end: float = 0.0
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return self.ndim + 4

    @property
    def cells(self) -> int:
        return int(np.prod([self.n[d] for d in range(self.ndim)]))


def padded_shape(ndim: int, n) -> tuple:
    P = [int(n[d]) + 2 * NG if d < ndim else 1 for d in range(3)]
    return (ndim + 4, P[2], P[1], P[0])


def interior(ndim: int, n) -> tuple:
    sl = [slice(None)]
    for d in (2, 1, 0):
        sl.append(slice(NG, NG + int(n[d])) if d < ndim else slice(None))
    return tuple(sl)


def _centres(ndim, n, lo, dx):
    """Cell-centre coordinate arrays (x, y, z) shaped like the interior (z, y, x)."""
    ax = []
    for d in range(3):
        if d < ndim:
            ax.append(lo[d] + (np.arange(n[d]) + 0.5) * dx[d])
        else:
            ax.append(np.zeros(1))
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _fill(ndim, n, fields):
    Q = np.zeros(padded_shape(ndim, n))
    sl = interior(ndim, n)
    for f, a in enumerate(fields):
        Q[(f,) + sl[1:]] = a
    return Q


def _two_state_1d(n, x0, left, right, length=1.0):
    """Sharp two-state 1D problem; left/right = (rho, u, p, gamma, P_inf)."""
    dx = length / n
    x = (np.arange(n) + 0.5) * dx
    L = x < x0
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    GL, PL = material(left[3], left[4])
    GR, PR = material(right[3], right[4])
    G = np.where(L, GL, GR)
    P = np.where(L, PL, PR)
    return dx, _fill(1, (n, 1, 1), [rho, u, p, G, P])


def gas_water_tube(n: int = 200) -> Case:
    """Water (1000, 0, 1e9, 4.4, 6e8) | air (50, 0, 1e5, 1.4, 0) at x = 0.7 on [0, 1],
    transmissive ends, t_end = 2.4e-4."""
    left = (1000.0, 0.0, 1.0e9, 4.4, 6.0e8)
    right = (50.0, 0.0, 1.0e5, 1.4, 0.0)
    dx, Q = _two_state_1d(n, 0.7, left, right)
    return Case("gas_water_tube", 1, (n, 1, 1), (dx, 1.0, 1.0), (("transmissive", "transmissive"),), Q,
                t_end=2.4e-4, meta={"left": left, "right": right, "x0": 0.7})


def interface_transport(n: int = 200) -> Case:
    """Sec. 5.1: (1, 100, 1, 7, 3000) on [0, 2] | (0.001, 100, 1, 1.4, 0) on [2, 4], t = 0.01."""
    left = (1.0, 100.0, 1.0, 7.0, 3000.0)
    right = (0.001, 100.0, 1.0, 1.4, 0.0)
    dx, Q = _two_state_1d(n, 2.0, left, right, length=4.0)
    return Case("interface_transport", 1, (n, 1, 1), (dx, 1.0, 1.0), (("transmissive", "transmissive"),), Q,
                t_end=0.01, meta={"left": left, "right": right, "x0": 2.0})


def shock_bubble_1d(n: int = 200) -> Case:
    """Sec. 5.3: four-state shock/bubble problem on [0, 1], t = 3.87."""
    states = [(0.25, (1.2199, 42.455, 1.0e4, 7.0, 3.31e3)),
              (0.4, (1.0, 0.0, 1.0, 7.0, 3.31e3)),
              (0.6, (1.0e-3, 0.0, 1.0, 1.4, 0.0)),
              (1.0, (1.0, 0.0, 1.0, 7.0, 3.31e3))]
    dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    cols = [np.zeros(n) for _ in range(5)]
    lo = 0.0
    for hi, s in states:
        m = (x >= lo) & (x < hi)
        G, P = material(s[3], s[4])
        for k, v in enumerate((s[0], s[1], s[2], G, P)):
            cols[k][m] = v
        lo = hi
    Q = _fill(1, (n, 1, 1), cols)
    return Case("shock_bubble_1d", 1, (n, 1, 1), (dx, 1.0, 1.0), (("transmissive", "transmissive"),), Q,
                t_end=3.87)


def water_shock_state(Ms: float, pre=(1000.0, 0.0, 1.0e5), mat=WATER):
    """Post-shock (rho, u, p) behind a shock of Mach number Ms running in -x into
    still water, from the Rankine-Hugoniot relations of the stiffened gas
    (those of the ideal gas in p + P_inf)."""
    g, pinf = mat
    rho1, _, p1 = pre
    c1 = math.sqrt(g * (p1 + pinf) / rho1)
    ratio = (g + 1.0) * Ms * Ms / ((g - 1.0) * Ms * Ms + 2.0)
    pbar2 = (p1 + pinf) * (1.0 + 2.0 * g / (g + 1.0) * (Ms * Ms - 1.0))
    u2 = -Ms * c1 * (1.0 - 1.0 / ratio)
    return rho1 * ratio, u2, pbar2 - pinf


def _volume_fraction(r, R, h):
    """Interface smeared linearly over two cells of size h."""
    return np.clip(0.5 + (R - r) / (2.0 * h), 0.0, 1.0)


def shock_bubble_2d(n: int = 1024, Ms: float = 1.5) -> Case:
    """Air bubble (rho 1, gamma 1.4) of radius 0.2 at (0.6, 0.5) in water
    (1000, 4.4, 6e8) at p = 1e5 on [0, 1]^2; a Ms = 1.5 water shock at x = 0.8
    moving -x (post-shock water on x > 0.8).  Transmissive boundaries."""
    h = 1.0 / n
    X, Y, _ = _centres(2, (n, n, 1), (0.0, 0.0, 0.0), (h, h, 1.0))
    X, Y = X[0], Y[0]
    r = np.hypot(X - 0.6, Y - 0.5)
    a = _volume_fraction(r, 0.2, h)             # air fraction
    Gw, Pw = material(*WATER)
    Ga, Pa = material(*AIR)
    rho = a * 1.0 + (1.0 - a) * 1000.0
    G = a * Ga + (1.0 - a) * Gw
    P = a * Pa + (1.0 - a) * Pw
    u = np.zeros_like(X)
    v = np.zeros_like(X)
    p = np.full_like(X, 1.0e5)
    rs, us, ps = water_shock_state(Ms)
    post = X > 0.8
    rho = np.where(post, rs, rho)
    u = np.where(post, us, u)
    p = np.where(post, ps, p)
    G = np.where(post, Gw, G)
    P = np.where(post, Pw, P)
    Q = _fill(2, (n, n, 1), [rho, u, v, p, G, P])
    bc = (("transmissive", "transmissive"), ("transmissive", "transmissive"))
    return Case("shock_bubble_2d", 2, (n, n, 1), (h, h, 1.0), bc, Q, steps=2000,
                meta={"Ms": Ms, "post_shock": (rs, us, ps)})


def _shock_cylinder(name, nx, ny, Lx, Ly, x_shock, centre, radius, pre, post, inner, bc, **kw) -> Case:
    """A planar shock at x = x_shock running in -x (post-shock state on
    x > x_shock) towards a cylinder of another material at rest in the
    pre-shock state.  States are (rho, u, p, gamma, P_inf); the cylinder's
    interface is smeared over two cells (rho, Gamma, Pi mixed in the volume
    fraction, p and u uniform)."""
    hx, hy = Lx / nx, Ly / ny
    X, Y, _ = _centres(2, (nx, ny, 1), (0.0, 0.0, 0.0), (hx, hy, 1.0))
    X, Y = X[0], Y[0]
    a = _volume_fraction(np.hypot(X - centre[0], Y - centre[1]), radius, min(hx, hy))  # cylinder fraction
    Go, Po = material(pre[3], pre[4])
    Gi, Pi_ = material(inner[3], inner[4])
    rho = a * inner[0] + (1.0 - a) * pre[0]
    G = a * Gi + (1.0 - a) * Go
    P = a * Pi_ + (1.0 - a) * Po
    u = np.full_like(X, pre[1])
    v = np.zeros_like(X)
    p = np.full_like(X, pre[2])
    shocked = X > x_shock
    Gs, Ps = material(post[3], post[4])
    rho = np.where(shocked, post[0], rho)
    u = np.where(shocked, post[1], u)
    p = np.where(shocked, post[2], p)
    G = np.where(shocked, Gs, G)
    P = np.where(shocked, Ps, P)
    Q = _fill(2, (nx, ny, 1), [rho, u, v, p, G, P])
    return Case(name, 2, (nx, ny, 1), (hx, hy, 1.0), bc, Q, **kw)


def haas_sturtevant(gas: str = "R22", nx: int = 3000, ny: int = 1000) -> Case:
    """Sec. 6.1: a Ms = 1.22 shock in air meets a cylinder of R22 (heavier than
    air) or helium (lighter) in a 267 x 89 mm channel (SI units).  Pre-shock
    air (1.4 kg/m^3, 0 m/s, 0.1 MPa), post-shock air (1.927, -114.42, 0.157
    MPa) right of x = 203 mm; cylinder of diameter 50 mm centred at (178, 44.5)
    mm: R22 (4.415, gamma 1.249) or He (0.255, gamma 1.648); P_inf = 0 for all
    (the single-phase limit).  Reflective walls at y = 0 and y = 89 mm,
    transmissive ends in x; MOOD is off for these runs."""
    inner = {"R22": (4.415, 0.0, 1.0e5, 1.249, 0.0), "He": (0.255, 0.0, 1.0e5, 1.648, 0.0)}[gas]
    return _shock_cylinder(f"haas_sturtevant_{gas}", nx, ny, 0.267, 0.089, 0.203, (0.178, 0.0445), 0.025,
                           (1.4, 0.0, 1.0e5, 1.4, 0.0), (1.927, -114.42, 1.57e5, 1.4, 0.0), inner,
                           (("transmissive", "transmissive"), ("reflective", "reflective")),
                           t_end={"R22": 420e-6, "He": 674e-6}[gas], meta={"mood": False, "Ms": 1.22})


def shock_droplet(n: int = 800) -> Case:
    """Sec. 6.2: a Ms = 2.0 shock in air meets a water droplet on a 20 x 20 mm
    domain (SI units).  Pre-shock air (1.2 kg/m^3, 0 m/s, 0.1 MPa, gamma 1.4),
    post-shock air (3.2, -434, 0.456 MPa) right of x = 16 mm; droplet of
    diameter 8 mm centred at (12, 10) mm: water (1000, 0.1 MPa, gamma 4.34,
    P_inf 0.484 GPa).  Transmissive boundaries; MOOD is off for this run."""
    return _shock_cylinder("shock_droplet", n, n, 0.02, 0.02, 0.016, (0.012, 0.010), 0.004,
                           (1.2, 0.0, 1.0e5, 1.4, 0.0), (3.2, -434.0, 4.56e5, 1.4, 0.0),
                           (1000.0, 0.0, 1.0e5, 4.34, 4.84e8),
                           (("transmissive", "transmissive"), ("transmissive", "transmissive")),
                           meta={"mood": False, "Ms": 2.0})


def drop_3d(n: int = 256, seed: int = 0) -> Case:
    """Water drop (r = 0.25) centred in air on the periodic unit cube, uniform
    u = (1, 0.5, 0.25), p = 1e5, density times (1 + 0.01 S/max|S|) with
    S = sum of 8 plane waves sin(2 pi k.x + theta) drawn from PCG64(seed)."""
    h = 1.0 / n
    X, Y, Z = _centres(3, (n, n, n), (0.0, 0.0, 0.0), (h, h, h))
    r = np.sqrt((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2)
    a = _volume_fraction(r, 0.25, h)            # water fraction
    Gw, Pw = material(*WATER)
    Ga, Pa = material(*AIR)
    rho = a * 1000.0 + (1.0 - a) * 1.0
    G = a * Gw + (1.0 - a) * Ga
    P = a * Pw + (1.0 - a) * Pa
    rng = np.random.Generator(np.random.PCG64(seed))
    S = np.zeros_like(X)
    for _ in range(8):
        k = rng.integers(-4, 5, size=3)
        th = rng.uniform(0.0, 2.0 * math.pi)
        S += np.sin(2.0 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + th)
    mx = np.abs(S).max()
    if mx > 0:
        rho = rho * (1.0 + 0.01 * S / mx)
    Q = _fill(3, (n, n, n), [rho, np.full_like(X, 1.0), np.full_like(X, 0.5), np.full_like(X, 0.25),
                            np.full_like(X, 1.0e5), G, P])
    bc = tuple(("periodic", "periodic") for _ in range(3))
    return Case("drop_3d", 3, (n, n, n), (h, h, h), bc, Q, steps=500, meta={"seed": seed})


def entropy_wave(n: int, ndim: int = 1, amp: float = 0.2, kind: str = "sine") -> Case:
    """Smooth density wave advected with u = 1 in x (and v = 1 in 2D, along the
    diagonal) through the periodic unit box: rho = 1 + amp sin(2 pi (x + y)) or the
    Gauss pulse 1 + amp exp(-300 ((x-0.5)^2 + ...)); p = 1, air."""
    h = 1.0 / n
    nn = tuple(n if d < ndim else 1 for d in range(3))
    X, Y, Z = _centres(ndim, nn, (0.0, 0.0, 0.0), (h, h, h))
    sl = (0,) * (3 - ndim)
    X, Y = X[sl] if ndim < 3 else X, Y[sl] if ndim < 3 else Y
    # cell averages (a finite-volume initial state), not centre values
    if kind == "sine":
        s = X if ndim == 1 else X + Y
        rho = 1.0 + amp * np.sin(2.0 * math.pi * s) * (math.sin(math.pi * h) / (math.pi * h)) ** ndim
    else:
        gx, gw = np.polynomial.legendre.leggauss(8)
        rho = np.zeros_like(X)
        for a, wa in zip(gx, gw):
            if ndim == 1:
                rho += 0.5 * wa * np.exp(-300.0 * (X + 0.5 * a * h - 0.5) ** 2)
            else:
                for b, wb in zip(gx, gw):
                    r2 = (X + 0.5 * a * h - 0.5) ** 2 + (Y + 0.5 * b * h - 0.5) ** 2
                    rho += 0.25 * wa * wb * np.exp(-300.0 * r2)
        rho = 1.0 + amp * rho
    G, P = material(*AIR)
    vel = [np.ones_like(rho) for _ in range(ndim)]
    Q = _fill(ndim, nn, [rho] + vel + [np.ones_like(rho), np.full_like(rho, G), np.full_like(rho, P)])
    bc = tuple(("periodic", "periodic") for _ in range(ndim))
    return Case(f"entropy_wave_{kind}", ndim, nn, tuple(h if d < ndim else 1.0 for d in range(3)), bc, Q,
                meta={"amp": amp, "kind": kind})


def _pick(rng, k):
    return rng.integers(0, 2, size=k)


def riemann_tubes(ntubes: int = 4096, lmin: int = 256, lmax: int = 8192, seed: int = 0):
    """Independent 1D Riemann tubes: lengths log-uniform in [lmin, lmax]; each side
    rho log-uniform in [1, 1000], p log-uniform in [1e5, 1e9], u uniform in
    [-100, 100], air or water with equal odds; interface at the tube's midpoint.
    A pair whose two rarefactions would come near a vacuum has its velocities
    redrawn: the velocity spread u_R - u_L must stay below half the sum of the
    two sides' rarefaction velocity gains down to the floor pressure p_f, the
    lowest pressure both materials admit (max(-P_inf,L, -P_inf,R): 0 when
    either side is air).  A side's gain is the isentropic rarefaction velocity
    2 c/(gamma-1) [1 - ((p_f + P_inf)/(p + P_inf))^((gamma-1)/(2 gamma))] with
    c^2 = gamma (p + P_inf)/rho.  Returns (offsets, Q) with tube t on padded
    cells [offsets[t], offsets[t+1]) of every field (3 ghosts each end)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = np.exp(rng.uniform(math.log(lmin), math.log(lmax), size=ntubes))
    lens = np.clip(np.rint(lens).astype(np.int64), lmin, lmax)
    off = np.zeros(ntubes + 1, dtype=np.int64)
    off[1:] = np.cumsum(lens + 2 * NG)
    total = int(off[-1])
    Q = np.zeros((5, total))
    mats = [AIR, WATER]
    for t in range(ntubes):
        side = []
        for _ in range(2):
            rho = math.exp(rng.uniform(math.log(1.0), math.log(1000.0)))
            p = math.exp(rng.uniform(math.log(1.0e5), math.log(1.0e9)))
            m = mats[int(rng.integers(0, 2))]
            side.append([rho, 0.0, p, m])
        p_floor = max(-side[0][3][1], -side[1][3][1])
        cap = 0.0
        for s in side:
            g, pinf = s[3]
            c = math.sqrt(g * (s[2] + pinf) / s[0])
            cap += 2.0 * c / (g - 1.0) * (1.0 - ((p_floor + pinf) / (s[2] + pinf)) ** ((g - 1.0) / (2.0 * g)))
        while True:
            uL, uR = rng.uniform(-100.0, 100.0, size=2)
            if uR - uL < 0.5 * cap:
                break
        side[0][1], side[1][1] = uL, uR
        L = int(lens[t])
        a = int(off[t]) + NG
        half = L // 2
        for k, s in enumerate(side):
            lo, hi = (a, a + half) if k == 0 else (a + half, a + L)
            G, P = material(*s[3])
            Q[0, lo:hi] = s[0]
            Q[1, lo:hi] = s[1]
            Q[2, lo:hi] = s[2]
            Q[3, lo:hi] = G
            Q[4, lo:hi] = P
    return off, Q


def random_state(ndim: int, n, seed: int = 0, kind: str = "two_phase") -> Case:
    """Random test state on a small grid.
    kind: 'smooth'   smooth random fields, single fluid;
          'shock'    piecewise-constant random states with jumps, single fluid;
          'two_phase' random air/water blobs with strong jumps in rho, p, Gamma, Pi."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nn = tuple(int(n[d]) if d < ndim else 1 for d in range(3))
    h = tuple(1.0 / nn[d] if d < ndim else 1.0 for d in range(3))
    X, Y, Z = _centres(ndim, nn, (0.0, 0.0, 0.0), h)

    def smooth_field(base, amp):
        f = np.full(X.shape, base)
        for _ in range(3):
            k = rng.integers(1, 4, size=3)
            th = rng.uniform(0, 2 * math.pi)
            arg = k[0] * X + (k[1] * Y if ndim > 1 else 0) + (k[2] * Z if ndim > 2 else 0)
            f = f + amp * rng.uniform(0.2, 1.0) * np.sin(2 * math.pi * arg + th)
        return f

    Ga, Pa = material(*AIR)
    Gw, Pw = material(*WATER)
    if kind == "smooth":
        rho = smooth_field(1.0, 0.15)
        vel = [smooth_field(0.0, 0.3) for _ in range(ndim)]
        p = smooth_field(1.0, 0.15)
        G = np.full(X.shape, Ga)
        P = np.full(X.shape, Pa)
    elif kind == "shock":
        cells = 4
        lab = np.zeros(X.shape, dtype=np.int64)
        for d, A in enumerate((X, Y, Z)[:ndim]):
            lab = lab * cells + np.minimum((A * cells).astype(np.int64), cells - 1)
        nl = cells ** ndim
        rho = np.exp(rng.uniform(np.log(0.125), np.log(1.0), size=nl))[lab]
        vel = [rng.uniform(-0.5, 0.5, size=nl)[lab] for _ in range(ndim)]
        p = np.exp(rng.uniform(np.log(0.1), np.log(1.0), size=nl))[lab]
        G = np.full(X.shape, Ga)
        P = np.full(X.shape, Pa)
    elif kind == "two_phase":
        a = np.zeros(X.shape)
        for _ in range(3):
            c = rng.uniform(0.2, 0.8, size=3)
            R = rng.uniform(0.1, 0.3)
            r2 = (X - c[0]) ** 2 + ((Y - c[1]) ** 2 if ndim > 1 else 0) + ((Z - c[2]) ** 2 if ndim > 2 else 0)
            a = np.maximum(a, _volume_fraction(np.sqrt(r2), R, h[0]))
        rho = a * 1.0 + (1.0 - a) * 1000.0
        G = a * Ga + (1.0 - a) * Gw
        P = a * Pa + (1.0 - a) * Pw
        vel = [smooth_field(0.0, 20.0) for _ in range(ndim)]
        p = np.where(X > rng.uniform(0.3, 0.7), 1.0e9, 1.0e5) * np.exp(smooth_field(0.0, 0.05))
    else:
        raise ValueError(kind)
    Q = _fill(ndim, nn, [rho] + vel + [p, G, P])
    bcname = "periodic" if kind == "smooth" else "transmissive"
    bc = tuple((bcname, bcname) for _ in range(ndim))
    return Case(f"random_{kind}", ndim, nn, h, bc, Q, meta={"seed": seed})
