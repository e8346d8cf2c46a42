"""The synthetic inputs of the shock-interface setups of Secs. 6.1 and 6.2
against the Rankine-Hugoniot relations and the geometry the paper states.

The post-shock states are taken from the paper's tables as printed.  Their
density and pressure ratios follow from the stated Mach numbers; the printed
post-shock velocities correspond to a slightly larger pre-shock sound speed
than the printed pre-shock air (343 m/s for the Ms 1.22 air shock, 347 m/s for
the Ms 2.0 one), which is what these tests pin."""
import math

import numpy as np
import pytest

from paper_1707_00592_gb300 import workloads as wl


def rh(Ms, gamma, rho1, p1, c1=None):
    """Post-shock (rho, u, p) of a shock of Mach Ms running in -x into still
    ideal gas (P_inf = 0); c1 defaults to the gas's own sound speed."""
    c1 = math.sqrt(gamma * p1 / rho1) if c1 is None else c1
    ratio = (gamma + 1) * Ms * Ms / ((gamma - 1) * Ms * Ms + 2)
    p2 = p1 * (1 + 2 * gamma / (gamma + 1) * (Ms * Ms - 1))
    return rho1 * ratio, -Ms * c1 * (1 - 1 / ratio), p2


def post_state(case):
    Q = case.Q[wl.interior(2, case.n)][:, 0]
    return Q[0][0, -1], Q[1][0, -1], Q[3][0, -1]  # right-most column: behind the shock


@pytest.mark.parametrize("gas,rho_in,gamma_in", [("R22", 4.415, 1.249), ("He", 0.255, 1.648)])
def test_haas_sturtevant_states_and_geometry(gas, rho_in, gamma_in):
    case = wl.haas_sturtevant(gas, 267, 89)  # 1 mm cells
    rho2, u2, p2 = post_state(case)
    r, _, p = rh(1.22, 1.4, 1.4, 1.0e5)
    assert abs(rho2 / r - 1) < 1e-3 and abs(p2 / p - 1) < 2e-3
    _, u343, _ = rh(1.22, 1.4, 1.4, 1.0e5, c1=343.0)
    assert abs(u2 / u343 - 1) < 1e-3
    assert case.bc == (("transmissive", "transmissive"), ("reflective", "reflective"))
    assert case.dx[0] == pytest.approx(1e-3) and case.dx[1] == pytest.approx(1e-3)
    Q = case.Q[wl.interior(2, case.n)][:, 0]  # (field, y, x)
    G_in = 1 / (gamma_in - 1)
    frac = (Q[4] - 2.5) / (G_in - 2.5)  # cylinder volume fraction from Gamma
    assert frac.sum() * 1e-6 == pytest.approx(math.pi * 0.025 ** 2, rel=1e-2)
    yc, xc = ((np.indices(frac.shape) + 0.5) * 1e-3 * frac).reshape(2, -1).sum(axis=1) / frac.sum()
    assert abs(xc - 0.178) < 1e-4 and abs(yc - 0.0445) < 1e-4  # centroid of the cylinder
    assert Q[0].max() == pytest.approx(max(rho_in, 1.927))
    assert np.all(Q[5] == 0.0)  # P_inf = 0 everywhere: the single-phase limit


def test_shock_droplet_states_and_geometry():
    case = wl.shock_droplet(200)  # 0.1 mm cells
    rho2, u2, p2 = post_state(case)
    r, _, _ = rh(2.0, 1.4, 1.2, 1.0e5)
    assert abs(rho2 / r - 1) < 1e-3
    _, _, p_atm = rh(2.0, 1.4, 1.2, 101325.0)  # the printed 0.456 MPa follows from 1 atm
    assert abs(p2 / p_atm - 1) < 1e-3
    _, u347, _ = rh(2.0, 1.4, 1.2, 1.0e5, c1=347.2)
    assert abs(u2 / u347 - 1) < 1e-3
    Q = case.Q[wl.interior(2, case.n)][:, 0]  # (field, y, x)
    Gw, Pw = wl.material(4.34, 4.84e8)
    frac = Q[5] / Pw
    assert frac.sum() * 1e-8 == pytest.approx(math.pi * 0.004 ** 2, rel=1e-2)
    assert Q[0].max() == pytest.approx(1000.0)


def test_riemann_tubes_keep_clear_of_vacuum():
    """Every tube of the batched configuration (seed 0) has a star state of the
    exact stiffened-gas Riemann solution with both sides' p* + P_inf > 0, and
    its velocity spread stays below half of what would open a vacuum at the
    floor pressure (the exact solver's own wave functions at that pressure)."""
    from oracle import exact_riemann as er
    off, Q = wl.riemann_tubes(ntubes=4096, lmin=256, lmax=8192, seed=0)
    for t in range(len(off) - 1):
        a, b = off[t] + wl.NG, off[t + 1] - wl.NG - 1
        sides = []
        for i in (a, b):
            rho, u, p, G, P = Q[:, i]
            gamma = 1.0 + 1.0 / G
            sides.append(er.Side(rho, u, p, gamma, P / (G + 1.0)))
        L, R = sides
        floor = max(-L.pinf, -R.pinf)
        with np.errstate(divide="ignore"):  # the slope is infinite at the floor
            gain = -(er._f(floor, L)[0] + er._f(floor, R)[0])
        assert R.u - L.u < 0.5 * gain, t
        ps, _ = er.star_state(L, R)
        assert ps > floor, t
