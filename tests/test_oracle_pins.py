"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None re-types the oracle's formulas:
the expected values are textbook closed forms (WENO5 and 3rd-order linear
schemes, exact polynomial reconstruction, the eigen-structure of the
primitive Jacobian, the Euler flux, the exact Riemann solution), hand-worked
values stored under tests/golden/, or invariants (conservation, symmetry,
pressure-velocity equilibrium)."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact_riemann as er
from paper_1707_00592_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


# --------------------------------------------------------------------------
# Sec. 3.3.1: WENO-IS reconstruction

def test_linear_weights_recover_weno5():
    """With tau5/(beta+eps) -> 0 the weights are d = (4,2,3,1)/10 and the
    reconstruction must be the 5th-order linear scheme (2,-13,47,27,-3)/60
    (Jiang & Shu); this also fixes the sign of candidate 1."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        v = rng.normal(size=5)
        val, dbg = oracle.weno_is(v, eps=1e300)
        expect = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        assert abs(val - expect) <= 1e-14 * (1 + np.abs(v).max())
        # alpha_k = d_k exactly (integers 4, 2, 3, 1)
        np.testing.assert_allclose(dbg[6:10], [4, 2, 3, 1], rtol=0, atol=1e-200)


def test_third_order_degeneration():
    """End of Sec. 3.3.1: d3 = d4 = 0 gives the 3rd-order scheme (-1, 5, 2)/6."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        v = rng.normal(size=5)
        val, _ = oracle.weno_is(v, eps=1e300, order=3)
        expect = (-v[1] + 5 * v[2] + 2 * v[3]) / 6.0
        assert abs(val - expect) <= 1e-14 * (1 + np.abs(v).max())


def test_quadratic_data_exact():
    """Any quadratic has tau5 = 0 exactly, so the weights are linear and the
    reconstruction of its cell averages is the exact face value."""
    # cell averages of x^2 over [j-1/2, j+1/2] are j^2 + 1/12; face x = 1/2
    v = np.array([j * j + 1.0 / 12.0 for j in range(-2, 3)])
    val, dbg = oracle.weno_is(v)
    assert dbg[5] == 0.0
    assert abs(val - 0.25) <= 2e-16
    rng = np.random.default_rng(3)
    for _ in range(100):
        a, b, c = rng.integers(-5, 6, size=3).astype(float)
        # averages of a x^2 + b x + c over unit cells centred on the integers
        v = np.array([a * (j * j + 1.0 / 12.0) + b * j + c for j in range(-2, 3)])
        val, dbg = oracle.weno_is(v)
        exact = a * 0.25 + b * 0.5 + c
        assert dbg[5] <= 1e-28  # zero up to the rounding of 1/12
        assert abs(val - exact) <= 1e-13 * (1 + abs(exact))


def test_tau5_on_cubic_and_quartic():
    """Eq. (tau-5) on point data j^3 and j^4 (j = -2..2): 36 and 624 by hand."""
    _, d3 = oracle.weno_is(np.array([float(j ** 3) for j in range(-2, 3)]))
    _, d4 = oracle.weno_is(np.array([float(j ** 4) for j in range(-2, 3)]))
    assert d3[5] == 36.0
    assert d4[5] == 624.0


def test_step_stencil_hand_values():
    """Hand-worked beta, beta12, tau5, alpha on the step 0 0 0 1 1 (1)."""
    g = read_golden("weno_is_step_stencil.txt")
    val, dbg = oracle.weno_is(np.array([0.0, 0.0, 0.0, 1.0, 1.0]))
    names = ["beta1", "beta2", "beta3", "beta4", "beta12", "tau5"]
    for k, nm in enumerate(names):
        assert dbg[k] == pytest.approx(g[nm], rel=1e-15, abs=0)
    assert dbg[6] == pytest.approx(g["alpha1"], rel=1e-14)
    assert dbg[8] == pytest.approx(g["alpha3"], rel=1e-14)
    assert abs(val - g["left"]) < 1e-30
    # right state at x_{i+1/2}: mirror stencil q_{i+3}, q_{i+2}, q_{i+1}, q_i, q_{i-1}
    valr, _ = oracle.weno_is(np.array([1.0, 1.0, 1.0, 0.0, 0.0]))
    assert abs(valr - g["right"]) < 1e-30


def test_basic_weights_hand_values():
    """Sec. 3.3.1, Eq. (weight-new) with q = 1 (the basic weights): alpha_1..alpha_4
    and the face value on the step stencil worked by hand with eps = 1; the
    modified weights of Eq. (weighting-modification) give another alpha_1 there."""
    g = read_golden("weno_basic_weights_step.txt")
    step = np.array([0.0, 0.0, 0.0, 1.0, 1.0])
    val, dbg = oracle.weno_is(step, eps=1.0, weights="basic")
    for k, nm in enumerate(["alpha1", "alpha2", "alpha3", "alpha4"]):
        assert dbg[6 + k] == pytest.approx(g[nm], rel=1e-15)
    assert val == pytest.approx(g["value"], rel=1e-15)
    # 3rd-order level (d3 = d4 = 0): (alpha1 q1 + alpha2 q2)/(alpha1 + alpha2) = 12/46
    val3, _ = oracle.weno_is(step, eps=1.0, order=3, weights="basic")
    assert val3 == pytest.approx(12.0 / 46.0, rel=1e-15)
    _, dbg_m = oracle.weno_is(step, eps=1.0, weights="modified")
    assert dbg_m[6] == pytest.approx(628.0 / 7.0, rel=1e-15)


def test_basic_weights_in_the_scheme():
    """Sec. 3.3.2: with the basic weights the 2-point candidates take too much
    weight near critical points of smooth data, where beta_1 or beta_2 are
    small, and the scheme falls to about 2nd order; the modified weights keep
    5th order on the same wave (test_convergence_1d_entropy_wave).  The sine
    wave has two critical points."""
    errs = []
    for n in (20, 40, 80):
        case = wl.entropy_wave(n, 1, amp=0.2, kind="sine")
        g = oracle.Grid(1, case.n, case.dx, case.bc, mood=False, weights="basic")
        h = 1.0 / n
        U = _fixed_dt_run(g, _U(case), 0.25, 0.5 * h ** (5.0 / 3.0))
        x = (np.arange(n) + 0.5) * h
        ex = 1.0 + 0.2 * np.sin(2 * np.pi * (x - 0.25)) * np.sin(np.pi * h) / (np.pi * h)
        errs.append(np.abs(U[0, 0, 0, 3:3 + n] - ex).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert max(orders) < 3.0, (errs, orders)


# --------------------------------------------------------------------------
# The comparison scheme WENO-JS (Jiang & Shu 1996; Secs. 5 and 6 compare with it)

def test_js_linear_weights_recover_weno5():
    """With eps >> beta the WENO-JS weights are d = (1, 6, 3)/10 and the face
    value is the 5th-order linear scheme (2, -13, 47, 27, -3)/60."""
    rng = np.random.default_rng(21)
    for _ in range(200):
        v = rng.normal(size=5)
        val, dbg = oracle.weno_is(v, eps=1e100, weights="js")
        expect = (2 * v[0] - 13 * v[1] + 47 * v[2] + 27 * v[3] - 3 * v[4]) / 60.0
        assert abs(val - expect) <= 1e-14 * (1 + np.abs(v).max())
        np.testing.assert_allclose(dbg[6:9] * 1e200, [1.0, 6.0, 3.0], rtol=1e-12)


def test_js_step_stencil_hand_values():
    """WENO-JS on the step 0 0 0 1 1 (1), eps = 1e-6, power 2: hand-worked
    indicators, weights and face values."""
    g = read_golden("weno_js_step_stencil.txt")
    val, dbg = oracle.weno_is(np.array([0.0, 0.0, 0.0, 1.0, 1.0]), weights="js")
    for k, nm in enumerate(["beta0", "beta1", "beta2"]):
        assert dbg[k] == pytest.approx(g[nm], rel=1e-15, abs=0)
    for k, nm in enumerate(["alpha0", "alpha1", "alpha2"]):
        assert dbg[6 + k] == pytest.approx(g[nm], rel=1e-14)
    assert val == pytest.approx(g["left"], rel=1e-12)
    valr, _ = oracle.weno_is(np.array([1.0, 1.0, 1.0, 0.0, 0.0]), weights="js")
    assert valr - 1.0 == pytest.approx(g["right_minus_one"], abs=2e-16)


def test_js_third_order_level():
    """Reading: under MOOD, the 3rd-order level of WENO-JS is the scheme's own
    (2-point candidates, modified weights, d3 = d4 = 0)."""
    rng = np.random.default_rng(22)
    for _ in range(50):
        v = rng.normal(size=5)
        a, _ = oracle.weno_is(v, eps=1e-6, order=3, weights="js")
        b, _ = oracle.weno_is(v, eps=1e-6, order=3, weights="modified")
        assert a == b


def test_js_whole_scheme_fifth_order():
    """The WENO-JS option in the whole scheme: 5th order on the smooth entropy wave."""
    errs = []
    for n in (20, 40, 80):
        case = wl.entropy_wave(n, 1, amp=0.2, kind="sine")
        g = oracle.Grid(1, case.n, case.dx, case.bc, mood=False, weights="js")
        h = 1.0 / n
        U = _fixed_dt_run(g, _U(case), 0.25, 0.5 * h ** (5.0 / 3.0))
        x = (np.arange(n) + 0.5) * h
        ex = 1.0 + 0.2 * np.sin(2 * np.pi * (x - 0.25)) * np.sin(np.pi * h) / (np.pi * h)
        errs.append(np.abs(U[0, 0, 0, 3:3 + n] - ex).mean())
    assert math.log2(errs[1] / errs[2]) > 4.5, errs


def test_weno_is_order_of_accuracy_pointwise():
    """Reconstruction error on a smooth function at fixed position falls as h^5
    (Sec. 3.3.1: tau5/(beta+eps) = O(h^(6-r)) keeps 5th order), including at a
    critical point, which the modification of Sec. 3.3.2 is designed for."""
    def err(h, x0):
        j = np.arange(-2, 3)
        # exact cell averages of sin(x) over [x0 + (j-1/2)h, x0 + (j+1/2)h]
        lo = x0 + (j - 0.5) * h
        hi = x0 + (j + 0.5) * h
        avg = (np.cos(lo) - np.cos(hi)) / h
        val, _ = oracle.weno_is(avg)
        return abs(val - math.sin(x0 + 0.5 * h))
    for x0 in (0.3, math.pi / 2 - 0.5 * 0.0):  # generic point and a critical point
        hs = [0.1, 0.05, 0.025]
        e = [err(h, x0) for h in hs]
        orders = [math.log(e[k] / e[k + 1], 2) for k in range(2)]
        assert min(orders) > 4.5, (x0, e, orders)


# --------------------------------------------------------------------------
# Sec. 3.2: characteristic decomposition

@pytest.mark.parametrize("nq", [5, 6, 7])
def test_eigenvectors_diagonalise_primitive_jacobian(nq):
    """L A R = diag(u-c, u.., u+c) and L R = I for the Jacobian A of
    Eq. (primitive-variable) (extended to nq = ndim + 4 primitives)."""
    rng = np.random.default_rng(nq)
    for _ in range(20):
        rho, c, u = rng.uniform(0.5, 2.0), rng.uniform(0.5, 3.0), rng.uniform(-1, 1)
        Lm, Rm = oracle.char_matrices(nq, rho, c)
        nt = nq - 5
        ip = 2 + nt
        A = np.eye(nq) * u
        A[0, 1] = rho
        A[1, ip] = 1.0 / rho
        A[ip, 1] = rho * c * c
        np.testing.assert_allclose(Lm @ Rm, np.eye(nq), atol=1e-15)
        lam = np.full(nq, u)
        lam[0] = u - c
        lam[-1] = u + c
        np.testing.assert_allclose(Lm @ A @ Rm, np.diag(lam), atol=1e-13)


# --------------------------------------------------------------------------
# Sec. 3.2.1: HLLC

def euler_flux(q):
    """Eq. (governing-equation) flux plus phi u for Gamma and Pi, sweep frame."""
    nq = q.size
    nt = nq - 5
    rho, un, p, G, P = q[0], q[1], q[2 + nt], q[3 + nt], q[4 + nt]
    ut = q[2:2 + nt]
    E = G * p + P + 0.5 * rho * (un * un + np.sum(ut * ut))
    return np.concatenate([[rho * un, rho * un * un + p], rho * un * ut, [(E + p) * un, G * un, P * un]])


@pytest.mark.parametrize("nq", [5, 6, 7])
def test_hllc_consistency(nq):
    """F_hat(q, q) = F(q) and u_HLLC = u for any admissible state."""
    rng = np.random.default_rng(10 + nq)
    for _ in range(100):
        q = np.empty(nq)
        q[0] = rng.uniform(0.1, 1000)
        q[1:nq - 3] = rng.uniform(-300, 300, size=nq - 4)
        G, P = wl.material(*(wl.AIR if rng.random() < 0.5 else wl.WATER))
        q[nq - 3] = rng.uniform(1e4, 1e9)
        q[nq - 2], q[nq - 1] = G, P
        F, us = oracle.hllc(q, q)
        np.testing.assert_allclose(F, euler_flux(q), rtol=1e-12, atol=1e-9 * np.abs(euler_flux(q)).max())
        assert us == pytest.approx(q[1], rel=1e-12, abs=1e-12)


def test_hllc_supersonic_upwinding_and_rest():
    """All waves moving right => F_hat = F(q_l); quiescent equal pressures => zero mass flux."""
    G, P = wl.material(*wl.AIR)
    ql = np.array([1.0, 10.0, 0.3, 1.0, G, P])
    qr = np.array([0.5, 12.0, -0.2, 0.8, G, P])
    F, us = oracle.hllc(ql, qr)
    np.testing.assert_allclose(F, euler_flux(ql), rtol=1e-13)
    ql = np.array([1000.0, 0.0, 0.0, 1e5, *wl.material(*wl.WATER)])
    qr = np.array([1.0, 0.0, 0.0, 1e5, *wl.material(*wl.AIR)])
    F, us = oracle.hllc(ql, qr)
    assert F[0] == 0.0 and us == 0.0
    assert F[1] == pytest.approx(1e5, rel=1e-14)


def test_hllc_wave_speeds_hand_values():
    """Eqs. (wave-speeds), (wave-speed), (flux-function), (hllc-flux) and
    (velocities) on a subsonic two-material face (S_l < 0 < S_r, u_l != u_r),
    worked by hand: Roe u_bar, the Einfeldt c2_bar, S_l, S_r, S*, the flux and
    the face velocity.  A printed typo in u_bar or c2_bar, or a dropped Einfeldt
    term, changes S_l and S_r and hence S* and every flux component."""
    g = read_golden("hllc_subsonic_face.txt")
    # gamma 2, P_inf 1 and gamma 1.4, P_inf 0: Gamma = 1/(gamma-1), Pi = gamma P_inf/(gamma-1)
    G_l, P_l, G_r, P_r = 1.0, 2.0, 2.5, 0.0
    ql = np.array([4.0, 1.0, 10.0, G_l, P_l])
    qr = np.array([1.0, -2.0, 5.0, G_r, P_r])
    F, us, w = oracle.hllc_waves(ql, qr)
    assert w[0] == pytest.approx(g["u_bar"], abs=1e-15)
    assert w[1] == pytest.approx(g["c2_bar"], rel=1e-15)
    for k, nm in ((2, "S_l"), (3, "S_r"), (4, "S_star")):
        assert w[k] == pytest.approx(g[nm], rel=1e-14), nm
    for m, nm in enumerate(["F_rho", "F_mom", "F_E", "F_Gamma", "F_Pi"]):
        assert F[m] == pytest.approx(g[nm], rel=1e-14), nm
    assert us == pytest.approx(g["u_star"], rel=1e-14)
    # the same face with a tangential velocity (nq = 6): the five fluxes are
    # unchanged and the tangential flux is the mass flux times the upwind v
    ql6 = np.array([4.0, 1.0, 0.5, 10.0, G_l, P_l])
    qr6 = np.array([1.0, -2.0, -0.25, 5.0, G_r, P_r])
    F6, us6, w6 = oracle.hllc_waves(ql6, qr6)
    np.testing.assert_allclose(w6[2:], w[2:], rtol=1e-15)
    np.testing.assert_allclose(F6[[0, 1, 4, 5]], F[[0, 1, 3, 4]], rtol=1e-14)
    assert F6[2] == pytest.approx(g["F_rho"] * 0.5, rel=1e-14)


def test_hllc_contact_speed_weak_waves():
    """Weak two-state problems (jumps of 1e-3): S_l < S* < S_r, and S* is the
    exact stiffened-gas solution's contact velocity to within the jump's size."""
    rng = np.random.default_rng(31)
    for _ in range(20):
        gam, pinf = (wl.AIR if rng.random() < 0.5 else wl.WATER)
        G, P = wl.material(gam, pinf)
        rho = 1.0 if gam == wl.AIR[0] else 1000.0
        p = 1.0e5
        c = math.sqrt(gam * (p + pinf) / rho)
        u = rng.uniform(-0.5, 0.5) * c
        d = 1e-3
        sides = []
        for k in range(2):
            sides.append((rho * (1 + d * rng.normal()), u + d * c * rng.normal(), p * (1 + d * rng.normal())))
        ql = np.array([sides[0][0], sides[0][1], sides[0][2], G, P])
        qr = np.array([sides[1][0], sides[1][1], sides[1][2], G, P])
        _, _, w = oracle.hllc_waves(ql, qr)
        ps, ust = er.star_state(er.Side(*sides[0], gam, pinf), er.Side(*sides[1], gam, pinf))
        assert w[2] < w[4] < w[3]
        assert abs(w[4] - ust) <= 1e-3 * c


def test_hllc_mirrored_states_zero_mass_flux():
    """A face between a state and its mirror image (u_n negated), as at a
    reflective wall: S* = 0, so no mass, Gamma or Pi crosses the face and the
    face velocity is 0, exactly."""
    rng = np.random.default_rng(32)
    for _ in range(100):
        G, P = wl.material(*(wl.AIR if rng.random() < 0.5 else wl.WATER))
        q = np.array([rng.uniform(0.5, 1000), rng.uniform(-300, 300), rng.uniform(-50, 50),
                      rng.uniform(1e4, 1e9), G, P])
        m = q.copy()
        m[1] = -m[1]
        F, us, w = oracle.hllc_waves(m, q)
        assert w[4] == 0.0 and us == 0.0
        assert F[0] == 0.0 and F[4] == 0.0 and F[5] == 0.0


# --------------------------------------------------------------------------
# exact Riemann solver (test-side reference)

def test_exact_riemann_toro_sod():
    g = read_golden("toro_sod_star.txt")
    ps, us = er.star_state(er.Side(1.0, 0.0, 1.0, 1.4, 0.0), er.Side(0.125, 0.0, 0.1, 1.4, 0.0))
    assert ps == pytest.approx(g["p_star"], abs=6e-6)
    assert us == pytest.approx(g["u_star"], abs=6e-6)


def test_exact_riemann_stiffened_jump_conditions():
    """Gas-water tube: the air-side shock satisfies the Rankine-Hugoniot
    conditions of the stiffened gas; pressure and velocity are continuous at
    the contact."""
    L = er.Side(1000.0, 0.0, 1e9, 4.4, 6e8)
    R = er.Side(50.0, 0.0, 1e5, 1.4, 0.0)
    ps, us = er.star_state(L, R)
    g = R.gamma
    S = R.u + R.c * math.sqrt((g + 1) / (2 * g) * (ps + R.pinf) / R.pbar + (g - 1) / (2 * g))
    rho_s, u_s, p_s, _ = er.sample(L, R, np.array([S - 1e-9 * abs(S)]))
    rho_s, u_s, p_s = rho_s[0], u_s[0], p_s[0]
    m1 = R.rho * (R.u - S)
    m2 = rho_s * (u_s - S)
    assert m1 == pytest.approx(m2, rel=1e-10)
    assert R.rho * R.u * (R.u - S) + R.p == pytest.approx(rho_s * u_s * (u_s - S) + p_s, rel=1e-10)
    e = lambda r, u, p, s: (p + s.gamma * s.pinf) / (s.gamma - 1) + 0.5 * r * u * u
    assert (e(R.rho, R.u, R.p, R) + R.p) * R.u - S * e(R.rho, R.u, R.p, R) == pytest.approx(
        (e(rho_s, u_s, p_s, R) + p_s) * u_s - S * e(rho_s, u_s, p_s, R), rel=1e-9)
    rl, ul_, pl_, _ = er.sample(L, R, np.array([us - 1e-6]))
    rr, ur_, pr_, _ = er.sample(L, R, np.array([us + 1e-6]))
    assert pl_[0] == pytest.approx(pr_[0], rel=1e-12) and ul_[0] == pytest.approx(ur_[0], rel=1e-12)


# --------------------------------------------------------------------------
# whole scheme

def _grid(case, **kw):
    return oracle.Grid(case.ndim, case.n, case.dx, case.bc, **kw)


def _U(case):
    return oracle.prim_to_cons(case.ndim, case.Q)


def test_gas_water_tube_converges_to_exact():
    """Sec. 5.2 style gas-liquid shock tube: L1(rho) against the exact
    stiffened-gas solution decreases under refinement and is small at N = 200."""
    errs = []
    for n in (100, 200, 400):
        case = wl.gas_water_tube(n)
        g = _grid(case)
        U, t, k = oracle.run(g, _U(case), case.t_end)
        L = er.Side(*case.meta["left"])
        R = er.Side(*case.meta["right"])
        edges = np.linspace(0.0, 1.0, n + 1)
        rho_ex, _, _ = er.cell_averages(L, R, case.meta["x0"], t, edges, sub=16)
        rho = U[0, 0, 0, 3:3 + n]
        errs.append(np.abs(rho - rho_ex).sum() / n)
        assert oracle.count_nonphysical(g, U) == 0
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / np.abs(rho_ex).mean() < 0.02


def test_interface_transport_equilibrium():
    """Sec. 5.1: a gas/liquid interface advected at uniform p, u keeps p and u
    uniform to round-off (the paper reports errors at the 1e-12 scale).  In the
    liquid E ~ 8.5e3 while Gamma p ~ 0.17, so recovering p from E loses about
    five digits per step: the bound on p is 1e-9, on u 1e-12."""
    case = wl.interface_transport(200)
    g = _grid(case)
    U, t, k = oracle.run(g, _U(case), case.t_end)
    Q = oracle.cons_to_prim(1, U)[:, 0, 0, 3:-3]
    assert k > 100
    assert np.abs(Q[2] - 1.0).max() < 1e-9
    assert np.abs(Q[1] - 100.0).max() / 100.0 < 1e-12


def test_drop_equilibrium_2d():
    """2D analogue: a smeared water drop advected diagonally in air at uniform
    p, u keeps p and u uniform (both directions' Gamma/Pi source terms)."""
    case = wl.random_state(2, (24, 24), seed=4, kind="two_phase")
    Q0 = case.Q.copy()
    Q0[1] = 0.0
    Q0[2] = 0.0
    sl = wl.interior(2, case.n)
    Q0[(1,) + sl[1:]] = 30.0
    Q0[(2,) + sl[1:]] = -20.0
    Q0[(3,) + sl[1:]] = 1e5
    g = oracle.Grid(2, case.n, case.dx, (("periodic", "periodic"),) * 2)
    U = oracle.prim_to_cons(2, Q0)
    for _ in range(20):
        U, _, _ = oracle.step(g, U)
    Q = oracle.cons_to_prim(2, U)[sl]
    assert np.abs(Q[3] / 1e5 - 1.0).max() < 1e-10
    assert np.abs(Q[1] / 30.0 - 1.0).max() < 1e-10
    assert np.abs(Q[2] / -20.0 - 1.0).max() < 1e-10


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_conservation_periodic(ndim):
    """Sec. 3.1: the flux form conserves rho, rho u_i and E exactly up to round-off
    on a periodic box."""
    n = (32, 16, 8)[ndim - 1]
    case = wl.random_state(ndim, (n,) * ndim, seed=ndim, kind="smooth")
    g = oracle.Grid(ndim, case.n, case.dx, case.bc)
    U = _U(case)
    sl = wl.interior(ndim, case.n)
    s0 = U[sl].reshape(case.nv, -1).sum(axis=1)
    for _ in range(5):
        U, _, _ = oracle.step(g, U)
    s1 = U[sl].reshape(case.nv, -1).sum(axis=1)
    for f in range(ndim + 2):
        scale = np.abs(U[(f,) + sl[1:]]).sum()
        assert abs(s1[f] - s0[f]) <= 1e-13 * scale


def _doubled(Q, ndim, axis_field):
    """The state mirrored about its low wall along the last active axis (the
    normal momentum component negated), followed by the state itself."""
    ax = {1: 3, 2: 2}[ndim]
    sl = [slice(None)] * 4
    inner = Q.copy()
    m = np.flip(inner, axis=ax).copy()
    m[axis_field] *= -1.0
    return np.concatenate([m, inner], axis=ax)


@pytest.mark.parametrize("ndim", [1, 2])
def test_reflective_walls_equal_doubled_periodic_domain(ndim):
    """Sec. 6.1 reflective (slip) walls: a box with walls on both ends of an
    axis advances exactly as the periodic box of twice the length that holds
    the state and its mirror image (normal velocity negated) -- the ghost cells
    of a wall are the mirror cells of that doubled box.  Bit for bit, dt
    included; this pins the reflective ghost fill against the periodic one."""
    n = (24,) if ndim == 1 else (12, 10)
    case = wl.random_state(ndim, n, seed=40 + ndim, kind="two_phase")
    sl = wl.interior(ndim, case.n)
    Qi = case.Q[sl]                     # interior primitives [f, z, y, x]
    d = ndim - 1                        # the walled axis: x in 1D, y in 2D
    bc = [("transmissive", "transmissive")] * ndim
    bc[d] = ("reflective", "reflective")
    g = oracle.Grid(ndim, case.n, case.dx, tuple(bc))
    n2 = list(case.n[:ndim])
    n2[d] *= 2
    bc2 = list(bc)
    bc2[d] = ("periodic", "periodic")
    g2 = oracle.Grid(ndim, tuple(n2), case.dx, tuple(bc2))
    Q2 = wl._fill(ndim, tuple(n2), list(_doubled(Qi, ndim, 1 + d)))
    U1, dt1, _ = oracle.step(g, _U(case))
    U2, dt2, _ = oracle.step(g2, oracle.prim_to_cons(ndim, Q2))
    assert dt1 == dt2
    sl2 = wl.interior(ndim, tuple(n2))
    half = [slice(None)] * 4
    ax = {1: 3, 2: 2}[ndim]
    half[ax] = slice(n[d], 2 * n[d])
    assert np.array_equal(U1[sl], U2[sl2][tuple(half)])


def test_reflective_box_conserves_mass_and_energy():
    """No mass or energy crosses a reflective wall: in a box walled on all sides
    the totals of rho and E change only by round-off over a step."""
    case = wl.random_state(2, (14, 12), seed=44, kind="two_phase")
    g = oracle.Grid(2, case.n, case.dx, (("reflective", "reflective"),) * 2)
    U = _U(case)
    sl = wl.interior(2, case.n)
    s0 = U[sl].reshape(case.nv, -1).sum(axis=1)
    for _ in range(3):
        U, _, _ = oracle.step(g, U)
    s1 = U[sl].reshape(case.nv, -1).sum(axis=1)
    for f in (0, 3):
        assert abs(s1[f] - s0[f]) <= 1e-13 * np.abs(U[(f,) + sl[1:]]).sum()


def test_mirror_symmetry_1d():
    """Reflecting x -> -x (u -> -u) commutes with a step (to round-off): pins the
    mirror stencil of the right state and the HLLC orientation."""
    case = wl.random_state(1, (64,), seed=7, kind="shock")
    g = oracle.Grid(1, case.n, case.dx, case.bc)
    Q = case.Q
    Qm = Q[:, :, :, ::-1].copy()
    Qm[1] *= -1
    U1, _, _ = oracle.step(g, oracle.prim_to_cons(1, Q), dt=1e-3)
    U2, _, _ = oracle.step(g, oracle.prim_to_cons(1, Qm), dt=1e-3)
    U2 = U2[:, :, :, ::-1].copy()
    U2[1] *= -1
    sl = wl.interior(1, case.n)
    for f in range(5):
        a, b = U1[(f,) + sl[1:]], U2[(f,) + sl[1:]]
        assert np.abs(a - b).max() <= 1e-12 * (np.abs(a).max() + 1e-300)


@pytest.mark.parametrize("ndim", [2, 3])
def test_axis_swap_symmetry_bitwise(ndim):
    """Swapping x and y (with u and v) gives the swapped result bit for bit: the
    y sweep does the x sweep's arithmetic in its own frame."""
    n = (12, 10, 8)
    case = wl.random_state(ndim, n, seed=11, kind="two_phase")
    g = oracle.Grid(ndim, case.n, case.dx, case.bc)
    # transpose the two innermost axes (y, x) and swap u, v
    Q = case.Q
    n2 = (n[1], n[0], n[2])
    Qs = np.swapaxes(Q, -1, -2).copy()
    Qs[[1, 2]] = Qs[[2, 1]]
    gs = oracle.Grid(ndim, n2, (case.dx[1], case.dx[0], case.dx[2]), case.bc)
    U1, _, _ = oracle.step(g, oracle.prim_to_cons(ndim, Q), dt=2e-7)
    U2, _, _ = oracle.step(gs, oracle.prim_to_cons(ndim, Qs), dt=2e-7)
    U2 = np.swapaxes(U2, -1, -2).copy()
    U2[[1, 2]] = U2[[2, 1]]
    sl = wl.interior(ndim, case.n)
    assert np.array_equal(U1[sl], U2[sl])


def _fixed_dt_run(g, U, t_end, dt):
    nsteps = int(math.ceil(t_end / dt - 1e-9))
    dt = t_end / nsteps
    for _ in range(nsteps):
        U, _, _ = oracle.step(g, U, dt=dt)
    return U


def test_convergence_1d_entropy_wave():
    """Sec. 4.1 style order test: a smooth density wave advected by the full
    Euler scheme with dt = 0.5 dx^(5/3); the L1 error of rho falls at 5th order."""
    errs = []
    ns = (20, 40, 80)
    t_end = 0.25
    for n in ns:
        case = wl.entropy_wave(n, 1, amp=0.2, kind="sine")
        g = oracle.Grid(1, case.n, case.dx, case.bc, mood=False)
        h = 1.0 / n
        U = _fixed_dt_run(g, _U(case), t_end, 0.5 * h ** (5.0 / 3.0))
        x = (np.arange(n) + 0.5) * h
        # exact cell averages of 1 + 0.2 sin(2 pi (x - t))
        ex = 1.0 + 0.2 * np.sin(2 * np.pi * (x - t_end)) * np.sin(np.pi * h) / (np.pi * h)
        errs.append(np.abs(U[0, 0, 0, 3:3 + n] - ex).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(ns) - 1)]
    assert orders[-1] > 4.5, (errs, orders)


@pytest.mark.slow
def test_convergence_2d_entropy_wave():
    """Sec. 4.2 style: diagonal wave in 2D, 5th order in L1."""
    errs = []
    ns = (12, 24, 48)
    t_end = 0.1
    for n in ns:
        case = wl.entropy_wave(n, 2, amp=0.2, kind="sine")
        g = oracle.Grid(2, case.n, case.dx, case.bc, mood=False)
        h = 1.0 / n
        U = _fixed_dt_run(g, _U(case), t_end, 0.5 * h ** (5.0 / 3.0))
        x = (np.arange(n) + 0.5) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        f = (np.sin(np.pi * h) / (np.pi * h)) ** 2
        ex = 1.0 + 0.2 * np.sin(2 * np.pi * (X + Y - 2 * t_end)) * f
        errs.append(np.abs(U[0, 0, 3:3 + n, 3:3 + n] - ex).mean())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(len(ns) - 1)]
    assert orders[-1] > 4.5, (errs, orders)


# --------------------------------------------------------------------------
# Sec. 3.4: MOOD cascade

def _two_phase_stencil(rng):
    """Six cells across a violent air/water jump, sweep frame (rho, u, v, p, G, P)."""
    Gw, Pw = wl.material(*wl.WATER)
    Ga, Pa = wl.material(*wl.AIR)
    qc = np.zeros((6, 6))
    k = rng.integers(1, 5)
    for j in range(6):
        water = (j < k) if rng.random() < 0.5 else (j >= k)
        qc[j] = [1000.0 if water else rng.uniform(1e-3, 1.0), rng.uniform(-500, 500), rng.uniform(-50, 50),
                 rng.choice([1e5, 1e9]) * rng.uniform(0.5, 2), Gw if water else Ga, Pw if water else Pa]
    cc = np.array([oracle.sound_speed(q[0], q[3], q[4], q[5]) for q in qc])
    return qc, cc


def test_mood_cascade_levels():
    """Each side ends admissible with MOOD on; level 1 is exactly the upwind
    cell's primitive state; level 3 is the reconstruction with d3 = d4 = 0; a
    side that MOOD lowered is inadmissible without MOOD."""
    rng = np.random.default_rng(5)
    seen = set()
    for _ in range(3000):
        qc, cc = _two_phase_stencil(rng)
        F, us, lev, qlr = oracle.face(qc, cc, mood=True)
        F0, us0, lev0, qlr0 = oracle.face(qc, cc, mood=False)
        assert lev0 == (5, 5)
        for side in range(2):
            q = qlr[side]
            assert q[0] > 0 and q[4] > 0 and (q[4] + 1) * q[3] + q[5] > 0
            seen.add(lev[side])
            if lev[side] == 5:
                np.testing.assert_array_equal(qlr[side], qlr0[side])
            else:
                q0 = qlr0[side]
                assert not (q0[0] > 0 and q0[4] > 0 and (q0[4] + 1) * q0[3] + q0[5] > 0)
            if lev[side] == 1:
                np.testing.assert_array_equal(q, qc[2 + side])
            if lev[side] == 3:
                rho_bar = 0.5 * (qc[2, 0] + qc[3, 0])
                c_bar = 0.5 * (cc[2] + cc[3])
                Lm, Rm = oracle.char_matrices(6, rho_bar, c_bar)
                w = qc @ Lm.T
                st = w[0:5] if side == 0 else w[5:0:-1]
                wt = np.array([oracle.weno_is(st[:, r], order=3)[0] for r in range(6)])
                np.testing.assert_allclose(q, Rm @ wt, rtol=1e-12, atol=1e-12 * np.abs(q).max())
    assert {3, 1} <= seen, seen


def test_mood_quiet_on_smooth_data():
    rng = np.random.default_rng(6)
    G, P = wl.material(*wl.AIR)
    for _ in range(200):
        x = np.arange(6) * 0.05
        qc = np.stack([1 + 0.3 * np.sin(x + rng.random()), 0.2 * np.cos(x), 0.1 * x, 1 + 0.2 * np.sin(2 * x),
                       np.full(6, G), np.full(6, P)], axis=1)
        cc = np.array([oracle.sound_speed(q[0], q[3], q[4], q[5]) for q in qc])
        _, _, lev, _ = oracle.face(qc, cc)
        assert lev == (5, 5)


# --------------------------------------------------------------------------
# Sec. 4 (time step): dt = CFL / max over cells of sum_d (|u_d| + c) / dx_d

def _sound_speed(rho, p, gamma, pinf):
    """Stiffened-gas sound speed from its definition, c^2 = gamma (p + P_inf) / rho."""
    return np.sqrt(gamma * (p + pinf) / rho)


def test_cfl_dt_uniform_state_closed_form():
    n, dx = (12, 9), (1.0 / 12, 1.0 / 9)
    gamma, pinf = wl.WATER
    G, P = wl.material(gamma, pinf)
    shape = (n[1], n[0])
    Q = wl._fill(2, n, [np.full(shape, 1000.0), np.full(shape, 3.0), np.full(shape, -2.0),
                        np.full(shape, 1.0e5), np.full(shape, G), np.full(shape, P)])
    g = oracle.Grid(2, n, dx, (("periodic", "periodic"),) * 2)
    c = _sound_speed(1000.0, 1.0e5, gamma, pinf)
    expect = 0.5 / ((3.0 + c) / dx[0] + (2.0 + c) / dx[1])
    assert oracle.cfl_dt(g, oracle.prim_to_cons(2, Q)) == pytest.approx(expect, rel=1e-13)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_cfl_dt_is_the_maximum_over_cells(ndim):
    """Brute force over the cells of a random two-phase state, with the sound
    speed from gamma = 1 + 1/Gamma and P_inf = Pi / (Gamma + 1)."""
    n = (40, 24, 10)[:ndim]
    case = wl.random_state(ndim, n, seed=11 + ndim, kind="two_phase")
    g = oracle.Grid(ndim, case.n, case.dx, case.bc)
    sl = wl.interior(ndim, case.n)
    Q = case.Q[sl].reshape(case.nv, -1)
    rho, vel, p, G, P = Q[0], Q[1:1 + ndim], Q[1 + ndim], Q[2 + ndim], Q[3 + ndim]
    c = _sound_speed(rho, p, 1.0 + 1.0 / G, P / (G + 1.0))
    rate = sum((np.abs(vel[d]) + c) / case.dx[d] for d in range(ndim))
    expect = 0.5 / rate.max()
    assert oracle.cfl_dt(g, oracle.prim_to_cons(ndim, case.Q)) == pytest.approx(expect, rel=1e-10)
    # raising the pressure of the cell that sets the step (p -> 4p) raises only
    # its sound speed: the step follows that cell's new rate
    k = int(np.argmax(rate))
    Q2 = case.Q.copy()
    idx = np.unravel_index(k, case.Q[sl][0].shape)
    full = tuple((s.start or 0) + i for s, i in zip(sl[1:], idx))
    Q2[(1 + ndim,) + full] *= 4.0  # p -> 4p raises c at that cell only
    c2 = c.copy()
    c2[k] = _sound_speed(rho[k], 4.0 * p[k], 1.0 + 1.0 / G[k], P[k] / (G[k] + 1.0))
    rate2 = sum((np.abs(vel[d]) + c2) / case.dx[d] for d in range(ndim))
    assert oracle.cfl_dt(g, oracle.prim_to_cons(ndim, Q2)) == pytest.approx(0.5 / rate2.max(), rel=1e-10)


# --------------------------------------------------------------------------
# Sec. 2, Eq. (material-equation) and Sec. 3.1: Gamma and Pi are advected,
# d/dt Gamma + u . grad Gamma = 0, so a uniform Gamma and Pi stay uniform
# under any velocity field: the face fluxes Gamma u* and the source
# Gamma (u*_{i+1/2} - u*_{i-1/2}) / dx cancel in every direction.

@pytest.mark.parametrize("ndim", [1, 2, 3])
@pytest.mark.parametrize("gas", ["air", "water"])
def test_uniform_material_stays_uniform(ndim, gas):
    n = (48, 20, 10)[:ndim]
    case = wl.random_state(ndim, n, seed=21 + ndim, kind="shock")
    G, P = wl.material(*(wl.AIR if gas == "air" else wl.WATER))
    sl = wl.interior(ndim, case.n)
    case.Q[(2 + ndim,) + sl[1:]] = G
    case.Q[(3 + ndim,) + sl[1:]] = P
    if gas == "water":  # a liquid state of the same shape: rho ~ 1000, p >= 1e5
        case.Q[(0,) + sl[1:]] *= 1000.0
        case.Q[(1 + ndim,) + sl[1:]] = 1.0e5 + case.Q[(1 + ndim,) + sl[1:]] * 1.0e3
    g = oracle.Grid(ndim, case.n, case.dx, case.bc)
    L, _ = oracle.rhs(g, oracle.prim_to_cons(ndim, case.Q))
    vel = case.Q[1:1 + ndim][(slice(None),) + sl[1:]]
    dumax = max(float(np.abs(np.diff(vel[d], axis=2 - d)).max()) for d in range(ndim))
    assert dumax > 0.1  # the velocity field has real jumps (u in [-0.5, 0.5])
    # a dropped or sign-flipped source would leave about value x dumax / dx
    for f, value in ((2 + ndim, G), (3 + ndim, P)):
        scale = max(abs(value), 1.0) * dumax / min(case.dx[:ndim])
        assert np.abs(L[(f,) + sl[1:]]).max() <= 1e-12 * scale
