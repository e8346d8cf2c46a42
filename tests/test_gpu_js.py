"""The comparison scheme WENO-JS (Jiang & Shu 1996; the paper compares with it
in Secs. 5 and 6) as the weights option WS_W_JS of both CUDA paths.

FP64 path: bit-exact against the oracle's WENO-JS (fields, dt, MOOD mask
bytes), as for the scheme itself.  Mixed path: within the FP32 tolerance of
the other mixed-precision tests."""
import numpy as np
import pytest

import oracle
from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402


def same(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return bool(np.all((a == b) | (np.isnan(a) & np.isnan(b))))


def flat_masks(ms):
    return np.concatenate([m.ravel() for m in ms]) if ms else np.zeros(0, np.uint8)


CASES = [
    (1, (61,), "smooth"), (1, (97,), "two_phase"), (2, (37, 29), "smooth"), (2, (33, 18), "shock"),
    (2, (40, 35), "two_phase"), (3, (13, 11, 9), "smooth"), (3, (12, 10, 14), "two_phase"),
]


@pytest.mark.parametrize("ndim,n,kind", CASES)
def test_js_flux_divergence_bitwise(ndim, n, kind):
    case = wl.random_state(ndim, n, seed=5, kind=kind)
    s = ws.Solver(ndim, case.n, case.dx, case.bc, weights="js")
    Uo = oracle.prim_to_cons(ndim, case.Q)
    L = s.flux_divergence(s.tensor(Uo))
    Lo, mo = oracle.rhs(oracle.Grid(ndim, case.n, case.dx, case.bc, weights="js"), Uo)
    sl = wl.interior(ndim, case.n)
    assert same(L.cpu().numpy()[sl], Lo[sl])
    _, mask = s.mood(with_mask=True)
    assert same(mask.cpu().numpy()[:s.nmask], flat_masks(mo))
    s.close()


@pytest.mark.parametrize("ndim,n,kind", [(1, (97,), "two_phase"), (2, (40, 35), "two_phase"),
                                         (3, (12, 10, 14), "two_phase")])
@pytest.mark.parametrize("mood", [True, False])
def test_js_step_bitwise(ndim, n, kind, mood):
    """Three steps with the oracle's time steps (the CFL reduction does not
    depend on the weights and is covered by the scheme's own step tests).  On
    the 3D state WENO-JS leaves an inadmissible cell after two steps, in the
    oracle and on the GPU alike, where WENO-IS does not; the oracle's CFL
    maximum skips the NaN sound speed of such a cell while the GPU's
    propagates it, so a CFL step would differ there."""
    case = wl.random_state(ndim, n, seed=7, kind=kind)
    s = ws.Solver(ndim, case.n, case.dx, case.bc, weights="js", mood=mood)
    g = oracle.Grid(ndim, case.n, case.dx, case.bc, weights="js", mood=mood)
    Uo = oracle.prim_to_cons(ndim, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(ndim, case.n)
    for _ in range(3):
        Uo, dto, mo = oracle.step(g, Uo, with_mask=True)
        s.step(U, dto)
        assert same(U.cpu().numpy()[sl], Uo[sl])
        _, mask = s.mood(with_mask=True)
        mask = mask.cpu().numpy().reshape(3, -1)
        for st in range(3):
            assert same(mask[st], flat_masks(mo[st]))
    s.close()


def test_js_tubes_bitwise():
    off, Q = wl.riemann_tubes(ntubes=12, lmin=16, lmax=80, seed=4)
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, weights="js")
    U = s.prim_to_cons(s.tensor(Q))
    Uo = U.cpu().numpy().copy()
    dts = s.step(U, want_dt=True)
    Uo, dto = oracle.tubes_step(off, Uo, eps=1e-6, mood=True, weights="js")
    assert same(dts, dto)
    assert same(U.cpu().numpy(), Uo)
    s.close()


@pytest.mark.parametrize("ndim,n,kind", CASES)
def test_js_mixed_flux_divergence_close(ndim, n, kind):
    """The mixed path's WENO-JS (FP32, weights scaled by the smallest
    (eps + beta)^2) against the oracle, to the tolerance of the scheme's own
    mixed-precision test: 2e-5 of each field's flux scale."""
    case = wl.random_state(ndim, n, seed=5, kind=kind)
    s = ws.Solver(ndim, case.n, case.dx, case.bc, precision="mixed", weights="js")
    Uo = oracle.prim_to_cons(ndim, case.Q)
    L = s.flux_divergence(s.tensor(Uo)).cpu().numpy()
    Lo, _ = oracle.rhs(oracle.Grid(ndim, case.n, case.dx, case.bc, weights="js"), Uo)
    sl = wl.interior(ndim, case.n)
    Qo = oracle.cons_to_prim(ndim, Uo)[sl]
    c = np.sqrt(((Qo[-2] + 1) * Qo[-3] + Qo[-1]) / (Qo[-2] * Qo[0]))
    speed = c + sum(np.abs(Qo[1 + d]) for d in range(ndim))
    dxmin = min(case.dx[:ndim])
    for f in range(case.nv):
        scale = np.abs(Uo[sl][f] * speed).max() / dxmin
        err = np.abs(L[sl][f] - Lo[sl][f]).max()
        assert err <= 2e-5 * scale, (f, err, scale)
    s.close()


def test_js_fused_step_close_to_oracle():
    """The fused 2D stage with WENO-JS: five steps of the 96^2 shock-bubble
    against the oracle's WENO-JS with the same time steps, L1 density."""
    case = wl.shock_bubble_2d(96)
    g = oracle.Grid(2, case.n, case.dx, case.bc, weights="js")
    Uo = oracle.prim_to_cons(2, case.Q)
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", weights="js")
    U = s.tensor(Uo)
    for _ in range(5):
        Uo, dt, _ = oracle.step(g, Uo)
        s.step(U, dt)
    sl = wl.interior(2, case.n)
    a, b = U.cpu().numpy()[sl][0], Uo[sl][0]
    assert np.abs(a - b).sum() / np.abs(b).sum() < 1e-5
    s.close()


def _mood_total(weights, n=256, steps=500):
    case = wl.shock_bubble_2d(n)
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", weights=weights)
    U = s.prim_to_cons(s.tensor(case.Q))
    tot = np.zeros((3, 3), np.int64)
    for _ in range(steps):
        s.step(U)
        tot += s.mood()[0]
    bad = s.nonphysical()
    s.close()
    return tot, bad


def test_mood_counts_js_above_is_on_shock_bubble():
    """Sec. 6.4 (MOOD counters of the shock-bubble case): WENO-JS needs the
    MOOD fallback on more face sides than WENO-IS.  The 2D shock-bubble at
    256^2 over 500 CFL steps (the physical time of the 2000-step 1024^2 run),
    face sides at 3rd and 1st order summed over both directions."""
    is_, bad_is = _mood_total("modified")
    js, bad_js = _mood_total("js")
    assert bad_is == 0 and bad_js == 0
    low_is = int(is_[:2, 1:].sum())
    low_js = int(js[:2, 1:].sum())
    assert low_is > 0
    assert low_js > low_is, (is_, js)


def test_shock_bubble_1d_needs_mood():
    """Sec. 5.3 shock/bubble in liquid (200 cells): with the MOOD cascade the
    scheme stays admissible through the shock's arrival at the bubble wall
    (x = 0.4, about step 66) and well beyond; without it the characteristic
    reconstruction at the liquid/gas face gives a negative gas pressure there
    and a cell turns inadmissible at step 71 -- the same in the oracle, which
    this path matches bit for bit.  (The paper runs this case without MOOD.)"""
    case = wl.shock_bubble_1d(200)
    res = {}
    for mood in (True, False):
        s = ws.Solver(1, case.n, case.dx, case.bc, mood=mood)
        U = s.prim_to_cons(s.tensor(case.Q))
        first_bad = None
        for k in range(1, 2001):
            s.step(U)
            if k >= 60 and k <= 80 or k % 250 == 0:
                if s.nonphysical():
                    first_bad = k
                    break
        res[mood] = first_bad
        s.close()
    assert res[True] is None
    assert res[False] == 71
