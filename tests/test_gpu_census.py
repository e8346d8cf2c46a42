"""Census step (ws_census_step): one RK3 step, bit-identical to ws_step, that
also counts how the reconstruction of Sec. 3.3 was evaluated: the
characteristic variables whose six stencil values are flat to 1e-6 of their
magnitude take the linear weights, the others WENO-IS.

The stationary-contact state (u = 0, uniform p, one gas, noisy density) fixes
the counts exactly: w1 = w6 = p/2, the tangential velocities, Gamma and Pi are
uniform, so of the nq characteristic variables only w2 = rho - p/c^2 has a
non-flat stencil at every face.  With a step that is zero in FP32 (1e-50)
the three stages see the same FP32 image, so each stage counts the same.  A
step that is merely small does not do: the HLLC momentum flux at a stationary
contact equals p only to FP32 rounding (the star flux is divided by S - S*),
so later stages see a velocity of order dt x rounding, and a stencil of such
values around zero is not flat.

The fused stage works on 32 x 15 tiles (x by the tile's second axis: y, or z
in the second 3D pass) and evaluates every face of a tile, so a face on the
edge between two tiles is evaluated by both; the census counts evaluations."""
import math

import numpy as np
import pytest

from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402


TX, TY = 32, 15


def n_faces(ndim, n):
    return sum(math.prod(n[e] + (1 if e == d else 0) for e in range(ndim)) for d in range(ndim))


def evaluated_faces(ndim, n):
    """Faces evaluated by the tiles of one RK stage (both 3D passes)."""
    def tiles(a, b):  # (width, height) of every tile over an a x b plane
        return [(min(TX, a - x0), min(TY, b - y0)) for x0 in range(0, a, TX) for y0 in range(0, b, TY)]
    if ndim == 2:
        return sum((w + 1) * h + w * (h + 1) for w, h in tiles(n[0], n[1]))
    xy = sum((w + 1) * h + w * (h + 1) for w, h in tiles(n[0], n[1])) * n[2]
    z = sum(w * (h + 1) for w, h in tiles(n[0], n[2])) * n[1]
    return xy + z


def test_evaluated_faces_cover_the_grid():
    # one tile: every face once
    assert evaluated_faces(2, (32, 15)) == n_faces(2, (32, 15))
    # two tiles side by side share one column of 15 x faces
    assert evaluated_faces(2, (64, 15)) == n_faces(2, (64, 15)) + 15


def contact_case(ndim, n, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(n[d] for d in reversed(range(ndim)))
    rho = 1.0 + 0.1 * rng.random(shape)
    G, P = wl.material(*wl.AIR)
    zero = np.zeros(shape)
    fields = [rho] + [zero] * ndim + [np.full(shape, 1.0e5), np.full(shape, G), np.full(shape, P)]
    h = tuple(1.0 / n[d] for d in range(ndim))
    bc = tuple(("periodic", "periodic") for _ in range(ndim))
    return wl.Case("contact", ndim, tuple(n), h, bc, wl._fill(ndim, n, fields))


@pytest.mark.parametrize("ndim,n", [(2, (70, 40)), (2, (64, 30)), (3, (40, 20, 17))])
def test_census_counts_on_a_stationary_contact(ndim, n):
    case = contact_case(ndim, n)
    s = ws.Solver(ndim, case.n, case.dx, case.bc, precision="mixed")
    U = s.prim_to_cons(s.tensor(case.Q))
    U0 = U.clone()
    c = s.census_step(U, 1e-50)
    nq = ndim + 4
    assert c["face_variables"] == 3 * nq * evaluated_faces(ndim, n)
    # only w2 is non-flat, at every face
    assert c["flat"] * nq == c["face_variables"] * (nq - 1)
    assert c["warp_passes"] % nq == 0
    assert c["warp_passes_weno"] * nq == c["warp_passes"]
    # a warp pass covers at most 32 faces
    assert 32 * c["warp_passes"] >= c["face_variables"]
    assert c["dt"] == 1e-50
    assert torch.equal(U, U0)  # the step is zero in FP32
    s.close()


def test_census_all_flat_on_a_uniform_state():
    n = (50, 33)
    case = contact_case(2, n)
    case.Q[0][wl.interior(2, n)[1:]] = 1.0
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
    U = s.prim_to_cons(s.tensor(case.Q))
    c = s.census_step(U)
    assert c["face_variables"] == 3 * 6 * evaluated_faces(2, n)
    assert c["flat"] == c["face_variables"]
    assert c["warp_passes_weno"] == 0
    s.close()


@pytest.mark.parametrize("kind", ["shock_bubble_2d", "drop_3d", "ragged_2d"])
def test_census_step_is_the_step(kind):
    """Census steps and plain steps from the same state give the same state,
    time step and MOOD record, bit for bit, over several steps."""
    if kind == "shock_bubble_2d":
        case = wl.shock_bubble_2d(160)
    elif kind == "drop_3d":
        case = wl.drop_3d(36, seed=1)
    else:
        case = wl.random_state(2, (77, 46), seed=9, kind="two_phase")
    s1 = ws.Solver(case.ndim, case.n, case.dx, case.bc, precision="mixed")
    s2 = ws.Solver(case.ndim, case.n, case.dx, case.bc, precision="mixed")
    U1 = s1.prim_to_cons(s1.tensor(case.Q))
    U2 = U1.clone()
    nq = case.ndim + 4
    for _ in range(4):
        dt1 = s1.step(U1, want_dt=True)
        c = s2.census_step(U2)
        assert c["dt"] == dt1
        assert torch.equal(U1, U2)
        m1, _ = s1.mood()
        m2, _ = s2.mood()
        assert np.array_equal(m1, m2)
        assert c["face_variables"] == 3 * nq * evaluated_faces(case.ndim, case.n)
        assert 0 <= c["flat"] <= c["face_variables"]
        assert 0 <= c["warp_passes_weno"] <= c["warp_passes"]
        assert 32 * c["warp_passes"] >= c["face_variables"]
    s1.close()
    s2.close()


def test_census_refused_off_the_fused_path():
    case = wl.random_state(2, (20, 18), seed=2, kind="smooth")
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="fp64")
    U = s.prim_to_cons(s.tensor(case.Q))
    with pytest.raises(RuntimeError, match="census"):
        s.census_step(U)
    s.close()
