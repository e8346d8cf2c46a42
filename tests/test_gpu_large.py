"""A grid whose state has more than 2^31 elements (65536 x 6000 cells in 2D,
6 fields: the Gamma and Pi fields of the last rows sit beyond element 2^31).

The grid is uniform air at rest except a 24 x 20 block of a random two-phase
state near its far corner.  One step changes only cells within 9 of the block
(three stages, three cells each), so a 56 x 52 grid holding the block with a
16-cell margin of the same air gives the oracle's answer for that corner: the
FP64 kernels must match it bit for bit, Δt included, and the mixed kernels to
1e-6 relative L1 per field.  Far from the block the big grid evolves as
uniform air: for the FP64 kernels bit for bit as the oracle's air (the
Shu-Osher combinations 3/4 U + 1/4 U1 and 1/3 U + 2/3 U2 round even where
L(U) = 0), for the mixed kernels' increment form not at all."""
import numpy as np
import pytest

import oracle
from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402

NX, NY = 65536, 6000
BX, BY = 24, 20        # block
MARGIN = 16            # air around the block in the small grid
DX = (1.0e-3, 1.0e-3)
BC = (("transmissive", "transmissive"), ("transmissive", "transmissive"))
NG = wl.NG


def background():
    G, P = wl.material(*wl.AIR)
    return [1.2, 0.0, 0.0, 1.0e5, G, P]


def block():
    return wl.random_state(2, (BX, BY), seed=5, kind="two_phase").Q[wl.interior(2, (BX, BY))][:, 0]


def small_case():
    n = (BX + 2 * MARGIN, BY + 2 * MARGIN)
    shape = (n[1], n[0])
    Q = wl._fill(2, n, [np.full(shape, v) for v in background()])
    Q[:, 0, NG + MARGIN:NG + MARGIN + BY, NG + MARGIN:NG + MARGIN + BX] = block()
    return n, Q


def big_state(s):
    """The big grid's conserved state, built on the device."""
    Q = s.tensor()
    for f, v in enumerate(background()):
        Q[f].fill_(v)
    x0, y0 = NX - BX - MARGIN, NY - BY - MARGIN
    Q[:, 0, NG + y0:NG + y0 + BY, NG + x0:NG + x0 + BX] = torch.tensor(block(), device="cuda")
    U = s.prim_to_cons(Q)
    del Q
    return U


def corner(U):
    """The big grid's cells that correspond to the small grid's interior."""
    x0, y0 = NX - BX - 2 * MARGIN, NY - BY - 2 * MARGIN
    return U[:, 0, NG + y0:NG + NY, NG + x0:NG + NX].cpu().numpy()


def far(U):
    return U[:, 0, NG:NG + 8, NG:NG + 8].cpu().numpy()


def free_bytes():
    torch.cuda.empty_cache()
    return torch.cuda.mem_get_info()[0]


@pytest.fixture(scope="module")
def reference():
    if free_bytes() < 150 * 2**30:
        pytest.skip("needs 150 GB of free device memory")
    n, Q = small_case()
    g = oracle.Grid(2, n, DX, BC)
    U0 = oracle.prim_to_cons(2, Q)
    U1, dt, _ = oracle.step(g, U0)
    return U1[wl.interior(2, n)][:, 0], dt


def test_state_beyond_2_31_elements_fp64(reference):
    ref, dto = reference
    s = ws.Solver(2, (NX, NY), DX, BC, precision="fp64")
    U = None
    try:
        assert s.size > 2**31
        U = big_state(s)
        dt = s.step(U, want_dt=True)
        assert dt == dto
        assert np.array_equal(corner(U), ref)
        # the small grid's first 8 x 8 cells are uniform air out of the block's reach
        assert np.array_equal(far(U), ref[:, :8, :8])
    finally:
        s.close()
        del U
        torch.cuda.empty_cache()


def test_state_beyond_2_31_elements_mixed(reference):
    ref, dto = reference
    s = ws.Solver(2, (NX, NY), DX, BC, precision="mixed")
    U = None
    try:
        U = big_state(s)
        f0 = far(U)
        s.step(U, dto)
        a = corner(U)
        mom = np.abs(ref[1]).sum() + np.abs(ref[2]).sum()
        for f in range(6):
            scale = mom if f in (1, 2) else np.abs(ref[f]).sum()
            assert np.abs(a[f] - ref[f]).sum() <= 1e-6 * scale, f
        assert np.array_equal(far(U), f0)
    finally:
        s.close()
        del U
        torch.cuda.empty_cache()


# 3D: 1024 x 1024 x 400 cells, 7 fields (3.0e9 elements; the E, Gamma and Pi
# fields of the last planes sit beyond element 2^31), the fused two-pass
# mixed stage, a 12 x 10 x 8 two-phase block at the far corner.
N3 = (1024, 1024, 400)
B3 = (12, 10, 8)
DX3 = (1.0e-3, 1.0e-3, 1.0e-3)
BC3 = (("transmissive", "transmissive"),) * 3


def block3():
    return wl.random_state(3, B3, seed=6, kind="two_phase").Q[wl.interior(3, B3)]


def background3():
    G, P = wl.material(*wl.AIR)
    return [1.2, 0.0, 0.0, 0.0, 1.0e5, G, P]


@pytest.fixture(scope="module")
def reference3():
    if free_bytes() < 200 * 2**30:
        pytest.skip("needs 200 GB of free device memory")
    n = tuple(B3[d] + 2 * MARGIN for d in range(3))
    shape = (n[2], n[1], n[0])
    Q = wl._fill(3, n, [np.full(shape, v) for v in background3()])
    Q[:, NG + MARGIN:NG + MARGIN + B3[2], NG + MARGIN:NG + MARGIN + B3[1],
      NG + MARGIN:NG + MARGIN + B3[0]] = block3()
    g = oracle.Grid(3, n, DX3, BC3)
    U1, dt, _ = oracle.step(g, oracle.prim_to_cons(3, Q))
    return U1[wl.interior(3, n)], dt


def test_state_beyond_2_31_elements_mixed_3d(reference3):
    ref, dto = reference3
    s = ws.Solver(3, N3, DX3, BC3, precision="mixed")
    try:
        _check_3d(s, ref, dto)
    finally:
        s.close()
        torch.cuda.empty_cache()


def _check_3d(s, ref, dto):
    assert s.size > 2**31
    Q = s.tensor()
    for f, v in enumerate(background3()):
        Q[f].fill_(v)
    o = [N3[d] - B3[d] - MARGIN for d in range(3)]
    Q[:, NG + o[2]:NG + o[2] + B3[2], NG + o[1]:NG + o[1] + B3[1], NG + o[0]:NG + o[0] + B3[0]] = \
        torch.tensor(block3(), device="cuda")
    U = s.prim_to_cons(Q)
    del Q
    f0 = U[:, NG:NG + 4, NG:NG + 4, NG:NG + 4].cpu().numpy()
    s.step(U, dto)
    c = [N3[d] - B3[d] - 2 * MARGIN for d in range(3)]
    a = U[:, NG + c[2]:NG + N3[2], NG + c[1]:NG + N3[1], NG + c[0]:NG + N3[0]].cpu().numpy()
    mom = sum(np.abs(ref[1 + d]).sum() for d in range(3))
    for f in range(7):
        scale = mom if 1 <= f <= 3 else np.abs(ref[f]).sum()
        assert np.abs(a[f] - ref[f]).sum() <= 1e-6 * scale, f
    assert np.array_equal(U[:, NG:NG + 4, NG:NG + 4, NG:NG + 4].cpu().numpy(), f0)
