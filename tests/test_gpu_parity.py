"""Parity of the FP64 CUDA path (through the C ABI) with the FP64 oracle.

Bar: bit-exact.  Both sides evaluate the same formulas, one IEEE operation at
a time in the same order, without FMA contraction, so every conserved field,
every flux divergence, every CFL step and every MOOD mask byte must match
exactly (compared with ==, so +0 and -0 count as equal).  This is stricter
than the required 1e-10 relative L-infinity bound and the bit-identical MOOD
mask."""
import numpy as np
import pytest

import oracle
from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402


def solver_for(case, **kw):
    return ws.Solver(case.ndim, case.n, case.dx, case.bc, **kw)


def ogrid(case, mood=True, weights="modified"):
    return oracle.Grid(case.ndim, case.n, case.dx, case.bc, mood=mood, weights=weights)


def same(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return bool(np.all((a == b) | (np.isnan(a) & np.isnan(b))))


def flat_masks(ms):
    return np.concatenate([m.ravel() for m in ms]) if ms else np.zeros(0, np.uint8)


CASES = [
    (1, (61,), "smooth"), (1, (50,), "shock"), (1, (97,), "two_phase"),
    (2, (37, 29), "smooth"), (2, (33, 18), "shock"), (2, (40, 35), "two_phase"),
    (3, (13, 11, 9), "smooth"), (3, (12, 10, 14), "two_phase"),
]


@pytest.mark.parametrize("ndim,n,kind", CASES)
def test_prim_to_cons_bitwise(ndim, n, kind):
    case = wl.random_state(ndim, n, seed=3, kind=kind)
    s = solver_for(case)
    U = s.prim_to_cons(s.tensor(case.Q))
    Uo = oracle.prim_to_cons(ndim, case.Q)
    assert same(U.cpu().numpy(), Uo)
    Q = s.cons_to_prim(U)
    sl = wl.interior(ndim, case.n)
    assert same(Q.cpu().numpy()[sl], oracle.cons_to_prim(ndim, Uo)[sl])


@pytest.mark.parametrize("ndim,n,kind", CASES)
@pytest.mark.parametrize("weights", ["modified", "basic"])
def test_flux_divergence_bitwise(ndim, n, kind, weights):
    case = wl.random_state(ndim, n, seed=5, kind=kind)
    s = solver_for(case, weights=weights)
    Uo = oracle.prim_to_cons(ndim, case.Q)
    U = s.tensor(Uo)
    L = s.flux_divergence(U)
    Lo, mo = oracle.rhs(ogrid(case, weights=weights), Uo)
    sl = wl.interior(ndim, case.n)
    assert same(L.cpu().numpy()[sl], Lo[sl])
    _, mask = s.mood(with_mask=True)
    assert same(mask.cpu().numpy()[:s.nmask], flat_masks(mo))


@pytest.mark.parametrize("ndim,n,kind", CASES)
@pytest.mark.parametrize("mood", [True, False])
def test_step_bitwise(ndim, n, kind, mood):
    case = wl.random_state(ndim, n, seed=7, kind=kind)
    s = solver_for(case, mood=mood)
    g = ogrid(case, mood=mood)
    Uo = oracle.prim_to_cons(ndim, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(ndim, case.n)
    for _ in range(3):
        dt = s.step(U, want_dt=True)
        Uo, dto, mo = oracle.step(g, Uo, with_mask=True)
        assert dt == dto
        assert same(U.cpu().numpy()[sl], Uo[sl])
        _, mask = s.mood(with_mask=True)
        mask = mask.cpu().numpy().reshape(3, -1)
        for st in range(3):
            assert same(mask[st], flat_masks(mo[st]))


def test_gas_water_tube_trajectory_bitwise():
    """The 1D gas-water shock tube (200 cells, water 1e9 Pa | air 1e5 Pa), run to
    t = 2.4e-4 s with CFL 0.5: every step, field and MOOD mask match."""
    case = wl.gas_water_tube(200)
    s = solver_for(case, check=True)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(1, case.Q)
    U = s.tensor(Uo)
    t = 0.0
    k = 0
    while t < case.t_end:
        dt = oracle.cfl_dt(g, Uo)
        dt = min(dt, case.t_end - t)
        s.step(U, dt)
        Uo, _, mo = oracle.step(g, Uo, dt=dt, with_mask=True)
        _, mask = s.mood(with_mask=True)
        sl = wl.interior(1, case.n)
        assert same(U.cpu().numpy()[sl], Uo[sl]), k
        mask = mask.cpu().numpy().reshape(3, -1)
        for st in range(3):
            assert same(mask[st], flat_masks(mo[st]))
        t += dt
        k += 1
    assert k > 200


def test_shock_bubble_2d_small_bitwise():
    """Down-sized 2D shock-bubble (96^2): 10 CFL steps, fields and MOOD masks."""
    case = wl.shock_bubble_2d(96)
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(2, case.n)
    for _ in range(10):
        dt = s.step(U, want_dt=True)
        Uo, dto, mo = oracle.step(g, Uo, with_mask=True)
        assert dt == dto
        assert same(U.cpu().numpy()[sl], Uo[sl])
        _, mask = s.mood(with_mask=True)
        mask = mask.cpu().numpy().reshape(3, -1)
        assert same(mask[2], flat_masks(mo[2]))


def test_shock_bubble_2d_long_trajectory_bitwise():
    """The 128^2 shock-bubble over 300 CFL steps, in which the shock crosses
    the bubble: the FP64 path stays bit for bit on the oracle's trajectory --
    every step's dt, and every 50 steps the state and that step's MOOD
    record."""
    case = wl.shock_bubble_2d(128)
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(2, case.n)
    for k in range(1, 301):
        dt = s.step(U, want_dt=True)
        Uo, dto, mo = oracle.step(g, Uo, with_mask=(k % 50 == 0))
        assert dt == dto, k
        if k % 50 == 0:
            assert same(U.cpu().numpy()[sl], Uo[sl]), k
            _, mask = s.mood(with_mask=True)
            mask = mask.cpu().numpy().reshape(3, -1)
            for st in range(3):
                assert same(mask[st], flat_masks(mo[st])), k


def test_drop_3d_small_bitwise():
    """Down-sized 3D periodic drop with density noise (20^3): 3 steps."""
    case = wl.drop_3d(20, seed=0)
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(3, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(3, case.n)
    for _ in range(3):
        s.step(U)
        Uo, _, _ = oracle.step(g, Uo)
    assert same(U.cpu().numpy()[sl], Uo[sl])


def test_full_size_drop_3d_one_step():
    """The 3D benchmark grid (256^3 periodic water drop with density noise):
    one CFL step of the FP64 kernels matches the oracle bit for bit (state,
    dt and every MOOD mask byte of the three stages)."""
    case = wl.drop_3d(256, seed=0)
    g = ogrid(case)
    Un = oracle.prim_to_cons(3, case.Q)
    del case.Q
    s = solver_for(case)
    U = s.tensor(Un)
    dt = s.step(U, want_dt=True)
    Uo, dto, mo = oracle.step(g, Un, with_mask=True)
    assert dt == dto
    sl = wl.interior(3, case.n)
    assert same(U.cpu().numpy()[sl], Uo[sl])
    _, mask = s.mood(with_mask=True)
    mask = mask.cpu().numpy().reshape(3, -1)
    for st in range(3):
        assert same(mask[st], flat_masks(mo[st])), st
    s.close()


def test_reflective_and_mixed_bcs_bitwise():
    case = wl.random_state(2, (21, 17), seed=9, kind="shock")
    case.bc = (("reflective", "transmissive"), ("periodic", "periodic"))
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    for _ in range(3):
        s.step(U)
        Uo, _, _ = oracle.step(g, Uo)
    sl = wl.interior(2, case.n)
    assert same(U.cpu().numpy()[sl], Uo[sl])


@pytest.mark.parametrize("n", [(1, 9), (9, 1), (6, 7), (2, 2)])
def test_degenerate_extents_bitwise(n):
    """Single-cell and tiny extents (transmissive): the face sweep of a
    direction with one cell sees a constant stencil."""
    case = wl.random_state(2, n, seed=2, kind="shock")
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    s.step(U)
    Uo, _, _ = oracle.step(g, Uo)
    sl = wl.interior(2, case.n)
    assert same(U.cpu().numpy()[sl], Uo[sl])


def test_tubes_bitwise():
    """Batched tubes of uneven length (6..300 cells) in one launch per kernel:
    per-tube CFL steps and states match the oracle tube by tube."""
    off, Q = wl.riemann_tubes(ntubes=64, lmin=6, lmax=300, seed=1)
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off)
    Qt = s.tensor(Q)
    U = s.prim_to_cons(Qt)
    Uo = oracle.prim_to_cons(1, Q.reshape(5, 1, 1, -1)).reshape(5, -1)
    assert same(U.cpu().numpy(), Uo)
    for _ in range(3):
        dts = s.step(U, want_dt=True)
        Uo, dto = oracle.tubes_step(off, Uo)
        assert same(dts, dto)
        Ug = U.cpu().numpy()
        for t in range(64):
            a, b = off[t] + 3, off[t + 1] - 3
            assert same(Ug[:, a:b], Uo[:, a:b]), t


def test_full_size_shock_bubble_one_step():
    """The 1024^2 shock-bubble workload in the benchmark's launch configuration:
    one CFL step matches the oracle bit for bit on every interior cell."""
    case = wl.shock_bubble_2d(1024)
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    dt = s.step(U, want_dt=True)
    Uo, dto, _ = oracle.step(g, Uo)
    assert dt == dto
    sl = wl.interior(2, case.n)
    assert same(U.cpu().numpy()[sl], Uo[sl])


def test_full_size_shock_bubble_mid_run():
    """The 1024^2 shock-bubble at a mid-run state (400 mixed-precision steps
    in: the shock inside the bubble), in the benchmark's launch configuration.
    One FP64 step matches the oracle bit for bit (state, dt and every MOOD mask
    byte of the three stages); the mixed kernels from the same state, with the
    same dt, agree with the oracle to 1e-6 relative L1 per field (a momentum
    component against the whole momentum) and on 99.9 % of the mask bytes."""
    case = wl.shock_bubble_2d(1024)
    s32 = solver_for(case, precision="mixed")
    U32 = s32.prim_to_cons(s32.tensor(case.Q))
    for _ in range(400):
        s32.step(U32)
    Un = U32.cpu().numpy()
    g = ogrid(case)
    Uo, dto, mo = oracle.step(g, Un, with_mask=True)
    sl = wl.interior(2, case.n)
    # FP64 kernels
    s64 = solver_for(case)
    U = s64.tensor(Un)
    dt = s64.step(U, want_dt=True)
    assert dt == dto
    assert same(U.cpu().numpy()[sl], Uo[sl])
    _, mask = s64.mood(with_mask=True)
    mask = mask.cpu().numpy().reshape(3, -1)
    for st in range(3):
        assert same(mask[st], flat_masks(mo[st])), st
    # mixed kernels
    Um = s32.tensor(Un)
    s32.step(Um, dto)
    a, b = Um.cpu().numpy()[sl], Uo[sl]
    mom = np.abs(b[1]).sum() + np.abs(b[2]).sum()
    for f in range(6):
        ref = mom if f in (1, 2) else np.abs(b[f]).sum()
        assert np.abs(a[f] - b[f]).sum() <= 1e-6 * ref, f
    _, mm = s32.mood(with_mask=True)
    mm = mm.cpu().numpy().reshape(3, -1)
    agree = np.mean([np.mean(mm[st] == flat_masks(mo[st])) for st in range(3)])
    assert agree >= 0.999
    s32.close()
    s64.close()


def test_run_host_matches_device_steps():
    case = wl.random_state(2, (30, 20), seed=4, kind="two_phase")
    s = solver_for(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    for _ in range(4):
        s.step(U)
    Uh = torch.tensor(Uo).pin_memory()
    ws.ws_run_host(s.ctx, Uh, 4)
    assert same(Uh.numpy(), U.cpu().numpy())


def test_nonphysical_state_reported():
    """A host-prepared state with a negative density is reported as
    WS_ENONPHYS by the step (no device trap); the context stays usable."""
    case = wl.random_state(1, (40,), seed=1, kind="shock")
    s = solver_for(case, check=True)
    Q = case.Q.copy()
    Q[0, 0, 0, 20] = -1.0
    U = s.prim_to_cons(s.tensor(Q))
    with pytest.raises(ws.WsError) as ei:
        s.step(U, 1e-4)
    assert ei.value.code == ws.WS_ENONPHYS
    assert s.nonphysical() > 0
    U2 = s.prim_to_cons(s.tensor(case.Q))
    s.step(U2, 1e-4)
    assert s.nonphysical() == 0


@pytest.mark.parametrize("bad", ["ndim", "dx", "periodic_one_side", "precision"])
def test_invalid_arguments(bad):
    kw = dict(ndim=2, n=(8, 8), dx=(0.1, 0.1), bc=(("transmissive",) * 2,) * 2)
    opts = {}
    if bad == "ndim":
        kw["ndim"] = 4
    elif bad == "dx":
        kw["dx"] = (0.1, -1.0)
    elif bad == "periodic_one_side":
        kw["bc"] = (("periodic", "transmissive"), ("transmissive", "transmissive"))
    else:
        opts = {"precision": "fp64", "learned": True}
    if kw["ndim"] > 3:
        g = ws.ws_grid()
        g.ndim = kw["ndim"]
    else:
        g, _ = ws.make_grid(kw["ndim"], kw["n"], kw["dx"], kw["bc"])
    with pytest.raises(ws.WsError) as ei:
        ws.ws_init(g, ws.make_opts(**opts), 0)
    assert ei.value.code == ws.WS_EINVAL


@pytest.mark.parametrize("make", [lambda: wl.haas_sturtevant("R22", 90, 30), lambda: wl.haas_sturtevant("He", 90, 30),
                                  lambda: wl.shock_droplet(48)], ids=["air_R22", "air_He", "shock_droplet"])
def test_shock_interface_setups_small_bitwise(make):
    """The shock-gas-cylinder (Sec. 6.1; reflective walls, ideal-gas limit)
    and shock-droplet (Sec. 6.2) setups, down-sized, with MOOD off as in the
    paper: 8 CFL steps bit-identical to the oracle, Δt included."""
    case = make()
    s = solver_for(case, mood=False)
    g = ogrid(case, mood=False)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    sl = wl.interior(2, case.n)
    for _ in range(8):
        dt = s.step(U, want_dt=True)
        Uo, dto, _ = oracle.step(g, Uo)
        assert dt == dto
    assert same(U.cpu().numpy()[sl], Uo[sl])


@pytest.mark.parametrize("make", [lambda: wl.haas_sturtevant("R22"), lambda: wl.haas_sturtevant("He"),
                                  lambda: wl.shock_droplet()], ids=["air_R22", "air_He", "shock_droplet"])
def test_shock_interface_setups_full_size(make):
    """The same setups at the benchmark's sizes (3000 x 1000 cylinders,
    800^2 droplet), MOOD off: one CFL step of the FP64 kernels bit-identical
    to the oracle, and the mixed kernels from the same state within 1e-6
    relative L1 per field (a momentum component against the whole momentum)."""
    case = make()
    g = ogrid(case, mood=False)
    Un = oracle.prim_to_cons(2, case.Q)
    Uo, dto, _ = oracle.step(g, Un)
    sl = wl.interior(2, case.n)
    s = solver_for(case, mood=False)
    U = s.tensor(Un)
    dt = s.step(U, want_dt=True)
    assert dt == dto
    assert same(U.cpu().numpy()[sl], Uo[sl])
    s.close()
    sm = solver_for(case, mood=False, precision="mixed")
    Um = sm.tensor(Un)
    sm.step(Um, dto)
    a, b = Um.cpu().numpy()[sl], Uo[sl]
    mom = np.abs(b[1]).sum() + np.abs(b[2]).sum()
    for f in range(6):
        ref = mom if f in (1, 2) else np.abs(b[f]).sum()
        err = np.abs(a[f] - b[f]).sum()
        assert (err <= 1e-6 * ref) if ref > 0 else err == 0.0, f
    sm.close()
