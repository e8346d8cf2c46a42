"""Mixed-precision path (FP32 projection / WENO-IS / HLLC, FP64 pressure
recovery, MOOD sign test and RK accumulation) against the FP64 oracle.

Tolerances follow from FP32 arithmetic (unit roundoff 6e-8): a single
evaluation of L(U) agrees with the oracle to ~1e-5 of the field's flux scale
(the divergence subtracts fluxes of neighbouring faces), and short
trajectories agree in L1 to well inside the 1e-4 relative density bound the
mixed form is held to."""
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
    return ws.Solver(case.ndim, case.n, case.dx, case.bc, precision="mixed", **kw)


def ogrid(case, mood=True):
    return oracle.Grid(case.ndim, case.n, case.dx, case.bc, mood=mood)


CASES = [(1, (61,), "smooth"), (1, (97,), "two_phase"), (2, (37, 29), "smooth"), (2, (33, 18), "shock"),
         (2, (40, 35), "two_phase"), (3, (13, 11, 9), "smooth"), (3, (12, 10, 14), "two_phase")]


@pytest.mark.parametrize("ndim,n,kind", CASES)
def test_flux_divergence_close(ndim, n, kind):
    case = wl.random_state(ndim, n, seed=5, kind=kind)
    s = solver_for(case)
    Uo = oracle.prim_to_cons(ndim, case.Q)
    L = s.flux_divergence(s.tensor(Uo)).cpu().numpy()
    Lo, mo = oracle.rhs(ogrid(case), Uo)
    sl = wl.interior(ndim, case.n)
    # flux scale of each field: |F| ~ |U| (|u| + c), divided by dx
    Qo = oracle.cons_to_prim(ndim, Uo)[sl]
    c = np.sqrt(((Qo[-2] + 1) * Qo[-3] + Qo[-1]) / (Qo[-2] * Qo[0]))
    speed = c + sum(np.abs(Qo[1 + d]) for d in range(ndim))
    dxmin = min(case.dx[:ndim])
    _, mask = s.mood(with_mask=True)
    agree = np.mean(mask.cpu().numpy()[:s.nmask] == np.concatenate([m.ravel() for m in mo]))
    assert agree > 0.99
    for f in range(case.nv):
        scale = np.abs(Uo[sl][f] * speed).max() / dxmin
        err = np.abs(L[sl][f] - Lo[sl][f]).max()
        assert err <= 2e-5 * scale, (f, err, scale)


def l1_rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def test_gas_water_tube_l1():
    """The gas-water shock tube to t = 2.4e-4 s: L1 density error vs the oracle."""
    case = wl.gas_water_tube(200)
    s = solver_for(case, check=True)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(1, case.Q)
    U = s.tensor(Uo)
    t = 0.0
    while t < case.t_end:
        dt = min(oracle.cfl_dt(g, Uo), case.t_end - t)
        s.step(U, dt)
        Uo, _, _ = oracle.step(g, Uo, dt=dt)
        t += dt
    sl = wl.interior(1, case.n)
    assert l1_rel(U.cpu().numpy()[sl][0], Uo[sl][0]) < 1e-5


def test_shock_bubble_small_l1():
    """96^2 shock-bubble, 40 steps with the oracle's time steps: L1 density error."""
    case = wl.shock_bubble_2d(96)
    s = solver_for(case, check=True)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    for _ in range(40):
        dt = oracle.cfl_dt(g, Uo)
        s.step(U, dt)
        Uo, _, _ = oracle.step(g, Uo, dt=dt)
    sl = wl.interior(2, case.n)
    assert l1_rel(U.cpu().numpy()[sl][0], Uo[sl][0]) < 1e-5


def test_interface_equilibrium_mixed():
    """Sec. 5.1 interface transport: p and u stay uniform to the accuracy FP32
    fluxes allow.  In the liquid E ~ 8.5e3 (Pi = 3.5e3, rho u^2/2 = 5e3) while
    Gamma p = 0.17, so a flux rounded to FP32 (6e-8 relative) moves p by about
    6e-8 x 8.5e3 / 0.17 = 3e-3 per rounding: the bound on p is 2e-2, on u 1e-4.
    (The FP64 path keeps both to ~1e-10.)"""
    case = wl.interface_transport(200)
    s = solver_for(case)
    U = s.prim_to_cons(s.tensor(case.Q))
    t = 0.0
    while t < case.t_end:
        dt = min(s.cfl_dt(U), case.t_end - t)
        s.step(U, dt)
        t += dt
    Q = s.cons_to_prim(U).cpu().numpy()[wl.interior(1, case.n)]
    assert np.abs(Q[2] - 1.0).max() < 2e-2
    assert np.abs(Q[1] / 100.0 - 1.0).max() < 1e-4


def test_mixed_cfl_close_to_fp64():
    case = wl.shock_bubble_2d(128)
    s = solver_for(case)
    Uo = oracle.prim_to_cons(2, case.Q)
    dt = s.cfl_dt(s.tensor(Uo))
    assert dt == pytest.approx(oracle.cfl_dt(ogrid(case), Uo), rel=1e-6)


@pytest.mark.parametrize("n,bc", [((37, 29), "transmissive"), ((70, 47), "periodic"), ((33, 16), "reflective"),
                                  ((5, 64), "transmissive"), ((64, 3), "periodic")])
def test_fused_stage_matches_generic(n, bc, monkeypatch):
    """The fused 2D stage kernel (tile + halo in shared memory, boundary
    conditions applied on load, increment-form RK3) and the generic kernels
    evaluate the same mixed-precision scheme: after 3 steps they agree to
    FP32 rounding, and their MOOD masks agree on almost every face."""
    case = wl.random_state(2, n, seed=21, kind="two_phase")
    case.bc = ((bc, bc), (bc, bc))
    Uo = oracle.prim_to_cons(2, case.Q)
    outs = []
    for fused in (True, False):
        if fused:
            monkeypatch.delenv("WS_NO_FUSED", raising=False)
        else:
            monkeypatch.setenv("WS_NO_FUSED", "1")
        s = solver_for(case)
        U = s.tensor(Uo)
        for _ in range(3):
            s.step(U, 1e-7)
        _, mask = s.mood(with_mask=True)
        outs.append((U.cpu().numpy(), mask.cpu().numpy()))
        s.close()
    sl = wl.interior(2, case.n)
    for f in range(6):
        a, b = outs[0][0][sl][f], outs[1][0][sl][f]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max() + 1e-300, f
    assert np.mean(outs[0][1] == outs[1][1]) > 0.99


def test_integer_pipe_conversions_match_hardware():
    """The mixed kernels convert FP64 <-> FP32 on the integer pipe; on normal
    FP32-range values (including exact rounding ties) the result must equal
    the hardware round-to-nearest-even cast bit for bit, and widening back
    must be exact; zero, inf and NaN keep their class."""
    rng = np.random.default_rng(0)
    mant = rng.uniform(1.0, 2.0, size=20000)
    expo = rng.integers(-125, 127, size=20000)
    x = mant * np.exp2(expo) * rng.choice([-1.0, 1.0], size=20000)
    f = rng.uniform(1, 2, size=2000).astype(np.float32).astype(np.float64) * np.exp2(rng.integers(-100, 100, 2000))
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    ties = f + 0.5 * ulp  # exactly half-way between two floats
    x = np.concatenate([x, ties, f, [0.0, -0.0, 1.0, -1.0, 3.4e38, 1.2e-38]])
    o32, o64 = ws.ws_convert_probe(torch.tensor(x, device="cuda"))
    ref = x.astype(np.float32)
    assert np.array_equal(o32.cpu().numpy().view(np.uint32), ref.view(np.uint32))
    assert np.array_equal(o64.cpu().numpy(), ref.astype(np.float64))
    sp = np.array([np.inf, -np.inf, np.nan, 1e300, 1e-300])
    s32, s64 = ws.ws_convert_probe(torch.tensor(sp, device="cuda"))
    s32 = s32.cpu().numpy()
    assert s32[0] == np.inf and s32[1] == -np.inf and np.isnan(s32[2]) and s32[3] == np.inf and s32[4] == 0.0
    assert np.isnan(s64.cpu().numpy()[2])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_graph_replay_identical(precision):
    """A CFL step replayed from the captured CUDA graph gives the same bits as
    the directly launched step, over several steps and a change of state buffer."""
    case = wl.random_state(2, (45, 38), seed=3, kind="two_phase")
    stream = torch.cuda.Stream()
    outs = []
    for graph in (False, True):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision=precision, stream=stream)
        ws.ws_set_graph(s.ctx, graph)
        Uo = oracle.prim_to_cons(2, case.Q)
        with torch.cuda.stream(stream):
            U = s.tensor(Uo)
            V = s.tensor(Uo)
            for _ in range(4):
                s.step(U)
            for _ in range(2):
                s.step(V)
            dt = s.step(U, want_dt=True)
        stream.synchronize()
        outs.append((U.cpu().numpy(), V.cpu().numpy(), dt))
        s.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def _tubes_case(ntubes=64, lmin=6, lmax=600, seed=1):
    off, Q = wl.riemann_tubes(ntubes=ntubes, lmin=lmin, lmax=lmax, seed=seed)
    return off, Q


def test_tubes_mixed_close_to_oracle():
    """Batched tubes in mixed precision (persistent kernel, chunks of 256..1024
    cells so that long tubes span several chunks): per-tube CFL steps and
    densities against the FP64 oracle, tube by tube."""
    off, Q = _tubes_case()
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision="mixed")
    U = s.prim_to_cons(s.tensor(Q))
    Uo = oracle.prim_to_cons(1, Q.reshape(5, 1, 1, -1)).reshape(5, -1)
    for _ in range(3):
        dts = s.step(U, want_dt=True)
        Uo, dto = oracle.tubes_step(off, Uo)
        np.testing.assert_allclose(dts, dto, rtol=2e-5)  # FP32 wave speeds
    Ug = U.cpu().numpy()
    for t in range(len(off) - 1):
        a, b = off[t] + 3, off[t + 1] - 3
        assert l1_rel(Ug[0, a:b], Uo[0, a:b]) < 2e-5, t
    counts, _ = s.mood()
    faces = sum(off[t + 1] - off[t] - 5 for t in range(len(off) - 1))
    assert counts[0].sum() == 2 * 3 * faces  # both sides of every face, 3 stages, direction x only
    assert s.nonphysical() == 0


def test_tubes_autotune_and_graph():
    """The autotuner picks one of the configurations; CUDA-graph replay of the
    persistent tube step gives the same bits as direct launches."""
    off, Q = _tubes_case(ntubes=200, lmin=256, lmax=2048, seed=3)
    stream = torch.cuda.Stream()
    outs = []
    for graph in (False, True):
        s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision="mixed", stream=stream)
        with torch.cuda.stream(stream):
            U = s.prim_to_cons(s.tensor(Q))
            choice = ws.ws_autotune(s.ctx, U, 2)
            assert 0 <= choice < 5
            ws.ws_set_graph(s.ctx, graph)
            for _ in range(3):
                s.step(U)
        stream.synchronize()
        outs.append(U.cpu().numpy())
        s.close()
    # both runs use their own autotuned chunking; results agree to FP32 rounding
    np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=1e-5)


def _sub_batch(off, U, tubes):
    """The padded segments of the chosen tubes, concatenated, with their offsets."""
    segs = [U[:, off[t]:off[t + 1]] for t in tubes]
    sub_off = np.zeros(len(tubes) + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum([sg.shape[1] for sg in segs])
    return sub_off, np.ascontiguousarray(np.concatenate(segs, axis=1))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tubes_full_size_sampled(precision):
    """The full batched configuration (4096 tubes of 256..8192 cells, 9.3M
    cells), launched as the benchmark launches it (autotuned, CUDA graph);
    32 sampled tubes are recomputed by the oracle one by one: bit-exact in
    FP64, within FP32 tolerances in mixed precision."""
    off, Q = wl.riemann_tubes(ntubes=4096, lmin=256, lmax=8192, seed=0)
    stream = torch.cuda.Stream()
    s = ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision=precision, stream=stream)
    with torch.cuda.stream(stream):
        U = s.prim_to_cons(s.tensor(Q))
        ws.ws_autotune(s.ctx, U, 1)
        ws.ws_set_graph(s.ctx, True)
        U0 = U.cpu().numpy()
        s.step(U)
    stream.synchronize()
    Ug = U.cpu().numpy()
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(4096, size=32, replace=False))
    sub_off, sub_U = _sub_batch(off, U0, pick)
    Uo, _ = oracle.tubes_step(sub_off, sub_U)
    for k, t in enumerate(pick):
        g = Ug[:, off[t] + 3:off[t + 1] - 3]
        o = Uo[:, sub_off[k] + 3:sub_off[k + 1] - 3]
        if precision == "fp64":
            assert np.array_equal(g, o), t
        else:
            assert l1_rel(g[0], o[0]) < 2e-5, t
    s.close()


def test_drop_3d_mixed_close_to_oracle():
    """3D periodic water drop with density noise (24^3), 4 CFL steps of the
    generic mixed kernels against the FP64 oracle."""
    case = wl.drop_3d(24, seed=0)
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(3, case.Q)
    U = s.tensor(Uo)
    for _ in range(4):
        dt = oracle.cfl_dt(g, Uo)
        s.step(U, dt)
        Uo, _, _ = oracle.step(g, Uo, dt=dt)
    sl = wl.interior(3, case.n)
    assert l1_rel(U.cpu().numpy()[sl][0], Uo[sl][0]) < 1e-5
    Q = s.cons_to_prim(U).cpu().numpy()[sl]
    assert np.abs(Q[4] / 1e5 - 1.0).max() < 5e-3  # pressure equilibrium at FP32 resolution of E - Pi


@pytest.mark.parametrize("n,bc", [((37, 19, 17), ("transmissive",) * 3), ((40, 16, 33), ("periodic",) * 3),
                                  ((33, 31, 16), ("reflective",) * 3),
                                  ((5, 7, 64), ("transmissive", "reflective", "periodic")),
                                  ((64, 4, 3), ("periodic", "transmissive", "reflective"))])
def test_fused_3d_matches_generic(n, bc, monkeypatch):
    """The fused 3D stage (x and y faces per z plane, then z faces per y plane
    with the RK stage) and the generic per-direction kernels evaluate the same
    mixed-precision scheme: after 3 steps they agree to FP32 rounding on every
    field, with ragged tiles in all three directions and each boundary kind,
    and their MOOD masks agree on almost every face."""
    case = wl.random_state(3, n, seed=23, kind="two_phase")
    case.bc = tuple((b, b) for b in bc)
    Uo = oracle.prim_to_cons(3, case.Q)
    outs = []
    for fused in (True, False):
        if fused:
            monkeypatch.delenv("WS_NO_FUSED", raising=False)
        else:
            monkeypatch.setenv("WS_NO_FUSED", "1")
        s = solver_for(case)
        U = s.tensor(Uo)
        for _ in range(3):
            s.step(U, 1e-7)
        _, mask = s.mood(with_mask=True)
        outs.append((U.cpu().numpy(), mask.cpu().numpy()))
        s.close()
    sl = wl.interior(3, case.n)
    for f in range(7):
        a, b = outs[0][0][sl][f], outs[1][0][sl][f]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max() + 1e-300, f
    assert np.mean(outs[0][1] == outs[1][1]) > 0.99


def test_fused_3d_close_to_oracle_with_masks():
    """Two CFL steps of the fused 3D stage on a ragged two-phase grid against
    the FP64 oracle: every field within FP32-level L1 error, and the per-stage
    MOOD masks of all three directions equal on almost every face."""
    case = wl.random_state(3, (35, 17, 19), seed=29, kind="two_phase")
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(3, case.Q)
    U = s.tensor(Uo)
    for _ in range(2):
        dt = oracle.cfl_dt(g, Uo)
        s.step(U, dt)
        Uo, _, mo = oracle.step(g, Uo, dt=dt, with_mask=True)
    sl = wl.interior(3, case.n)
    Ug = U.cpu().numpy()[sl]
    for f in range(7):
        assert l1_rel(Ug[f], Uo[sl][f]) < 1e-5, f
    _, mask = s.mood(with_mask=True)
    m = mask.cpu().numpy()
    want = np.concatenate([np.concatenate([d.ravel() for d in mo[st]]) for st in range(3)])
    assert m.size == want.size
    assert np.mean(m == want) > 0.99


@pytest.mark.parametrize("n,bc,nsteps", [((70, 47), "transmissive", 1), ((64, 200), "transmissive", 1),
                                         ((64, 200), "periodic", 3), ((33, 10), "reflective", 2),
                                         ((40, 130), "periodic", 0)])
def test_run_host_banded_matches_device_steps(n, bc, nsteps):
    """ws_run_host on the fused 2D path copies the state in and out by bands
    of tile rows, overlapped with stage 0 of the first step and stage 2 of the
    last; the result, Δt and MOOD masks equal those of ws_step on a device
    copy bit for bit (1 to 8 bands, periodic wrap-around, zero steps)."""
    case = wl.random_state(2, n, seed=31, kind="two_phase")
    case.bc = ((bc, bc), (bc, bc))
    Uo = oracle.prim_to_cons(2, case.Q)
    s = solver_for(case)
    U = s.tensor(Uo)
    dts = [s.step(U, want_dt=True) for _ in range(nsteps)]
    _, mask = s.mood(with_mask=True)
    s.close()
    s2 = solver_for(case)
    Uh = torch.tensor(Uo).pin_memory()
    dt_used = np.zeros(1)
    ws.ws_run_host(s2.ctx, Uh, nsteps, 0.0, dt_used)
    _, mask2 = s2.mood(with_mask=True)
    s2.close()
    assert np.array_equal(Uh.numpy(), U.cpu().numpy())
    if nsteps:
        assert dt_used[0] == dts[-1]
        assert np.array_equal(mask.cpu().numpy(), mask2.cpu().numpy())


def _fp64_vs_mixed(case, nsteps):
    """Run the FP64 path (bit-identical to the oracle, see the parity tests)
    and the mixed path from the same state with the FP64 path's CFL steps."""
    s64 = ws.Solver(case.ndim, case.n, case.dx, case.bc, precision="fp64")
    s32 = solver_for(case)
    U64 = s64.prim_to_cons(s64.tensor(case.Q))
    U32 = s32.prim_to_cons(s32.tensor(case.Q))
    for _ in range(nsteps):
        dt = s64.step(U64, want_dt=True)
        s32.step(U32, dt)
    _, m64 = s64.mood(with_mask=True)
    _, m32 = s32.mood(with_mask=True)
    torch.cuda.synchronize()
    sl = wl.interior(case.ndim, case.n)
    out = (U32[sl].double(), U64[sl], float((m64 == m32).float().mean().item()))
    s64.close()
    s32.close()
    return out


def _l1_by_field(a, b, ndim):
    """Relative L1 difference per field; a momentum component is measured
    against the whole momentum (a component that is nearly zero everywhere,
    like the transverse momentum of a planar shock, has no scale of its own)."""
    mom = sum(float(b[1 + d].abs().sum()) for d in range(ndim))
    out = []
    for f in range(a.shape[0]):
        err = float((a[f] - b[f]).abs().sum())
        ref = mom if 1 <= f <= ndim else float(b[f].abs().sum())
        out.append(err / ref if ref > 0 else err)  # a field that is zero everywhere must stay exactly zero
    return out


def test_full_size_2d_mixed_vs_fp64():
    """The benchmark grid (1024^2 shock-bubble), fused 2D mixed stage against
    the FP64 path over 3 CFL steps: every field within 1e-6 relative L1 (a
    momentum component against the whole momentum) and
    MOOD masks equal on at least 99.99 % of the faces."""
    a, b, agree = _fp64_vs_mixed(wl.shock_bubble_2d(1024), 3)
    for f, e in enumerate(_l1_by_field(a, b, 2)):
        assert e < 1e-6, (f, e)
    assert agree > 0.9999


def test_full_size_3d_mixed_vs_fp64():
    """The 3D benchmark grid (256^3 periodic water drop), fused two-pass 3D
    mixed stage against the FP64 path over one CFL step: every field within
    1e-6 relative L1 (a momentum component against the whole momentum) and
    MOOD masks equal on at least 99.99 % of the faces."""
    a, b, agree = _fp64_vs_mixed(wl.drop_3d(256, seed=0), 1)
    for f, e in enumerate(_l1_by_field(a, b, 3)):
        assert e < 1e-6, (f, e)
    assert agree > 0.9999


@pytest.mark.parametrize("make", [lambda: wl.haas_sturtevant("R22", 150, 50), lambda: wl.haas_sturtevant("He", 150, 50),
                                  lambda: wl.shock_droplet(64)], ids=["air_R22", "air_He", "shock_droplet"])
def test_shock_interface_setups_mixed_close_to_oracle(make):
    """The Sec. 6.1 and 6.2 setups, down-sized, MOOD off: 10 steps of the
    fused mixed stage with the oracle's time steps, every field within 1e-5
    relative L1 (a momentum component against the whole momentum)."""
    case = make()
    s = solver_for(case, mood=False)
    g = ogrid(case, mood=False)
    Uo = oracle.prim_to_cons(2, case.Q)
    U = s.tensor(Uo)
    for _ in range(10):
        dt = oracle.cfl_dt(g, Uo)
        s.step(U, dt)
        Uo, _, _ = oracle.step(g, Uo, dt=dt)
    sl = wl.interior(2, case.n)
    a = torch.tensor(U.cpu().numpy()[sl])
    b = torch.tensor(Uo[sl])
    for f, e in enumerate(_l1_by_field(a, b, 2)):
        assert e < 1e-5, (f, e)


@pytest.mark.parametrize("ndim,n", [(2, (1, 9)), (2, (9, 1)), (2, (2, 2)), (2, (33, 1)), (3, (1, 1, 7)),
                                    (3, (5, 1, 1)), (3, (2, 2, 2)), (3, (1, 16, 3))])
def test_fused_degenerate_extents_close_to_oracle(ndim, n):
    """The fused mixed stages on grids one or two cells wide in some
    directions (one partial tile, the halo mostly boundary images): 3 steps
    with the oracle's time steps, every field within 1e-5 relative L1 (a
    momentum component against the whole momentum)."""
    case = wl.random_state(ndim, n, seed=41, kind="shock")
    s = solver_for(case)
    g = ogrid(case)
    Uo = oracle.prim_to_cons(ndim, case.Q)
    U = s.tensor(Uo)
    for _ in range(3):
        dt = oracle.cfl_dt(g, Uo)
        s.step(U, dt)
        Uo, _, _ = oracle.step(g, Uo, dt=dt)
    sl = wl.interior(ndim, case.n)
    a = torch.tensor(U.cpu().numpy()[sl])
    b = torch.tensor(Uo[sl])
    for f, e in enumerate(_l1_by_field(a, b, ndim)):
        assert e < 1e-5, (f, e)


@pytest.mark.parametrize("kind", ["drop_3d", "tubes"])
def test_run_host_unbanded_matches_device_steps(kind):
    """ws_run_host on the paths that copy the whole state in and out (the
    fused 3D stage, the batched tubes): the result and the last step's time
    steps equal those of ws_step on a device copy, bit for bit."""
    if kind == "drop_3d":
        case = wl.drop_3d(20, seed=2)
        Uo = oracle.prim_to_cons(3, case.Q)
        make = lambda: solver_for(case)  # noqa: E731
        nt = 1
    else:
        off, Q = _tubes_case(ntubes=40, lmin=64, lmax=700, seed=8)
        Uo = oracle.prim_to_cons(1, Q.reshape(5, 1, 1, -1)).reshape(5, -1)
        make = lambda: ws.Solver(1, (1,), (1.0,), tube_offsets=off, precision="mixed")  # noqa: E731
        nt = len(off) - 1
    s = make()
    U = s.tensor(Uo)
    for _ in range(3):
        dts = s.step(U, want_dt=True)
    s.close()
    s2 = make()
    Uh = torch.tensor(Uo).pin_memory()
    dt_used = np.zeros(max(nt, 1))
    ws.ws_run_host(s2.ctx, Uh, 3, 0.0, dt_used)
    s2.close()
    assert np.array_equal(Uh.numpy(), U.cpu().numpy())
    assert np.array_equal(dt_used[:nt], np.atleast_1d(dts))


@pytest.mark.parametrize("ndim,n,bc", [(2, (70, 47), "transmissive"), (2, (33, 65), "periodic"),
                                       (2, (40, 31), "reflective"), (2, (100, 64), "periodic"),
                                       (2, (104, 50), "reflective"), (2, (512, 300), "transmissive"),
                                       (3, (37, 19, 17), "transmissive"),
                                       (3, (16, 20, 33), "periodic"), (3, (72, 40, 12), "reflective")])
def test_stage_configs_bit_identical(ndim, n, bc):
    """Every fused-stage configuration ws_autotune chooses among (tile shape,
    CTA size, loads cell by cell or as TMA boxes, launch mode) gives the same
    state, dt and MOOD record bit for bit: the per-face arithmetic does not
    depend on the tile, and a TMA box holds the values the cell-by-cell loads
    read (the larger 2D and 3D grids have tiles whose halo lies inside the
    grid, the ones that load by TMA).  ws_autotune then keeps one of them and reports
    it."""
    kind = "two_phase"
    case = wl.random_state(ndim, n, seed=23, kind=kind)
    bcs = tuple((bc, bc) for _ in range(ndim))
    stream = torch.cuda.Stream()
    ref = None
    s = ws.Solver(ndim, case.n, case.dx, bcs, precision="mixed", stream=stream)
    cands = list(range(16)) if ndim == 2 else list(range(8))
    with torch.cuda.stream(stream):
        U0 = s.prim_to_cons(s.tensor(case.Q))
        with pytest.raises(ws.WsError):
            ws.ws_set_stage_config(s.ctx, len(cands))
        for k in cands:
            ws.ws_set_stage_config(s.ctx, k)
            cfg = ws.ws_get_stage_config(s.ctx)
            assert cfg["index"] == k and cfg["schedule"] == k % 2
            assert cfg["tma"] == (k // 2) % 2
            rows = -(-n[1] // 15)
            if ndim == 2 and k >= 12:  # 32 x 15 rows closed by 32 x 7 rows
                assert 0 <= cfg["tail_rows"] <= rows and cfg["tile_y"] == 15 and cfg["threads"] == 512
            else:
                assert cfg["tail_rows"] == -1
            U = U0.clone()
            dts = [s.step(U, want_dt=True) for _ in range(3)]
            _, mask = s.mood(with_mask=True)
            got = (U.cpu().numpy(), dts, mask.cpu().numpy())
            if ref is None:
                ref = got
            else:
                assert np.array_equal(got[0], ref[0]), cfg
                assert got[1] == ref[1], cfg
                assert np.array_equal(got[2], ref[2]), cfg
        choice = ws.ws_autotune(s.ctx, U0, 2)
        assert choice in cands
        assert ws.ws_get_stage_config(s.ctx)["index"] == choice
        U = U0.clone()
        for _ in range(3):
            s.step(U)
        assert np.array_equal(U.cpu().numpy(), ref[0])
    s.close()


@pytest.mark.parametrize("n,bc,cfg", [((96, 96), "transmissive", 2), ((70, 47), "periodic", 1),
                                      ((100, 64), "periodic", 3), ((65, 40), "reflective", 10)])
def test_resident_steps_bit_identical(n, bc, cfg):
    """ws_set_resident: the FP32 image of the state carried from one step's
    stage 2 to the next step's stage 0 gives the same states, time steps and
    MOOD record, bit for bit, as converting the FP64 state every step; calls
    in between that touch the state (a census step on another state, a flux
    divergence) make the next step start over from the FP64 state."""
    if n == (96, 96):
        case = wl.shock_bubble_2d(96)
        bcs = case.bc
    else:
        case = wl.random_state(2, n, seed=31, kind="two_phase")
        bcs = ((bc, bc), (bc, bc))
    stream = torch.cuda.Stream()
    out = []
    with torch.cuda.stream(stream):
        for resident in (False, True):
            s = ws.Solver(2, case.n, case.dx, bcs, precision="mixed", stream=stream)
            ws.ws_set_stage_config(s.ctx, cfg)
            if resident:
                ws.ws_set_resident(s.ctx, True)
            U = s.prim_to_cons(s.tensor(case.Q))
            rec = []
            for k in range(12):
                if k == 5:  # calls on the context between steps
                    V = U.clone()
                    s.census_step(V)
                    s.flux_divergence(U.clone())
                dt = s.step(U, want_dt=True)
                _, mask = s.mood(with_mask=True)
                rec.append((dt, mask.cpu().numpy()))
            out.append((U.cpu().numpy(), rec))
            s.close()
    (a, ra), (b, rb) = out
    assert np.array_equal(a, b)
    for (dta, ma), (dtb, mb) in zip(ra, rb):
        assert dta == dtb
        assert np.array_equal(ma, mb)


@pytest.mark.parametrize("n,bc,cfg", [((37, 19, 17), "transmissive", 1), ((16, 20, 33), "periodic", 4),
                                      ((72, 40, 12), "transmissive", 3), ((72, 40, 12), "periodic", 7)])
def test_resident_steps_bit_identical_3d(n, bc, cfg):
    """The carried image in 3D: written by the second pass of stage 2, read by
    both passes of the next stage 0; bit-identical to ordinary steps."""
    case = wl.random_state(3, n, seed=32, kind="two_phase")
    bcs = tuple((bc, bc) for _ in range(3))
    out = []
    for resident in (False, True):
        s = ws.Solver(3, case.n, case.dx, bcs, precision="mixed")
        ws.ws_set_stage_config(s.ctx, cfg)
        if resident:
            ws.ws_set_resident(s.ctx, True)
        U = s.prim_to_cons(s.tensor(case.Q))
        dts = [s.step(U, want_dt=True) for _ in range(6)]
        out.append((U.cpu().numpy(), dts))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_resident_needs_fused_stages():
    for prec, ndim, n in (("fp64", 2, (20, 20)), ("mixed", 1, (40,))):
        case = wl.random_state(ndim, n, seed=2, kind="two_phase")
        s = ws.Solver(ndim, case.n, case.dx, case.bc, precision=prec)
        with pytest.raises(ws.WsError) as ei:
            ws.ws_set_resident(s.ctx, True)
        assert ei.value.code == ws.WS_ENOTSUP
        s.close()
