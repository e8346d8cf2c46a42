"""Learned smooth-face gate: the GPU training kernels against the FP64 MLP
oracle, and the face sampler's features and labels against the FP64 scheme
oracle."""
import numpy as np
import pytest

import oracle
from oracle import mlp_oracle as mo
from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402


def cuda(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_forward_matches_oracle():
    rng = np.random.default_rng(0)
    p = mo.init(3)
    X = rng.normal(size=(3000, mo.NIN))
    logits = torch.empty(3000, dtype=torch.float32, device="cuda")
    ws.ws_mlp_forward(cuda(p, torch.float32), cuda(X, torch.float32), logits)
    torch.cuda.synchronize()
    z, _ = mo.forward(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(logits.cpu().numpy(), z, rtol=1e-4, atol=1e-4 * np.abs(z).max())


def test_gradient_matches_oracle():
    """FP32 gradient of the weighted BCE against the FP64 back-propagation
    (itself pinned by finite differences)."""
    rng = np.random.default_rng(1)
    p = mo.init(4)
    X = rng.normal(size=(5000, mo.NIN))
    y = (rng.random(5000) < 0.3).astype(np.uint8)
    grad = torch.empty(mo.NPARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ws.ws_mlp_grad(cuda(p, torch.float32), cuda(X, torch.float32), cuda(y, torch.uint8), 2.5, grad, loss)
    torch.cuda.synchronize()
    p32 = p.astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    g = mo.grad(p32, X32, y, 2.5)
    gg = grad.cpu().numpy()
    assert np.abs(gg - g).max() <= 2e-4 * np.abs(g).max()
    assert loss.item() == pytest.approx(mo.loss(p32, X32, y, 2.5), rel=1e-4)


def test_gradient_is_deterministic():
    """The gradient and loss sums are formed in fixed point, so the order in
    which threads and blocks add their contributions does not change a bit:
    repeated calls (with enough samples to fill every block) agree exactly,
    and with the oracle as above."""
    rng = np.random.default_rng(5)
    p = mo.init(6)
    X = rng.normal(size=(200_000, mo.NIN))
    y = (rng.random(200_000) < 0.25).astype(np.uint8)
    P, Xd, yd = cuda(p, torch.float32), cuda(X, torch.float32), cuda(y, torch.uint8)
    out = []
    for _ in range(4):
        grad = torch.empty(mo.NPARAM, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        ws.ws_mlp_grad(P, Xd, yd, 3.0, grad, loss)
        torch.cuda.synchronize()
        out.append((grad.cpu().numpy(), loss.item()))
    for g, l in out[1:]:
        assert np.array_equal(g, out[0][0])
        assert l == out[0][1]
    g64 = mo.grad(p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64), y, 3.0)
    assert np.abs(out[0][0] - g64).max() <= 2e-4 * np.abs(g64).max()


def test_adam_step():
    rng = np.random.default_rng(2)
    p = rng.normal(size=mo.NPARAM)
    g = rng.normal(size=mo.NPARAM)
    P, M, V = cuda(p, torch.float32), torch.zeros(mo.NPARAM, device="cuda"), torch.zeros(mo.NPARAM, device="cuda")
    ws.ws_mlp_adam(P, M, V, cuda(g, torch.float32), 1, 1e-3)
    torch.cuda.synchronize()
    # step 1 of Adam: m_hat = g, v_hat = g^2, so p -= lr g / (|g| + eps)
    expect = p - 1e-3 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(P.cpu().numpy(), expect, rtol=1e-5, atol=1e-6)


def oracle_face_features(qc, cc):
    """FP64 features and label of one face from the oracle's own functions,
    and whether every decision behind the label clears the FP32 noise of the
    kernel's evaluation.  The kernel's characteristic values carry about 3e-7
    of the scale of the terms the projection adds (p and rho_bar c_bar u_n for
    the acoustic variables, rho and p / c_bar^2 for the entropy variable; a few
    FP32 ulps), and WENO-IS minus the linear-weight value about twice that; a
    flatness test within 3e-7 of that scale of its threshold, a |WENO-IS -
    linear| > 1e-6 range comparison within 6e-7 of it, or an admissibility test
    within 1e-5 of its terms' scale of zero, counts as undecided."""
    nq = qc.shape[1]
    rho_bar = 0.5 * (qc[2, 0] + qc[3, 0])
    c_bar = 0.5 * (cc[2] + cc[3])
    Lm, Rm = oracle.char_matrices(nq, rho_bar, c_bar)
    w = qc @ Lm.T
    ip = nq - 3
    term = {0: 0.5 * np.max(np.abs(qc[:, ip]) + np.abs(rho_bar * c_bar * qc[:, 1])),
            nq - 1: 0.5 * np.max(np.abs(qc[:, ip]) + np.abs(rho_bar * c_bar * qc[:, 1])),
            1: np.max(np.abs(qc[:, 0]) + np.abs(qc[:, ip]) / (c_bar * c_bar))}
    feats = []
    rough = False
    robust = True
    full = np.zeros((2, nq))
    flat_gamma = False
    for r in range(nq):
        col = w[:, r]
        span = col.max() - col.min()
        mag = max(abs(col.max()), abs(col.min()))
        eta = 3e-7 * max(term.get(r, mag), mag)
        rng_ = span + 1e-30
        flat_r = span <= 1e-6 * mag
        shear = 2 <= r < ip
        if not shear and span > 0.0 and abs(span - 1e-6 * mag) < eta:
            robust = False
        if r == ip:
            flat_gamma = flat_r
        for side in range(2):
            v = col[0:5] if side == 0 else col[5:0:-1]
            f, _ = oracle.weno_is(v)
            lin = v[2] + (2 * (v[0] - v[2]) - 13 * (v[1] - v[2]) + 27 * (v[3] - v[2]) - 3 * (v[4] - v[2])) / 60.0
            flat = flat_r or (r == ip + 1 and flat_gamma)
            if not shear and not flat:
                if abs(f - lin) > 1e-6 * rng_:
                    rough = True
                if abs(abs(f - lin) - 1e-6 * rng_) < 2 * eta:
                    robust = False
            full[side, r] = f
    cond = []
    for r in (0, 1, nq - 1, nq - 3):
        col = w[:, r]
        span = col.max() - col.min()
        mag = max(abs(col.max()), abs(col.min()))
        inv = 1.0 / (span + 1e-30) if span > 1e-6 * mag else 0.0
        feats.append((col - col.mean()) * inv)
        cond.append(np.full(6, span > 1e-3 * mag or span == 0.0))
    for side in range(2):
        q = Rm @ full[side]
        if not (q[0] > 0 and q[-2] > 0 and (q[-2] + 1) * q[-3] + q[-1] > 0):
            rough = True
        if abs(q[0]) < 1e-5 * np.abs(qc[:, 0]).max():
            robust = False
        if abs((q[-2] + 1) * q[-3] + q[-1]) < 1e-5 * (abs((q[-2] + 1) * q[-3]) + abs(q[-1])):
            robust = False
    return np.concatenate(feats), int(rough), np.concatenate(cond), robust


@pytest.mark.parametrize("kind,stride,least", [("shock_bubble", 3, 0.75), ("two_phase", 7, 0.25)])
def test_face_samples_match_oracle(kind, stride, least):
    """Features and labels of the sampled faces against the FP64 scheme
    oracle: every label whose decisions clear the FP32 noise band agrees
    exactly.  On the shock-bubble (15 steps in) most faces are decided; on a
    random two-phase state, with a jump at nearly every face, far fewer."""
    if kind == "shock_bubble":
        case = wl.shock_bubble_2d(96)
        g = oracle.Grid(2, case.n, case.dx, case.bc)
        Uo = oracle.prim_to_cons(2, case.Q)
        for _ in range(15):
            Uo, _, _ = oracle.step(g, Uo)
    else:
        case = wl.random_state(2, (64, 48), seed=6, kind=kind)
        Uo = oracle.prim_to_cons(2, case.Q)
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
    U = s.tensor(Uo)
    nmax = 8000
    feats = torch.empty((nmax, 24), dtype=torch.float32, device="cuda")
    labels = torch.empty(nmax, dtype=torch.uint8, device="cuda")
    n = ws.ws_face_samples(s.ctx, U, stride, nmax, feats, labels)
    F = feats.cpu().numpy()[:n]
    Lb = labels.cpu().numpy()[:n]
    Uf = oracle.fill_ghosts(oracle.Grid(2, case.n, case.dx, case.bc), Uo)
    Q = oracle.cons_to_prim(2, Uf)
    nx, ny = case.n[0], case.n[1]
    decided = 0
    out = 0
    for d in range(2):
        fe = [nx + (d == 0), ny + (d == 1)]
        nf = fe[0] * fe[1]
        for sidx in range((nf + stride - 1) // stride):
            f = sidx * stride
            fx, fy = f % fe[0], f // fe[0]
            c = [fx, fy]
            c[d] -= 1
            cells = []
            for j in range(6):
                cc_ = [3 + c[0], 3 + c[1]]
                cc_[d] += j - 2
                cells.append(Q[:, 0, cc_[1], cc_[0]])
            cells = np.array(cells)
            perm = [0, 1 + d, 2 - d, 3, 4, 5]
            qc = cells[:, perm]
            cc = np.array([oracle.sound_speed(q[0], q[3], q[4], q[5]) for q in qc])
            feat, lab, cond, robust = oracle_face_features(qc, cc)
            # features of stencils flat to < 1e-3 of their magnitude carry FP32 noise
            np.testing.assert_allclose(F[out][cond], feat[cond], atol=2e-3)
            if robust:
                assert Lb[out] == lab, (d, f)
                decided += 1
            out += 1
    assert out == n
    assert decided >= least * n, (decided, n)


def _shock_bubble_state(n):
    case = wl.shock_bubble_2d(n)
    s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
    U = s.prim_to_cons(s.tensor(case.Q))
    for _ in range(15):  # let the shock enter the bubble
        s.step(U)
    return case, s, U


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as FP64."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_logits(p, X):
    """The MLP oracle's forward pass with the roundings of the tensor-core
    gate: BF16 features, weights and hidden activations, exact products,
    biases in FP32 (accumulation in FP64 here, FP32 on the GPU)."""
    w = mo.unpack(p)
    h1 = bf16(np.maximum(bf16(X) @ bf16(w["W1"]).T + w["b1"].astype(np.float32), 0.0))
    h2 = bf16(np.maximum(h1 @ bf16(w["W2"]).T + w["b2"].astype(np.float32), 0.0))
    return h2 @ bf16(w["W3"]) + np.float32(w["b3"][0]), h2


def test_tensor_core_gate_matches_mlp_oracle():
    """The gate's decisions inside the fused stage kernel (BF16 features and
    weights on the tensor cores, FP32 accumulation) against the FP64 MLP oracle
    on the sampled features of the same faces.  A face is exempt when BF16
    rounding decides it: the oracle logit and the logit with the kernel's BF16
    roundings lie on different sides of the threshold, or the rounded logit is
    within reach of the threshold for a one-step change in the BF16 rounding of
    its most influential feature (the two feature computations differ in the
    last FP32 bits) plus FP32 accumulation noise.  Every other face agrees
    exactly, and they are nearly all the faces."""
    from paper_1707_00592_gb300 import learned
    case, s, U = _shock_bubble_state(96)
    P = torch.tensor(learned.init_params(7), dtype=torch.float32, device="cuda")
    nf = s.nmask
    feats = torch.empty((nf, 24), dtype=torch.float32, device="cuda")
    labels = torch.empty(nf, dtype=torch.uint8, device="cuda")
    n = ws.ws_face_samples(s.ctx, U, 1, nf, feats, labels)
    assert n == nf
    X = feats.cpu().numpy().astype(np.float64)
    p64 = P.cpu().numpy().astype(np.float64)
    z, _ = mo.forward(p64, X)
    # the threshold: the median logit of the faces with non-zero features
    # (every flat face has the same logit, which must not sit on the threshold)
    thr = float(np.median(z[np.abs(X).max(axis=1) > 0]))
    ws.ws_set_mlp(s.ctx, P, thr)
    smooth = torch.empty(nf, dtype=torch.uint8, device="cuda")
    ws.ws_gate_eval(s.ctx, U, smooth)
    torch.cuda.synchronize()
    got = smooth.cpu().numpy().astype(bool)
    zb, h2 = bf16_logits(p64, X)
    w = mo.unpack(p64)
    influence = np.abs(w["W3"]) @ np.abs(w["W2"]) @ np.abs(w["W1"])  # first-order d z / d x_k bound
    reach = 2.0 ** -8 * np.max(np.abs(X) * influence[None, :], axis=1)
    reach += 1e-5 * (np.abs(h2) @ np.abs(bf16(w["W3"])) + abs(w["b3"][0]))
    decided = (np.sign(z - thr) == np.sign(zb - thr)) & (np.abs(zb - thr) > reach)
    assert np.array_equal(got[decided], (z < thr)[decided])
    nonflat = np.abs(X).max(axis=1) > 0
    assert decided.mean() > 0.95, decided.mean()
    assert decided[nonflat].mean() > 0.85, decided[nonflat].mean()
    s.close()


@pytest.mark.parametrize("per_step", [False, True])
def test_gate_closed_equals_plain_step_bitwise(per_step):
    """With a threshold no logit falls below, every face keeps WENO-IS and the
    gated kernel reproduces the plain fused kernel bit for bit, whether the MLP
    runs in every RK stage or once per step (stages 1 and 2 reusing stage 0's
    decisions)."""
    from paper_1707_00592_gb300 import learned
    flags = ws.GATE_REDO_DRIFT | ws.GATE_REDO_NONPHYS | (ws.GATE_PER_STEP if per_step else 0)
    case = wl.random_state(2, (70, 47), seed=8, kind="two_phase")
    Uo = oracle.prim_to_cons(2, case.Q)
    outs = []
    for gated in (False, True):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
        if gated:
            P = torch.tensor(learned.init_params(1), dtype=torch.float32, device="cuda")
            ws.ws_set_mlp(s.ctx, P, -1e30, flags)
        U = s.tensor(Uo)
        for _ in range(3):
            s.step(U)
        outs.append(U.cpu().numpy())
        if gated:
            st = ws.ws_gate_stats(s.ctx)
            assert st["steps"] == 3 and st["smooth_faces"] == 0 and st["redone"] == 0
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_gate_open_without_redo_runs_linear_weights():
    """Threshold above every logit, no redo: every face takes the linear
    weights for all but the shear variable (MOOD still applies).  On a smooth
    periodic wave the result stays within 1e-5 (L1) of the plain WENO-IS step."""
    from paper_1707_00592_gb300 import learned
    case = wl.entropy_wave(64, 2, amp=0.2, kind="sine")
    Uo = oracle.prim_to_cons(2, case.Q)
    outs = []
    for gated in (False, True):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
        if gated:
            P = torch.tensor(learned.init_params(1), dtype=torch.float32, device="cuda")
            ws.ws_set_mlp(s.ctx, P, 1e30, 0)
        U = s.tensor(Uo)
        for _ in range(10):
            s.step(U)
        outs.append(U.cpu().numpy())
        if gated:
            st = ws.ws_gate_stats(s.ctx)
            assert st["smooth_faces"] + st["constant_faces"] == st["faces"] > 0 and st["redone"] == 0
        s.close()
    sl = wl.interior(2, case.n)
    a, b = outs[1][sl][0], outs[0][sl][0]
    assert np.abs(a - b).sum() / np.abs(b).sum() < 1e-5


def test_gate_open_per_step_equals_per_stage_bitwise():
    """Threshold above every logit: every stage's decisions are 'smooth', so
    reusing stage 0's decisions in stages 1 and 2 gives the per-stage result
    bit for bit (the reuse launches read the stored decisions and stage the
    own cells in shared memory; the arithmetic is the same)."""
    from paper_1707_00592_gb300 import learned
    case = wl.random_state(2, (70, 47), seed=9, kind="smooth")  # linear weights stay stable here
    Uo = oracle.prim_to_cons(2, case.Q)
    outs = []
    for flags in (0, ws.GATE_PER_STEP):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
        P = torch.tensor(learned.init_params(1), dtype=torch.float32, device="cuda")
        ws.ws_set_mlp(s.ctx, P, 1e30, flags)
        U = s.tensor(Uo)
        for _ in range(3):
            s.step(U, 1e-7)
        outs.append(U.cpu().numpy())
        st = ws.ws_gate_stats(s.ctx)
        assert st["steps"] == 3 and st["redone"] == 0 and st["smooth_faces"] > 0
        s.close()
    assert np.isfinite(outs[0]).all()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("graph", [False, True])
def test_gate_redo_restores_and_equals_plain(graph):
    """Linear weights everywhere on a two-phase state fail the drift check, so
    every gated step is redone without the gate from the stage-0 backup of U:
    the result equals the plain path bit for bit and every step counts as
    redone.  graph=True runs the step as one CUDA graph whose redo branch is a
    conditional node set on the device; graph=False launches the redo stages
    with a device-side run-if flag."""
    from paper_1707_00592_gb300 import learned
    case = wl.random_state(2, (70, 47), seed=12, kind="two_phase")
    Uo = oracle.prim_to_cons(2, case.Q)
    outs = []
    for gated in (False, True):
        stream = torch.cuda.Stream() if graph else None
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed", stream=stream)
        if gated:
            P = torch.tensor(learned.init_params(1), dtype=torch.float32, device="cuda")
            ws.ws_set_mlp(s.ctx, P, 1e30, ws.GATE_REDO_DRIFT | ws.GATE_REDO_NONPHYS)
        with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
            U = s.tensor(Uo)
            for _ in range(4):
                s.step(U, 1e-7)
            torch.cuda.synchronize()
        outs.append(U.cpu().numpy())
        if gated:
            st = ws.ws_gate_stats(s.ctx)
            assert st["steps"] == 4 and st["redone"] == 4, st
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_trained_gate_ab():
    """A/B of the trained gate on a 256^2 shock-bubble (60 CFL steps): the
    plain mixed path, the gated path (MLP trained on the GPU by this library's
    kernels, threshold at recall 0.999), and the linear weights everywhere
    (no gate, no redo).  The gate keeps the result within 1e-6 (L1) of the
    plain path while sending most faces to the linear weights; the linear
    weights everywhere either break down or err by orders of magnitude more.
    Timings are printed (the gate's MLP costs about what it saves on this
    workload; see the benchmark notes)."""
    import time
    from paper_1707_00592_gb300 import learned
    P, thr, rep = learned.train_gate(total=1_000_000, epochs=3)
    assert rep["recall"] >= 0.998
    case = wl.shock_bubble_2d(256)
    res = {}
    for mode in ("plain", "gated", "gated_per_step", "linear"):
        s = ws.Solver(2, case.n, case.dx, case.bc, precision="mixed")
        if mode == "gated":
            ws.ws_set_mlp(s.ctx, P, thr)
        elif mode == "gated_per_step":
            ws.ws_set_mlp(s.ctx, P, thr, ws.GATE_REDO_DRIFT | ws.GATE_REDO_NONPHYS | ws.GATE_PER_STEP)
        elif mode == "linear":
            ws.ws_set_mlp(s.ctx, P, 1e30, 0)
        U = s.prim_to_cons(s.tensor(case.Q))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(60):
            s.step(U, 2e-7)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / 60
        st = ws.ws_gate_stats(s.ctx) if mode != "plain" else None
        res[mode] = (U.cpu().numpy()[wl.interior(2, case.n)][0], dt, st)
        s.close()
    ref = res["plain"][0]
    l1 = {m: float(np.abs(r[0] - ref).sum() / np.abs(ref).sum()) for m, r in res.items()}
    print({m: (l1[m], round(r[1] * 1e3, 4), r[2]) for m, r in res.items()})
    gst = res["gated"][2]
    assert l1["gated"] < 1e-6
    assert l1["gated_per_step"] < 1e-6
    assert gst["smooth_faces"] > 0.3 * gst["faces"]
    assert not np.isfinite(l1["linear"]) or l1["linear"] > 100 * max(l1["gated"], 1e-12)
