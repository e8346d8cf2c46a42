"""The allocation-free flux divergence (ws_flux_divergence_noalloc).

Some callers cannot call cudaMalloc: an application whose device memory
belongs to another allocator or a fixed budget, or a loop that must not
allocate once running.  They cannot create a context, so this entry point
takes the grid and options directly and keeps its scratch in a fixed-size
array inside the library.  These tests call it through the C ABI and check
that it returns exactly what the context-based ws_flux_divergence returns
(the tolerance of the other GPU tests: bit for bit), on two calls in a row,
and that a grid too large for the array is refused with a clear message.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_1707_00592_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1707_00592_gb300 as ws  # noqa: E402


def same(a, b):
    return bool(np.all((a == b) | (np.isnan(a) & np.isnan(b))))


@pytest.mark.parametrize("ndim,n,kind,opt", [(2, (40, 35), "two_phase", {}), (3, (12, 10, 14), "two_phase", {}),
                                             (1, (97,), "shock", {}), (2, (40, 35), "two_phase", {"mood": False}),
                                             (2, (33, 20), "two_phase", {"weights": "basic"}),
                                             (1, (97,), "shock", {"weights": "js"})])
def test_noalloc_matches_context_path_twice(ndim, n, kind, opt):
    stream = torch.cuda.current_stream()
    cases = [wl.random_state(ndim, n, seed=s, kind=kind) for s in (11, 12)]
    s = ws.Solver(ndim, cases[0].n, cases[0].dx, cases[0].bc, stream=stream, **opt)
    grid, _ = ws.make_grid(ndim, cases[0].n, cases[0].dx, cases[0].bc)
    opts = ws.make_opts(**opt)
    sl = wl.interior(ndim, cases[0].n)
    free = []
    for case in cases:  # two calls in a row, different states
        U = s.prim_to_cons(s.tensor(case.Q))
        L_ref = s.flux_divergence(U.clone())
        L = torch.full_like(U, float("nan"))
        torch.cuda.synchronize()
        before = torch.cuda.mem_get_info()[0]
        ws.ws_flux_divergence_noalloc(grid, opts, stream.cuda_stream, U, L)
        torch.cuda.synchronize()
        free.append((before, torch.cuda.mem_get_info()[0]))
        assert same(L.cpu().numpy()[sl], L_ref.cpu().numpy()[sl])
    # the second call allocates nothing on the device
    assert free[1][0] == free[1][1]
    s.close()


def test_noalloc_rejects_grid_beyond_scratch():
    grid, _ = ws.make_grid(2, (314, 314), (1.0 / 314, 1.0 / 314))
    U = torch.zeros(6 * 320 * 320, device="cuda", dtype=torch.float64)
    L = torch.zeros_like(U)
    with pytest.raises(ws.WsError) as ei:
        ws.ws_flux_divergence_noalloc(grid, ws.make_opts(), 0, U, L)
    assert ei.value.code == ws.WS_EINVAL
    assert "static scratch" in str(ei.value)


def test_noalloc_rejects_bad_options_and_buffers():
    grid, _ = ws.make_grid(2, (20, 20), (0.05, 0.05))
    U = torch.zeros(6 * 26 * 26, device="cuda", dtype=torch.float64)
    L = torch.zeros_like(U)
    for kw, code in (({"mood": 2}, ws.WS_EINVAL), ({"precision": 7}, ws.WS_EINVAL),
                     ({"precision": ws.PRECISION["mixed"]}, ws.WS_ENOTSUP)):
        o = ws.make_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        with pytest.raises(ws.WsError) as ei:
            ws.ws_flux_divergence_noalloc(grid, o, 0, U, L)
        assert ei.value.code == code
    with pytest.raises(ValueError):
        ws.ws_flux_divergence_noalloc(grid, ws.make_opts(), 0, U[:-1], L)
    with pytest.raises(ValueError):
        ws.ws_flux_divergence_noalloc(grid, ws.make_opts(), 0, U.float(), L)
