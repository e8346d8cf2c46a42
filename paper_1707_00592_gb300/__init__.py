"""Python binding of libws_gb300.so (include/ws.h): argument marshalling only.

Every step of the solver runs in the library's CUDA kernels; torch provides
device memory and streams.  There is no CPU fallback: if the library is not
built, or no GPU is present, the calls raise.

The functions keep the C names (``ws_init``, ``ws_step``, ...); ``Solver``
bundles a context with its grid for convenience.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libws_gb300.so")
HEADER = os.path.join(HERE, "..", "include", "ws.h")

WS_OK, WS_EINVAL, WS_ECUDA, WS_ENONPHYS, WS_ETIMEOUT, WS_ENOTSUP = range(6)
BC = {"transmissive": 0, "periodic": 1, "reflective": 2}
PRECISION = {"fp64": 0, "mixed": 1}
WEIGHTS = {"modified": 0, "basic": 1, "js": 2}
NG = 3


class WsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ws error {code}: {msg}")
        self.code = code


class ws_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 6), ("ntubes", ctypes.c_int64),
                ("tube_offsets", ctypes.POINTER(ctypes.c_int64))]


class ws_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("weights", ctypes.c_int), ("mood", ctypes.c_int),
                ("learned", ctypes.c_int), ("eps", ctypes.c_double), ("cfl", ctypes.c_double),
                ("check", ctypes.c_int)]


_lib = None


def header_symbols() -> list:
    """Names of the entry points declared in include/ws.h."""
    with open(HEADER) as f:
        txt = f.read()
    return re.findall(r"^WS_API[^(]*?\b(ws_\w+)\(", txt, flags=re.M)


def load():
    """Load the built library (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    sig = {
        "ws_init": (ctypes.c_int, [ctypes.POINTER(ws_grid), ctypes.POINTER(ws_opts), vp, ctypes.POINTER(vp)]),
        "ws_state_size": (ctypes.c_int64, [vp]),
        "ws_mask_size": (ctypes.c_int64, [vp]),
        "ws_prim_to_cons": (ctypes.c_int, [vp, vp, vp]),
        "ws_cons_to_prim": (ctypes.c_int, [vp, vp, vp]),
        "ws_flux_divergence": (ctypes.c_int, [vp, vp, vp]),
        "ws_cfl_dt": (ctypes.c_int, [vp, vp, dp]),
        "ws_step": (ctypes.c_int, [vp, vp, ctypes.c_double, dp]),
        "ws_run_host": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.c_double, dp]),
        "ws_get_mood": (ctypes.c_int, [vp, vp, ctypes.POINTER(ctypes.c_int64)]),
        "ws_nonphysical": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "ws_census_step": (ctypes.c_int, [vp, vp, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_int64)]),
        "ws_last_error": (ctypes.c_char_p, [vp]),
        "ws_init_error": (ctypes.c_char_p, []),
        "ws_destroy": (None, [vp]),
        "ws_profile": (ctypes.c_int, [vp, ctypes.c_int]),
        "ws_set_graph": (ctypes.c_int, [vp, ctypes.c_int]),
        "ws_set_stage_config": (ctypes.c_int, [vp, ctypes.c_int]),
        "ws_set_resident": (ctypes.c_int, [vp, ctypes.c_int]),
        "ws_get_stage_config": (ctypes.c_int, [vp] + [ctypes.POINTER(ctypes.c_int)] * 7),
        "ws_autotune": (ctypes.c_int, [vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "ws_set_mlp": (ctypes.c_int, [vp, vp, ctypes.c_float, ctypes.c_int]),
        "ws_gate_eval": (ctypes.c_int, [vp, vp, vp]),
        "ws_gate_stats": (ctypes.c_int, [vp, dp]),
        "ws_face_samples": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.c_int64, vp, vp,
                                           ctypes.POINTER(ctypes.c_int64)]),
        "ws_mlp_forward": (ctypes.c_int, [vp, vp, ctypes.c_int64, vp, vp]),
        "ws_mlp_grad": (ctypes.c_int, [vp, vp, vp, ctypes.c_int64, ctypes.c_float, vp, vp, vp]),
        "ws_mlp_adam": (ctypes.c_int, [vp, vp, vp, vp, ctypes.c_int64, ctypes.c_float, vp]),
        "ws_profile_read": (ctypes.c_int, [vp, dp, ctypes.POINTER(ctypes.c_int64)]),
        "ws_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, dp]),
        "ws_convert_probe": (ctypes.c_int, [ctypes.c_int64, vp, vp, vp]),
        "ws_flux_divergence_noalloc": (ctypes.c_int, [ctypes.POINTER(ws_grid), ctypes.POINTER(ws_opts), vp, vp, vp,
                                                      ctypes.c_char_p, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc):
    if rc != WS_OK:
        L = load()
        msg = (L.ws_last_error(ctx) if ctx else L.ws_init_error()).decode()
        raise WsError(rc, msg)


def make_grid(ndim, n, dx, bc=None, tube_offsets=None):
    g = ws_grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = int(n[d]) if d < ndim else 1
        g.dx[d] = float(dx[d]) if d < ndim else 1.0
    bc = bc or tuple(("transmissive", "transmissive") for _ in range(ndim))
    for d in range(ndim):
        g.bc[2 * d] = BC[bc[d][0]]
        g.bc[2 * d + 1] = BC[bc[d][1]]
    keep = None
    if tube_offsets is not None:
        keep = np.ascontiguousarray(tube_offsets, dtype=np.int64)
        g.ntubes = keep.size - 1
        g.tube_offsets = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    return g, keep


def make_opts(precision="fp64", weights="modified", mood=True, learned=False, eps=0.0, cfl=0.5, check=False):
    o = ws_opts()
    o.precision = PRECISION[precision]
    o.weights = WEIGHTS[weights]
    o.mood = int(bool(mood))
    o.learned = int(bool(learned))
    o.eps = float(eps)
    o.cfl = float(cfl)
    o.check = int(bool(check))
    return o


def ws_init(grid: ws_grid, opts: ws_opts, stream: int = 0):
    ctx = ctypes.c_void_p()
    _check(None, load().ws_init(ctypes.byref(grid), ctypes.byref(opts), ctypes.c_void_p(stream), ctypes.byref(ctx)))
    return ctx


def ws_state_size(ctx) -> int:
    return int(load().ws_state_size(ctx))


def ws_mask_size(ctx) -> int:
    return int(load().ws_mask_size(ctx))


def ws_prim_to_cons(ctx, Q, U):
    _check(ctx, load().ws_prim_to_cons(ctx, _ptr(Q), _ptr(U)))


def ws_cons_to_prim(ctx, U, Q):
    _check(ctx, load().ws_cons_to_prim(ctx, _ptr(U), _ptr(Q)))


def ws_flux_divergence(ctx, U, L):
    _check(ctx, load().ws_flux_divergence(ctx, _ptr(U), _ptr(L)))


def ws_cfl_dt(ctx, U) -> float:
    dt = ctypes.c_double(0.0)
    _check(ctx, load().ws_cfl_dt(ctx, _ptr(U), ctypes.byref(dt)))
    return dt.value


def ws_step(ctx, U, dt: float = 0.0, dt_used: np.ndarray | None = None):
    p = dt_used.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if dt_used is not None else None
    _check(ctx, load().ws_step(ctx, _ptr(U), ctypes.c_double(dt), p))


def ws_run_host(ctx, U_host, nsteps: int, dt: float = 0.0, dt_used: np.ndarray | None = None):
    p = dt_used.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if dt_used is not None else None
    _check(ctx, load().ws_run_host(ctx, _ptr(U_host), int(nsteps), ctypes.c_double(dt), p))


def ws_get_mood(ctx, mask=None, counts: bool = True):
    c = (ctypes.c_int64 * 9)() if counts else None
    _check(ctx, load().ws_get_mood(ctx, _ptr(mask), c))
    return np.array(list(c), dtype=np.int64).reshape(3, 3) if counts else None


def ws_nonphysical(ctx) -> int:
    n = ctypes.c_int64(0)
    _check(ctx, load().ws_nonphysical(ctx, ctypes.byref(n)))
    return n.value


CENSUS_KEYS = ("face_variables", "flat", "warp_passes", "warp_passes_weno")


def ws_census_step(ctx, U, dt: float = 0.0) -> dict:
    """One RK3 step of U with the counts of flat-stencil (linear-weight) and
    WENO-IS evaluations of the reconstruction (Sec. 3.3), summed over the
    three stages."""
    c = (ctypes.c_int64 * 4)()
    dt_used = ctypes.c_double(0.0)
    _check(ctx, load().ws_census_step(ctx, _ptr(U), ctypes.c_double(dt), ctypes.byref(dt_used), c))
    return {**dict(zip(CENSUS_KEYS, (int(v) for v in c))), "dt": dt_used.value}


KERNEL_CLASSES = ["ghost", "prim", "cfl", "face", "update", "other"]
NKERNEL = 8


MLP_NPARAM = 1889
MLP_NIN = 24


def ws_face_samples(ctx, U, stride: int, max_out: int, feats, labels) -> int:
    n = ctypes.c_int64(0)
    _check(ctx, load().ws_face_samples(ctx, _ptr(U), int(stride), int(max_out), _ptr(feats), _ptr(labels),
                                       ctypes.byref(n)))
    return n.value


def _stream_ptr(stream):
    return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)


def ws_mlp_forward(params, X, logits, stream=None):
    rc = load().ws_mlp_forward(_ptr(params), _ptr(X), X.shape[0], _ptr(logits), _stream_ptr(stream))
    if rc != WS_OK:
        raise WsError(rc, "ws_mlp_forward failed")


def ws_mlp_grad(params, X, y, pos_weight, grad, loss, stream=None):
    rc = load().ws_mlp_grad(_ptr(params), _ptr(X), _ptr(y), X.shape[0], ctypes.c_float(pos_weight), _ptr(grad),
                            _ptr(loss), _stream_ptr(stream))
    if rc != WS_OK:
        raise WsError(rc, "ws_mlp_grad failed")


def ws_mlp_adam(params, m, v, grad, step, lr, stream=None):
    rc = load().ws_mlp_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), int(step), ctypes.c_float(lr),
                            _stream_ptr(stream))
    if rc != WS_OK:
        raise WsError(rc, "ws_mlp_adam failed")


GATE_REDO_MOOD, GATE_REDO_DRIFT, GATE_REDO_NONPHYS, GATE_PER_STEP = 1, 2, 4, 8


def ws_set_mlp(ctx, params, threshold: float, flags: int = GATE_REDO_DRIFT | GATE_REDO_NONPHYS):
    _check(ctx, load().ws_set_mlp(ctx, _ptr(params), ctypes.c_float(threshold), int(flags)))


def ws_gate_eval(ctx, U, smooth):
    _check(ctx, load().ws_gate_eval(ctx, _ptr(U), _ptr(smooth)))


def ws_gate_stats(ctx) -> dict:
    out = (ctypes.c_double * 6)()
    _check(ctx, load().ws_gate_stats(ctx, out))
    return {"steps": int(out[0]), "redone": int(out[1]), "smooth_faces": out[2], "faces": out[3],
            "max_drift": out[4], "constant_faces": out[5]}


def ws_autotune(ctx, U, steps: int = 3) -> int:
    choice = ctypes.c_int(-1)
    _check(ctx, load().ws_autotune(ctx, _ptr(U), int(steps), ctypes.byref(choice)))
    return choice.value


def ws_set_resident(ctx, enable: bool):
    _check(ctx, load().ws_set_resident(ctx, int(bool(enable))))


def ws_set_stage_config(ctx, index: int):
    _check(ctx, load().ws_set_stage_config(ctx, int(index)))


def ws_get_stage_config(ctx) -> dict:
    v = [ctypes.c_int(0) for _ in range(7)]
    _check(ctx, load().ws_get_stage_config(ctx, *[ctypes.byref(x) for x in v]))
    return dict(zip(("index", "tile_x", "tile_y", "threads", "schedule", "tma", "tail_rows"), (x.value for x in v)))


def ws_set_graph(ctx, enable: bool):
    _check(ctx, load().ws_set_graph(ctx, int(bool(enable))))


def ws_profile(ctx, enable: bool, reset: bool = True):
    _check(ctx, load().ws_profile(ctx, (1 if reset else 2) if enable else 0))


def ws_profile_read(ctx):
    """{class: (ms, launches)} since the last ws_profile(ctx, True)."""
    ms = (ctypes.c_double * NKERNEL)()
    n = (ctypes.c_int64 * NKERNEL)()
    _check(ctx, load().ws_profile_read(ctx, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_CLASSES)}


def ws_peak_probe(kind: str, blocks: int = 0) -> float:
    """Measured FMA peak in TFLOP/s (2 flops per FMA); kind 'fp64' or 'fp32'."""
    t = ctypes.c_double(0.0)
    rc = load().ws_peak_probe({"fp64": 0, "fp32": 1}[kind], int(blocks), ctypes.byref(t))
    if rc != WS_OK:
        raise WsError(rc, "peak probe failed")
    return t.value


def ws_flux_divergence_noalloc(grid: ws_grid, opts: ws_opts, stream: int, U, L):
    """L(U) without any device allocation (static scratch inside the library);
    for callers that cannot call cudaMalloc.  U and L must be contiguous
    float64 CUDA tensors on one device, each holding at least one padded state
    of the grid (the C side cannot check buffer sizes); the call runs with that
    device current.  Raises ValueError on a bad tensor and WsError with the
    library's message on a failing call."""
    import torch
    nv = grid.ndim + 4
    need = nv
    for d in range(max(1, min(grid.ndim, 3))):
        need *= int(grid.n[d]) + 2 * NG
    for name, t in (("U", U), ("L", L)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} doubles; the grid's padded state needs {need}")
    if U.device != L.device:
        raise ValueError("U and L must be on the same device")
    buf = ctypes.create_string_buffer(256)
    with torch.cuda.device(U.device):
        rc = load().ws_flux_divergence_noalloc(ctypes.byref(grid), ctypes.byref(opts), ctypes.c_void_p(stream),
                                               _ptr(U), _ptr(L), buf, 256)
    if rc != WS_OK:
        raise WsError(rc, buf.value.decode())


def ws_convert_probe(x):
    """(FP32, widened FP64) images of a float64 CUDA tensor under the mixed
    kernels' integer-pipe conversions."""
    import torch
    o32 = torch.empty(x.numel(), dtype=torch.float32, device=x.device)
    o64 = torch.empty(x.numel(), dtype=torch.float64, device=x.device)
    rc = load().ws_convert_probe(x.numel(), _ptr(x), _ptr(o32), _ptr(o64))
    if rc != WS_OK:
        raise WsError(rc, "convert probe failed")
    return o32, o64


def ws_destroy(ctx):
    if ctx:
        load().ws_destroy(ctx)


class Solver:
    """A context plus its grid; state tensors are torch float64 on the GPU with
    the padded SoA layout of include/ws.h."""

    def __init__(self, ndim, n, dx, bc=None, tube_offsets=None, stream=None, **opts):
        import torch
        load()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.torch = torch
        self.ndim = ndim
        self.n = tuple(int(n[d]) if d < ndim else 1 for d in range(3))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.grid, self._keep = make_grid(ndim, n, dx, bc, tube_offsets)
        self.opts = make_opts(**opts)
        self.ctx = ws_init(self.grid, self.opts, self.stream.cuda_stream)
        self.size = ws_state_size(self.ctx)
        self.nmask = ws_mask_size(self.ctx)
        self.ntubes = 0 if tube_offsets is None else len(tube_offsets) - 1

    def shape(self):
        if self.ntubes:
            return (5, self.size // 5)
        P = [self.n[d] + 2 * NG if d < self.ndim else 1 for d in range(3)]
        return (self.ndim + 4, P[2], P[1], P[0])

    def tensor(self, a=None):
        t = self.torch.zeros(self.shape(), dtype=self.torch.float64, device="cuda")
        if a is not None:
            t.copy_(self.torch.as_tensor(np.ascontiguousarray(a)).reshape(self.shape()))
        return t

    def prim_to_cons(self, Q):
        U = self.tensor()
        ws_prim_to_cons(self.ctx, Q, U)
        return U

    def cons_to_prim(self, U):
        Q = self.tensor()
        ws_cons_to_prim(self.ctx, U, Q)
        return Q

    def flux_divergence(self, U):
        L = self.tensor()
        ws_flux_divergence(self.ctx, U, L)
        return L

    def cfl_dt(self, U):
        return ws_cfl_dt(self.ctx, U)

    def step(self, U, dt=0.0, want_dt=False):
        if want_dt:
            out = np.zeros(max(1, self.ntubes))
            ws_step(self.ctx, U, dt, out)
            return out if self.ntubes else float(out[0])
        ws_step(self.ctx, U, dt)
        return None

    def mood(self, with_mask=False):
        mask = None
        if with_mask:
            mask = self.torch.zeros(3 * self.nmask, dtype=self.torch.uint8, device="cuda")
        counts = ws_get_mood(self.ctx, mask, True)
        return counts, mask

    def nonphysical(self):
        return ws_nonphysical(self.ctx)

    def census_step(self, U, dt=0.0):
        return ws_census_step(self.ctx, U, dt)

    def close(self):
        if self.ctx:
            ws_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
