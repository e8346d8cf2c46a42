"""FP64 CPU oracle of the WENO-IS / MOOD / HLLC / SSP-RK3 scheme (arXiv 1707.00592).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  The arithmetic lives in
``weno_is_oracle.c`` (plain C, ``-O2 -ffp-contract=off``, no fast-math); this
module compiles it with gcc and marshals numpy arrays through ctypes.  It
shares no code with the CUDA library and never calls it.

Arrays use the padded structure-of-arrays layout ``U[field, z, y, x]`` with
3 ghost layers on both sides of every active direction; fields are
``(rho, rho u_1..rho u_ndim, E, Gamma, Pi)`` with ``Gamma = 1/(gamma-1)`` and
``Pi = gamma P_inf/(gamma-1)`` (Sec. 2, Eqs. eos and material-properties).
Parity status of each function is stated in the repository's design notes;
every function here is pinned by a ``-m "not gpu"`` test.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "weno_is_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libweno_is_oracle.so")
NG = 3

BC = {"transmissive": 0, "periodic": 1, "reflective": 2}
WEIGHTS = {"modified": 0, "basic": 1, "js": 2}


def default_eps(weights: str) -> float:
    """WENO epsilon: 1e-40 for WENO-IS (the paper leaves it open), 1e-6 for
    WENO-JS (Jiang & Shu's value)."""
    return 1e-6 if weights == "js" else 1e-40

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build``."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


class _Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", ctypes.c_int * 6), ("eps", ctypes.c_double), ("mood", ctypes.c_int),
                ("weights", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_weno_is.restype = ctypes.c_double
        L.or_weno_is.argtypes = [dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
        L.or_cfl_dt.restype = ctypes.c_double
        L.or_step.restype = ctypes.c_double
        L.or_count_nonphysical.restype = ctypes.c_int64
        L.or_sound_speed.restype = ctypes.c_double
        L.or_sound_speed.argtypes = [ctypes.c_double] * 4
        L.or_get_threads.restype = ctypes.c_int
        assert L.or_grid_sizeof() == ctypes.sizeof(_Grid)
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


@dataclass
class Grid:
    """Uniform Cartesian grid: ``n`` interior cells and ``dx`` per active direction."""
    ndim: int
    n: tuple
    dx: tuple
    bc: tuple = ()          # ((lo, hi), ...) per direction, names from BC
    eps: float = None       # None: default_eps(weights)
    mood: bool = True
    weights: str = "modified"
    _c: _Grid = field(default=None, repr=False, compare=False)

    def __post_init__(self):
        if self.eps is None:
            self.eps = default_eps(self.weights)
        if not self.bc:
            self.bc = tuple(("transmissive", "transmissive") for _ in range(self.ndim))
        g = _Grid()
        g.ndim = self.ndim
        for d in range(3):
            g.n[d] = int(self.n[d]) if d < self.ndim else 1
            g.dx[d] = float(self.dx[d]) if d < self.ndim else 1.0
            g.bc[2 * d] = BC[self.bc[d][0]] if d < self.ndim else 0
            g.bc[2 * d + 1] = BC[self.bc[d][1]] if d < self.ndim else 0
        g.eps = float(self.eps)
        g.mood = int(bool(self.mood))
        g.weights = WEIGHTS[self.weights]
        self._c = g

    @property
    def nv(self) -> int:
        return self.ndim + 4

    @property
    def padded_shape(self) -> tuple:
        P = [int(self.n[d]) + 2 * NG if d < self.ndim else 1 for d in range(3)]
        return (self.nv, P[2], P[1], P[0])

    def interior(self) -> tuple:
        sl = [slice(None)]
        for d in (2, 1, 0):
            sl.append(slice(NG, NG + int(self.n[d])) if d < self.ndim else slice(None))
        return tuple(sl)

    def mask_shapes(self) -> list:
        out = []
        for d in range(self.ndim):
            ext = [int(self.n[e]) if e < self.ndim else 1 for e in range(3)]
            ext[d] += 1
            out.append((ext[2], ext[1], ext[0]))
        return out


def fill_ghosts(g: Grid, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    lib().or_fill_ghosts(ctypes.byref(g._c), _dp(U))
    return U


def rhs(g: Grid, U: np.ndarray, with_mask: bool = True):
    """L(U) of Sec. 3.1 on the interior (ghosts are filled first from the BCs).

    Returns ``(L, masks)``: L on the padded layout (ghost entries 0), masks a
    list of uint8 arrays per direction (bits 0-1: left order code, 2-3: right;
    code 0/1/2 = 5th/3rd/1st order)."""
    Uf = fill_ghosts(g, U)
    L = np.zeros_like(Uf)
    masks = [np.zeros(s, dtype=np.uint8) for s in g.mask_shapes()] if with_mask else []
    mptr = (ctypes.POINTER(ctypes.c_uint8) * 3)()
    for d, m in enumerate(masks):
        mptr[d] = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    lib().or_rhs(ctypes.byref(g._c), _dp(Uf), _dp(L), mptr if with_mask else None)
    return L, masks


def cfl_dt(g: Grid, U: np.ndarray, cfl: float = 0.5) -> float:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return float(lib().or_cfl_dt(ctypes.byref(g._c), _dp(U), ctypes.c_double(cfl)))


def step(g: Grid, U: np.ndarray, dt: float = 0.0, cfl: float = 0.5, with_mask: bool = False):
    """One SSP-RK3 step; ``dt <= 0`` takes the CFL step.  Returns ``(U, dt, masks)``;
    masks is ``[stage][direction]`` when requested."""
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    masks = None
    arr = None
    if with_mask:
        masks = [[np.zeros(s, dtype=np.uint8) for s in g.mask_shapes()] for _ in range(3)]
        arr = ((ctypes.POINTER(ctypes.c_uint8) * 3) * 3)()
        for s in range(3):
            for d, m in enumerate(masks[s]):
                arr[s][d] = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    dtu = lib().or_step(ctypes.byref(g._c), _dp(U), ctypes.c_double(dt), ctypes.c_double(cfl), arr)
    return U, float(dtu), masks


def run(g: Grid, U: np.ndarray, t_end: float, cfl: float = 0.5, max_steps: int = 10**9):
    """Advance to ``t_end`` with CFL steps (the last one clipped).  Returns ``(U, t, steps)``."""
    t = 0.0
    k = 0
    while t < t_end and k < max_steps:
        dt = cfl_dt(g, U, cfl)
        if t + dt > t_end:
            dt = t_end - t
        U, _, _ = step(g, U, dt)
        t += dt
        k += 1
    return U, t, k


def count_nonphysical(g: Grid, U: np.ndarray) -> int:
    U = np.ascontiguousarray(U, dtype=np.float64)
    return int(lib().or_count_nonphysical(ctypes.byref(g._c), _dp(U)))


def prim_to_cons(ndim: int, Q: np.ndarray) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    U = np.empty_like(Q)
    ncell = Q[0].size
    lib().or_prim_to_cons_array(ctypes.c_int(ndim), ctypes.c_int64(ncell), _dp(Q), _dp(U))
    return U


def cons_to_prim(ndim: int, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    Q = np.empty_like(U)
    ncell = U[0].size
    lib().or_cons_to_prim_array(ctypes.c_int(ndim), ctypes.c_int64(ncell), _dp(U), _dp(Q))
    return Q


def weno_is(v, eps: float = None, order: int = 5, weights: str = "modified"):
    """Left face value at x_{i+1/2} from (q_{i-2}..q_{i+2}); returns (value, dbg) with
    dbg = (beta1..beta4, beta12, tau5, alpha1..alpha4), or for WENO-JS at order 5
    (beta0, beta1, beta2, 0, 0, tau5, alpha0, alpha1, alpha2, 0)."""
    if eps is None:
        eps = default_eps(weights)
    v = np.ascontiguousarray(v, dtype=np.float64)
    dbg = np.zeros(10)
    val = lib().or_weno_is(_dp(v), ctypes.c_double(eps), ctypes.c_int(order),
                           ctypes.c_int(WEIGHTS[weights]), _dp(dbg))
    return float(val), dbg


def char_matrices(nq: int, rho_bar: float, c_bar: float):
    Lm = np.zeros((nq, nq))
    Rm = np.zeros((nq, nq))
    lib().or_char_matrices(ctypes.c_int(nq), ctypes.c_double(rho_bar), ctypes.c_double(c_bar), _dp(Lm), _dp(Rm))
    return Lm, Rm


def hllc(ql, qr):
    """HLLC flux of Sec. 3.2.1 in the sweep frame; returns (Fhat, u_hllc)."""
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    nq = ql.size
    F = np.zeros(nq)
    us = ctypes.c_double(0.0)
    lib().or_hllc(ctypes.c_int(nq), _dp(ql), _dp(qr), _dp(F), ctypes.byref(us))
    return F, us.value


def hllc_waves(ql, qr):
    """or_hllc with the wave-speed estimates; returns (Fhat, u_hllc, waves) with
    waves = (u_bar, c2_bar, S_l, S_r, S*) of Eqs. (wave-speeds), (wave-speed)."""
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    nq = ql.size
    F = np.zeros(nq)
    us = ctypes.c_double(0.0)
    w = np.zeros(5)
    lib().or_hllc_waves(ctypes.c_int(nq), _dp(ql), _dp(qr), _dp(F), ctypes.byref(us), _dp(w))
    return F, us.value, w


def face(qc, cc, eps: float = None, mood: bool = True, weights: str = "modified"):
    """One face from the sweep-frame primitives of 6 cells; returns (Fhat, u_hllc, levels, qlr)."""
    if eps is None:
        eps = default_eps(weights)
    qc = np.ascontiguousarray(qc, dtype=np.float64)
    cc = np.ascontiguousarray(cc, dtype=np.float64)
    nq = qc.shape[1]
    F = np.zeros(nq)
    us = ctypes.c_double(0.0)
    lev = (ctypes.c_int * 2)()
    qlr = np.zeros((2, nq))
    lib().or_face(ctypes.c_int(nq), _dp(qc), _dp(cc), ctypes.c_double(eps), ctypes.c_int(int(mood)),
                  ctypes.c_int(WEIGHTS[weights]), _dp(F), ctypes.byref(us), lev, _dp(qlr))
    return F, us.value, (lev[0], lev[1]), qlr


def sound_speed(rho, p, Gam, Pi) -> float:
    return float(lib().or_sound_speed(rho, p, Gam, Pi))


def tubes_step(offsets: np.ndarray, U: np.ndarray, cfl: float = 0.5, eps: float = None, mood: bool = True,
               weights: str = "modified"):
    """One CFL step of every independent 1D tube (padded segments given by ``offsets``).
    Returns ``(U, dts)``."""
    if eps is None:
        eps = default_eps(weights)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    U = np.ascontiguousarray(U, dtype=np.float64).copy()
    nt = offsets.size - 1
    dts = np.zeros(nt)
    lib().or_tubes_step(ctypes.c_int64(nt), offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        ctypes.c_int64(U.shape[1]), _dp(U), ctypes.c_double(cfl), ctypes.c_double(eps),
                        ctypes.c_int(int(mood)), ctypes.c_int(WEIGHTS[weights]), _dp(dts))
    return U, dts
