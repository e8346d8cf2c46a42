"""Flop counts of the method, from an op-counting build of the oracle.

TEST INFRASTRUCTURE ONLY: ``flop_count.cpp`` compiles ``weno_is_oracle.c`` a
second time with a counting scalar type (one flop per add, subtract,
multiply, divide, square root, min, max or comparison; none for operations
with a trivial operand -- an exact zero, or +-1 in a product -- which on
generic data are the structural zeros and ones of the oracle's dense
characteristic products and HLLC selection vectors).  The counts are those of
the oracle's own code; the benchmark's flop table is checked against them.

Generic data: every state value non-zero and not +-1, both sides a
stiffened gas (P_inf > 0, so Pi != 0), no MOOD retry, S* != 0 and S_k != S*.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "flop_count.cpp")
ORACLE_SRC = os.path.join(HERE, "weno_is_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libweno_is_oracle_count.so")
KINDS = ("add", "mul", "div", "sqrt", "minmax", "cmp")
WEIGHTS = {"modified": 0, "basic": 1, "js": 2}

_lib = None


def build(force: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(SRC), os.path.getmtime(ORACLE_SRC))
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-I", HERE, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _counts(c) -> dict:
    return dict(zip(KINDS, (int(v) for v in c)))


def face(qc, cc, eps: float = 1e-40, mood: bool = True, weights: str = "modified"):
    """Counts of one oracle face (sweep-frame primitives qc[6][nq], sound speeds
    cc[6]) and the MOOD levels it used."""
    qc = np.ascontiguousarray(qc, dtype=np.float64)
    cc = np.ascontiguousarray(cc, dtype=np.float64)
    c = (ctypes.c_longlong * 6)()
    lev = (ctypes.c_int * 2)()
    lib().fc_face(ctypes.c_int(qc.shape[1]), _dp(qc), _dp(cc), ctypes.c_double(eps), ctypes.c_int(int(mood)),
                  ctypes.c_int(WEIGHTS[weights]), c, lev)
    return _counts(c), (lev[0], lev[1])


def weno(v, eps: float = 1e-40, order: int = 5, weights: str = "modified") -> dict:
    """Counts of one reconstruction (one characteristic variable, one side)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    c = (ctypes.c_longlong * 6)()
    lib().fc_weno(_dp(v), ctypes.c_double(eps), ctypes.c_int(order), ctypes.c_int(WEIGHTS[weights]), c)
    return _counts(c)


def hllc(ql, qr) -> dict:
    """Counts of one HLLC flux between sweep-frame states."""
    ql = np.ascontiguousarray(ql, dtype=np.float64)
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    c = (ctypes.c_longlong * 6)()
    lib().fc_hllc(ctypes.c_int(ql.size), _dp(ql), _dp(qr), c)
    return _counts(c)


def cell_prim(ndim: int, U) -> dict:
    U = np.ascontiguousarray(U, dtype=np.float64)
    c = (ctypes.c_longlong * 6)()
    lib().fc_cell_prim(ctypes.c_int(ndim), _dp(U), c)
    return _counts(c)


def rhs_and_step(ndim: int, n, dx, bc, U, eps: float = 1e-40, mood: bool = True, weights: str = "modified"):
    """Counts of one oracle flux divergence and of one oracle SSP-RK3 step
    (CFL step included) of the padded state U."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    nn = (ctypes.c_int * 3)(*[int(n[d]) if d < ndim else 1 for d in range(3)])
    dd = (ctypes.c_double * 3)(*[float(dx[d]) if d < ndim else 1.0 for d in range(3)])
    bb = (ctypes.c_int * 6)(*bc)
    c1 = (ctypes.c_longlong * 6)()
    c2 = (ctypes.c_longlong * 6)()
    lib().fc_rhs_step(ctypes.c_int(ndim), nn, dd, bb, ctypes.c_double(eps), ctypes.c_int(int(mood)),
                      ctypes.c_int(WEIGHTS[weights]), _dp(U), c1, c2)
    return _counts(c1), _counts(c2)


def total(c: dict) -> int:
    return sum(c.values())
