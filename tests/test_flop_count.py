"""The benchmark's flop table against the op-counting build of the oracle.

The measurement's algorithmic flops (the roofline numerator) are the
method's operations as the oracle performs them: oracle/flop_count.cpp
compiles the oracle again with a counting scalar type, one flop per add,
subtract, multiply, divide, square root, min, max or comparison, none for an
operation with a trivial operand (an exact zero, or +-1 in a product), which
removes the structural zeros and ones of the oracle's dense characteristic
products.  On generic data -- every value distinct from its neighbours and
non-zero, both sides stiffened gases, no MOOD retry, S* > 0 -- the count of
a face is the same for every face, and the table in bench.py must equal it,
term by term."""
import os
import sys

import numpy as np
import pytest

import oracle
from oracle import flops
from paper_1707_00592_gb300 import workloads as wl

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

G1, P1 = wl.material(4.4, 6e8)
G2, P2 = wl.material(2.35, 3e8)


def generic_cells(rng, shape, ndim):
    """Primitive fields (rho, u_1..u_ndim, p, Gamma, Pi): mixtures of two
    stiffened gases in random proportions, velocities of one sign (S* > 0 on
    every face), all values distinct."""
    a = rng.uniform(0.05, 0.95, size=shape)
    Q = np.empty((ndim + 4,) + shape)
    Q[0] = rng.uniform(900, 1100, size=shape)
    for d in range(ndim):
        Q[1 + d] = rng.uniform(40, 60, size=shape)
    Q[1 + ndim] = rng.uniform(1e8, 1.5e8, size=shape)
    Q[2 + ndim] = a * G1 + (1 - a) * G2
    Q[3 + ndim] = a * P1 + (1 - a) * P2
    return Q


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_face_count_equals_bench_table(ndim):
    rng = np.random.default_rng(ndim)
    nq = ndim + 4
    seen = set()
    for _ in range(40):
        qc = generic_cells(rng, (6,), ndim).T.copy()  # [cell][nq], sweep frame = axis order
        cc = np.array([oracle.sound_speed(q[0], q[nq - 3], q[nq - 2], q[nq - 1]) for q in qc])
        c, lev = flops.face(qc, cc)
        assert lev == (5, 5)
        seen.add(flops.total(c))
    assert seen == {bench.face_flops(ndim)}


def test_face_count_terms():
    """The terms of bench.face_flops, each counted on its own oracle routine."""
    rng = np.random.default_rng(7)
    assert flops.total(flops.weno(rng.normal(size=5))) == bench.WENO_FLOPS
    for nq in (5, 6, 7):
        ndim = nq - 4
        q = generic_cells(rng, (2,), ndim).T.copy()
        assert flops.total(flops.hllc(q[0], q[1])) == bench.hllc_flops(nq)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_cell_counts_equal_bench_table(ndim):
    """Per cell and stage: the primitive recovery with the sound speed, and the
    flux divergence with the Gamma/Pi source -- from whole oracle flux
    divergences on two periodic grids, less their faces."""
    rng = np.random.default_rng(10 + ndim)
    U = oracle.prim_to_cons(ndim, generic_cells(rng, (1, 1, 1), ndim))
    assert flops.total(flops.cell_prim(ndim, U[:, 0, 0, 0].copy())) == bench.prim_flops(ndim)
    sizes = {1: [(16,), (23,)], 2: [(8, 6), (10, 7)], 3: [(5, 4, 6), (7, 5, 4)]}[ndim]
    for n in sizes:
        shape = tuple(reversed([n[d] + 6 if d < ndim else 1 for d in range(3)]))
        U = oracle.prim_to_cons(ndim, generic_cells(rng, shape, ndim))
        cells = int(np.prod(n))
        faces = sum((n[d] + 1) * cells // n[d] for d in range(ndim))
        dx = [1.0 / n[d] for d in range(ndim)]
        r, _ = flops.rhs_and_step(ndim, n, dx, [1] * 6, U)
        # the oracle recomputes the primitives of each of a face's six cells
        per_faces = faces * (6 * bench.prim_flops(ndim) + bench.face_flops(ndim))
        assert flops.total(r) - per_faces == cells * bench.divergence_flops(ndim)
