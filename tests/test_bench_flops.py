"""The bench's flop bookkeeping: the per-face count of the method (setup,
projection, WENO-IS on every variable and side, back-projection, MOOD test,
HLLC) and the count the fused kernel executes when flat stencils take the
linear weights (13 flops a side instead of WENO-IS's 100)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_method_counts_per_face():
    assert bench.face_flops(1) == 12 + 48 + 200 * 5 + 16 + 6 + 114 + 55
    assert bench.face_flops(2) == 1470
    assert bench.face_flops(3) == 1689


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_executed_counts(ndim):
    nq = ndim + 4
    full = bench.face_flops(ndim)
    assert bench.executed_face_flops(ndim, 0.0) == full
    # every variable flat: WENO-IS (100 a side) replaced by the linear weights (13)
    assert bench.executed_face_flops(ndim, 1.0) == full - 2 * nq * 87
    a, b = bench.executed_face_flops(ndim, 0.3), bench.executed_face_flops(ndim, 0.7)
    assert full > a > b > bench.executed_face_flops(ndim, 1.0)


def test_cell_update_bytes():
    # three stages read U^n and U^(s) and write U^(s+1): (2 + 3 + 3) nv doubles
    assert [bench.cell_update_bytes(d) for d in (1, 2, 3)] == [320, 384, 448]
