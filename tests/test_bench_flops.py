"""The bench's flop bookkeeping: the per-face count of the method (setup,
projection, WENO-IS on every variable and side, back-projection, MOOD test,
HLLC; counted by the op-counting build of the oracle, tests/test_flop_count.py)
and the count the fused kernel executes when flat stencils take the linear
weights (13 flops a side instead of WENO-IS's 99)."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_method_counts_per_face():
    assert [bench.face_flops(d) for d in (1, 2, 3)] == [1251, 1469, 1687]
    # one RK stage of the 1024^2 grid: 2 x 1024 x 1025 faces, 1024^2 cells
    assert bench.stage_flops(2, (1024, 1024)) == 2 * 1024 * 1025 * 1469 + 1024 * 1024 * (16 + 46)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_executed_counts(ndim):
    nq = ndim + 4
    full = bench.face_flops(ndim)
    assert bench.executed_face_flops(ndim, 0.0) == full
    # every variable flat: WENO-IS (99 a side) replaced by the linear weights (13)
    assert bench.executed_face_flops(ndim, 1.0) == full - 2 * nq * 86
    a, b = bench.executed_face_flops(ndim, 0.3), bench.executed_face_flops(ndim, 0.7)
    assert full > a > b > bench.executed_face_flops(ndim, 1.0)


def test_cell_update_bytes():
    # three stages read U^n and U^(s) and write U^(s+1): (2 + 3 + 3) nv doubles
    assert [bench.cell_update_bytes(d) for d in (1, 2, 3)] == [320, 384, 448]


def test_reference_arm_line():
    """`bench.py --impl reference` runs the FP64 oracle on the host cores and
    prints one JSON line with the contract's keys, on the same workload
    configuration as the GPU arm."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "cell-updates/s per RK3 step" and d["unit"] == "cell-updates/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["config"]["workload"] == "shock_bubble_2d_1024x1024"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
