"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point include/ws.h declares; the ctypes structs match
the C layout (checked by compiling the header with gcc)."""
import ctypes
import os
import subprocess
import tempfile

import pytest

import paper_1707_00592_gb300 as ws
from paper_1707_00592_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return ws.load()


def test_exports_every_declared_symbol(lib):
    names = ws.header_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ws.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ws_grid), offsetof(ws_grid, ntubes),
         offsetof(ws_grid, tube_offsets), sizeof(ws_opts), offsetof(ws_opts, eps), offsetof(ws_opts, check));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(v) for v in subprocess.check_output([exe]).split()]
    assert vals == [ctypes.sizeof(ws.ws_grid), ws.ws_grid.ntubes.offset, ws.ws_grid.tube_offsets.offset,
                    ctypes.sizeof(ws.ws_opts), ws.ws_opts.eps.offset, ws.ws_opts.check.offset]


def test_init_without_gpu_fails_cleanly(lib):
    """With no CUDA device (this CPU container) ws_init either reports an error
    code or succeeds on a real device; it never crashes the process."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    g, _ = ws.make_grid(1, (10,), (0.1,))
    with pytest.raises(ws.WsError):
        ws.ws_init(g, ws.make_opts(), 0)


def _grid(ndim, n, dx, bc=None, tubes=None):
    return ws.make_grid(ndim, n, dx, bc, tubes)


@pytest.mark.parametrize("desc,args,opts", [
    ("no dimensions", (0, (10,), (0.1,)), {}),
    ("four dimensions", (3, (4, 4, 4), (0.1,) * 3), {"ndim": 4}),
    ("empty grid", (1, (0,), (0.1,)), {}),
    ("empty 2D extent", (2, (16, 0), (0.1, 0.1)), {}),
    ("zero cell size", (2, (8, 8), (0.1, 0.0)), {}),
    ("negative cell size", (1, (8,), (-0.1,)), {}),
    ("periodic on one side only", (1, (8,), (0.1,), (("periodic", "transmissive"),)), {}),
    ("two cells between reflective walls", (1, (2,), (0.1,), (("reflective", "reflective"),)), {}),
    ("tubes in 2D", (2, (8, 8), (0.1, 0.1), None, [0, 20, 40]), {}),
    ("bad precision", (1, (8,), (0.1,)), {"precision": 7}),
    ("bad mood flag", (1, (8,), (0.1,)), {"mood": 2}),
    ("learned gate in FP64", (2, (8, 8), (0.1, 0.1)), {"learned": True}),
])
def test_init_rejects_invalid_input(lib, desc, args, opts):
    """Empty or inconsistent grids and options are refused with WS_EINVAL
    and a message, before any device work (so also without a GPU)."""
    g, keep = _grid(*args)
    o = ws.make_opts()
    for k, v in opts.items():
        if k == "ndim":
            g.ndim = v  # a value the Python helper cannot express
        else:
            setattr(o, k, int(v))
    with pytest.raises(ws.WsError) as e:
        ws.ws_init(g, o, 0)
    assert e.value.code == ws.WS_EINVAL, (desc, e.value)
    assert str(e.value), desc
