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
