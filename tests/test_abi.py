"""The C ABI library without a GPU: it builds for sm_103a, loads, exports
every function include/pasgal.h declares, and the Python mirrors of the ABI
structs have the C layout.  No compute call is made (there is no device)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pasgal.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:pg_status|void|const char \*)\s*(pg_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_17101_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path), path


def test_every_declared_symbol_is_exported(lib):
    L, path = lib
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    nm = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pg_\w+)$", nm, re.M))
    assert set(names) <= exported
    import paper_2404_17101_gb300 as pg
    assert sorted(pg.EXPORTS) == names


def test_struct_layouts_match_c():
    import paper_2404_17101_gb300 as pg
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "pasgal.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(pg_config), sizeof(pg_round_trace), sizeof(pg_stats),
         offsetof(pg_config, script), offsetof(pg_round_trace, features), offsetof(pg_stats, kernel_ms));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(pg.Config), ctypes.sizeof(pg.RoundTrace), ctypes.sizeof(pg.Stats),
            pg.Config.script.offset, pg.RoundTrace.features.offset, pg.Stats.kernel_ms.offset]
    assert got == want


def test_no_cpu_fallback_without_library(monkeypatch):
    import paper_2404_17101_gb300 as pg
    monkeypatch.setattr(pg, "_lib", None)
    with pytest.raises(RuntimeError):
        pg.load("/nonexistent/libpasgal_gb.so")


def test_bfs_noalloc_wrapper_rejects_bad_buffers_before_any_launch():
    """The C ABI cannot see buffer sizes, so the binding checks dtype,
    contiguity, sizes and device before calling pg_bfs_noalloc; each failure
    is a ValueError raised before the library is even loaded (CPU tensors)."""
    import torch
    import paper_2404_17101_gb300 as pg
    off = torch.tensor([0, 1, 2], dtype=torch.int32)
    idx = torch.tensor([1, 0], dtype=torch.int32)
    with pytest.raises(ValueError, match="fewer than n"):
        pg.bfs_noalloc(off, idx, 0, torch.empty(1, dtype=torch.int32))
    with pytest.raises(ValueError, match="int32 or uint32"):
        pg.bfs_noalloc(off, idx, 0, torch.empty(2, dtype=torch.int64))
    with pytest.raises(ValueError, match="contiguous"):
        pg.bfs_noalloc(off, idx, 0, torch.empty(4, dtype=torch.int32)[::2])
    with pytest.raises(ValueError, match="CUDA device"):
        pg.bfs_noalloc(off, idx, 0, torch.empty(2, dtype=torch.int32))
