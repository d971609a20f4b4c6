"""The C ABI library without a GPU: it builds for sm_103a, loads, exports
every function include/pasgal.h declares, and the Python mirrors of the ABI
structs have the C layout.  No compute call is made (there is no device)."""
import ctypes
import os
import re
import subprocess
import tempfile

import numpy as np
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


class _FakeLib:
    """Stands in for the library: records the calls that got through."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture
def fake_graph(monkeypatch):
    import paper_2404_17101_gb300 as pg
    fake = _FakeLib()
    monkeypatch.setattr(pg, "load", lambda *a, **k: fake)
    monkeypatch.setattr(pg, "_stream_ptr", lambda stream=None: ctypes.c_void_p(0))
    G = pg.Graph(ctypes.c_void_p(1), 4, 6, False)
    yield pg, G, fake
    G._h = None  # never hand the fake handle to the real library


def test_graph_wrappers_check_buffers_before_any_call(fake_graph):
    """The C ABI sees pointers and no sizes: every Graph method that takes a
    caller buffer checks its type, contiguity and size first (ValueError),
    and only a buffer that passes reaches the library."""
    import torch
    pg, G, fake = fake_graph
    bad_u32 = [(torch.empty(3, dtype=torch.int32), "fewer than"),
               (torch.empty(4, dtype=torch.float32), "dtype"),
               (torch.empty(8, dtype=torch.int32)[::2], "contiguous"),
               (np.empty(3, dtype=np.uint32), "fewer than"),
               (np.empty(4, dtype=np.int64), "dtype"),
               ([0, 0, 0, 0], "expected")]
    for out, msg in bad_u32:
        with pytest.raises(ValueError, match=msg):
            G.bfs(0, out=out)
        with pytest.raises(ValueError, match=msg):
            G.scc(out=out)
    ro = np.zeros(4, dtype=np.uint32)
    ro.flags.writeable = False
    with pytest.raises(ValueError, match="writeable"):
        G.bfs(0, out=ro)
    for out, msg in [(torch.empty(3, dtype=torch.int64), "fewer than"),
                     (torch.empty(4, dtype=torch.int32), "dtype"),
                     (np.empty(4, dtype=np.uint32), "dtype")]:
        with pytest.raises(ValueError, match=msg):
            G.sssp(0, out=out)
    with pytest.raises(ValueError, match="CUDA tensor"):
        G.count_reached(torch.zeros(4, dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA tensor"):
        G.bfs_multi([0, 1], out=torch.empty(8, dtype=torch.int32))
    with pytest.raises(ValueError, match="fewer than"):
        G.set_transpose(np.zeros(4, dtype=np.uint32), np.zeros(6, dtype=np.uint32))
    with pytest.raises(ValueError, match="fewer than"):
        G.set_transpose(np.zeros(5, dtype=np.uint32), np.zeros(5, dtype=np.uint32))
    assert fake.calls == []
    # host buffers of the right shape go through (the library stages them)
    G.bfs(0, out=np.empty(4, dtype=np.uint32))
    G.bfs(0, out=torch.empty(4, dtype=torch.int32))
    G.scc(out=np.empty(4, dtype=np.uint32))
    G.sssp(0, out=np.empty(4, dtype=np.uint64))
    G.set_transpose(np.zeros(5, dtype=np.uint32), np.zeros(6, dtype=np.uint32))
    assert fake.calls == ["pg_bfs", "pg_bfs", "pg_scc", "pg_sssp", "pg_graph_set_transpose"]


def test_mlp_wrappers_check_shapes_before_any_call(fake_graph):
    import torch
    pg, _, fake = fake_graph
    P = torch.zeros(pg.PG_MLP_NPARAMS, dtype=torch.float32)
    X = torch.zeros(3, 5, dtype=torch.float32)
    with pytest.raises(ValueError, match="B x 5"):
        pg.mlp_forward(P, torch.zeros(3, 4))
    with pytest.raises(ValueError, match="fewer than"):
        pg.mlp_forward(P[:-1], X)
    with pytest.raises(ValueError, match="CUDA tensor"):
        pg.mlp_forward(P, X)  # CPU tensors: the kernels need device memory
    with pytest.raises(ValueError, match="CUDA tensor"):
        pg.mlp_adam(P, P.clone(), P.clone(), P.clone(), 1)
    with pytest.raises(ValueError, match="params must be"):
        pg.mlp_adam(np.zeros(4), None, None, None, 1)
    assert fake.calls == []
