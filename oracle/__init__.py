"""CPU oracle for the traversal results -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports, links or calls anything here, and shares no
code with it.

Contents:
  * ``bfs``            sequential FIFO-queue BFS (the paper's sequential
                       baseline, Sec. 4 Setup; BFS table "*" column):
                       hop distance from the source, 0xFFFFFFFF if
                       unreachable (Sec. 2.2).
  * ``bfs_multi``      one queue BFS per source (source-major k x n).
  * ``reach``          forward / backward reachability for <= 64 sources as
                       one bit per source (Sec. 2.1, reachability search).
  * ``floyd_warshall`` / ``warshall``  brute-force all-pairs hop distances
                       and transitive closure for tiny graphs; they pin the
                       queue BFS against an independent definition.
  * ``reached_edges``  (n_r, m_r): reached vertices and the sum of their
                       out-degrees, the traversed-edge count used for TEPS.
  * ``scc``            strongly connected components by Tarjan's algorithm
                       (the paper's sequential SCC baseline, Sec. 4 Setup),
                       labelled by the smallest vertex id of each component.
  * ``sssp``           single-source shortest paths with non-negative
                       uint32 arc weights (Sec. 2.2, the SSSP paragraph) by
                       Dijkstra's algorithm; uint64 distances,
                       0xFFFFFFFFFFFFFFFF if unreachable.
  * ``floyd_warshall_w`` brute-force all-pairs weighted distances (n <= 64).
  * ``mlp``            fp64 forward / backward / Adam of the schedule MLP.

Parity status: every function here is pinned by closed forms, brute force
or finite differences in tests/test_oracle.py (see that file's docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
INF = 0xFFFFFFFF
INF64 = 0xFFFFFFFFFFFFFFFF


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain serial C, -O2, no threads)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u32, vp = ctypes.c_uint32, ctypes.c_void_p
        lib.oracle_bfs.argtypes = [u32, vp, vp, u32, vp]
        lib.oracle_bfs_multi.argtypes = [u32, vp, vp, vp, u32, vp]
        lib.oracle_reach.argtypes = [u32, vp, vp, vp, u32, vp]
        lib.oracle_reach_backward.argtypes = [u32, vp, vp, vp, u32, vp]
        lib.oracle_transpose.argtypes = [u32, vp, vp, vp, vp]
        lib.oracle_floyd_warshall.argtypes = [u32, vp, vp, vp]
        lib.oracle_warshall.argtypes = [u32, vp, vp, vp]
        lib.oracle_reached_edges.argtypes = [u32, vp, vp, vp, vp]
        lib.oracle_scc.argtypes = [u32, vp, vp, vp]
        lib.oracle_sssp.argtypes = [u32, vp, vp, vp, u32, vp]
        lib.oracle_floyd_warshall_w.argtypes = [u32, vp, vp, vp, vp]
        lib.oracle_reached_edges.restype = None
        _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def bfs(g, src: int) -> np.ndarray:
    off, idx = _u32(g.offsets), _u32(g.indices)
    dist = np.empty(g.n, dtype=np.uint32)
    rc = _load().oracle_bfs(g.n, off.ctypes.data, idx.ctypes.data, int(src), dist.ctypes.data)
    if rc:
        raise ValueError(f"oracle_bfs rc={rc}")
    return dist


def bfs_multi(g, srcs) -> np.ndarray:
    off, idx, s = _u32(g.offsets), _u32(g.indices), _u32(srcs)
    dist = np.empty((len(s), g.n), dtype=np.uint32)
    rc = _load().oracle_bfs_multi(g.n, off.ctypes.data, idx.ctypes.data, s.ctypes.data, len(s),
                                  dist.ctypes.data)
    if rc:
        raise ValueError(f"oracle_bfs_multi rc={rc}")
    return dist


def reach(g, srcs, backward: bool = False) -> np.ndarray:
    """uint64 mask per vertex; bit j <-> srcs[j]."""
    off, idx, s = _u32(g.offsets), _u32(g.indices), _u32(srcs)
    mask = np.empty(g.n, dtype=np.uint64)
    fn = _load().oracle_reach_backward if backward else _load().oracle_reach
    rc = fn(g.n, off.ctypes.data, idx.ctypes.data, s.ctypes.data, len(s), mask.ctypes.data)
    if rc:
        raise ValueError(f"oracle_reach rc={rc}")
    return mask


def transpose(g):
    off, idx = _u32(g.offsets), _u32(g.indices)
    toff = np.empty(g.n + 1, dtype=np.uint32)
    tidx = np.empty(max(g.m, 1), dtype=np.uint32)
    _load().oracle_transpose(g.n, off.ctypes.data, idx.ctypes.data, toff.ctypes.data,
                             tidx.ctypes.data)
    return toff, tidx[: g.m]


def floyd_warshall(g) -> np.ndarray:
    off, idx = _u32(g.offsets), _u32(g.indices)
    D = np.empty((g.n, g.n), dtype=np.uint32)
    rc = _load().oracle_floyd_warshall(g.n, off.ctypes.data, idx.ctypes.data, D.ctypes.data)
    if rc:
        raise ValueError(f"oracle_floyd_warshall rc={rc}")
    return D


def warshall(g) -> np.ndarray:
    off, idx = _u32(g.offsets), _u32(g.indices)
    R = np.empty((g.n, g.n), dtype=np.uint8)
    rc = _load().oracle_warshall(g.n, off.ctypes.data, idx.ctypes.data, R.ctypes.data)
    if rc:
        raise ValueError(f"oracle_warshall rc={rc}")
    return R.astype(bool)


def reached_edges(g, dist) -> tuple[int, int]:
    off, d = _u32(g.offsets), _u32(dist)
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().oracle_reached_edges(g.n, off.ctypes.data, d.ctypes.data, ctypes.byref(a),
                                 ctypes.byref(b))
    return int(a.value), int(b.value)


def scc(g) -> np.ndarray:
    """Per-vertex SCC label: the smallest vertex id in the vertex's component."""
    off, idx = _u32(g.offsets), _u32(g.indices)
    lab = np.empty(g.n, dtype=np.uint32)
    rc = _load().oracle_scc(g.n, off.ctypes.data, idx.ctypes.data, lab.ctypes.data)
    if rc:
        raise RuntimeError(f"oracle_scc failed ({rc})")
    return lab


def sssp(g, weights, src: int) -> np.ndarray:
    """Shortest-path distances (uint64) from src with arc weights `weights`
    (uint32, one per arc of g)."""
    off, idx, w = _u32(g.offsets), _u32(g.indices), _u32(weights)
    if len(w) != g.m:
        raise ValueError("one weight per arc")
    dist = np.empty(g.n, dtype=np.uint64)
    rc = _load().oracle_sssp(g.n, off.ctypes.data, idx.ctypes.data, w.ctypes.data, int(src),
                             dist.ctypes.data)
    if rc:
        raise ValueError(f"oracle_sssp rc={rc}")
    return dist


def floyd_warshall_w(g, weights) -> np.ndarray:
    off, idx, w = _u32(g.offsets), _u32(g.indices), _u32(weights)
    D = np.empty((g.n, g.n), dtype=np.uint64)
    rc = _load().oracle_floyd_warshall_w(g.n, off.ctypes.data, idx.ctypes.data, w.ctypes.data,
                                         D.ctypes.data)
    if rc:
        raise ValueError(f"oracle_floyd_warshall_w rc={rc}")
    return D
