"""Seeded synthetic graph generators (input side only).

This module builds the CSR inputs that both the CUDA library and the oracle
read.  It computes no traversal result: it only draws graphs, coordinates
and source vertices from counter-based random streams (SplitMix64 of
seed + counter), so every graph is a pure function of its arguments.

The families mirror the shapes of the paper's inputs (Table 1 and the
appendix graph table): synthetic grids (REC/SREC), k-nearest-neighbour
graphs (CH5/GL5/COS5), road-like large-diameter graphs and R-MAT stand-ins
for the social/web low-diameter graphs.  The named workloads at the bottom
(`grid_1000`, `knn_10m`, `rmat_24`, `dgrid_4000`, `knn_30m_k3`,
`strip_20m`) are the five benchmark configurations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("m", ctypes.c_uint32),
                ("offsets", ctypes.POINTER(ctypes.c_uint32)),
                ("indices", ctypes.POINTER(ctypes.c_uint32))]


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc + OpenMP (portable C, no arch flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-Wall", "-Wno-unknown-pragmas", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        lib.gg_grid.argtypes = [u32, u32, P(_CSR)]
        lib.gg_dgrid.argtypes = [u32, u32, dbl, u64, u32, P(_CSR)]
        lib.gg_knn.argtypes = [u32, u32, u64, P(_CSR), ctypes.c_void_p]
        lib.gg_rmat.argtypes = [u32, u32, dbl, dbl, dbl, u64, i32, P(_CSR)]
        lib.gg_random.argtypes = [u32, u32, i32, i32, u64, P(_CSR)]
        lib.gg_from_arcs.argtypes = [u32, u32, ctypes.c_void_p, ctypes.c_void_p, i32, i32, P(_CSR)]
        lib.gg_pick_sources.argtypes = [u32, ctypes.c_void_p, u32, u64, ctypes.c_void_p]
        lib.gg_free.argtypes = [P(_CSR)]
        lib.gg_read_adj.argtypes = [ctypes.c_char_p, P(_CSR)]
        lib.gg_write_adj.argtypes = [ctypes.c_char_p, u32, u32, ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_read_gbbs_bin.argtypes = [ctypes.c_char_p, P(_CSR)]
        lib.gg_edge_weights.argtypes = [u32, ctypes.c_void_p, ctypes.c_void_p, u32, u32, u64,
                                        ctypes.c_void_p]
        lib.gg_write_gbbs_bin.argtypes = [ctypes.c_char_p, u32, u32, ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_rand.argtypes = [u64, u64, u64]
        lib.gg_rand.restype = u64
        for f in ("gg_grid", "gg_dgrid", "gg_knn", "gg_rmat", "gg_random", "gg_from_arcs",
                  "gg_pick_sources", "gg_num_threads", "gg_read_adj", "gg_write_adj",
                  "gg_read_gbbs_bin", "gg_write_gbbs_bin", "gg_edge_weights"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A CSR graph: offsets[n+1], indices[m] (uint32), lists sorted."""
    n: int
    m: int
    offsets: np.ndarray
    indices: np.ndarray
    directed: bool
    name: str = ""
    meta: dict = field(default_factory=dict)

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))


def _take(csr: _CSR, directed: bool, name: str, **meta) -> Graph:
    lib = _load()
    n, m = int(csr.n), int(csr.m)
    off = np.ctypeslib.as_array(csr.offsets, shape=(n + 1,)).copy()
    idx = (np.ctypeslib.as_array(csr.indices, shape=(m,)).copy() if m
           else np.zeros(0, dtype=np.uint32))
    lib.gg_free(ctypes.byref(csr))
    return Graph(n, m, off, idx, directed, name, dict(meta))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"graphgen: {what} failed with code {rc}")


def grid(rows: int, cols: int) -> Graph:
    """Undirected 4-neighbour grid, vertex (r, c) -> r*cols + c."""
    c = _CSR()
    _check(_load().gg_grid(rows, cols, ctypes.byref(c)), "grid")
    return _take(c, False, f"grid_{rows}x{cols}", rows=rows, cols=cols)


def strip(length: int) -> Graph:
    """1 x length grid strip (a path), the adversarial chain."""
    g = grid(1, length)
    g.name = f"strip_1x{length}"
    return g


def dgrid(rows: int, cols: int, seed: int, p_both: float = 0.5,
          shortcut_frac: float = 1e-4, shortcuts: int | None = None) -> Graph:
    """Directed grid; shortcuts default to round(shortcut_frac * grid arcs)."""
    lib = _load()
    if shortcuts is None:
        base = _CSR()
        _check(lib.gg_dgrid(rows, cols, p_both, seed, 0, ctypes.byref(base)), "dgrid")
        arcs = int(base.m)
        lib.gg_free(ctypes.byref(base))
        shortcuts = int(round(shortcut_frac * arcs))
    c = _CSR()
    _check(lib.gg_dgrid(rows, cols, p_both, seed, shortcuts, ctypes.byref(c)), "dgrid")
    return _take(c, True, f"dgrid_{rows}x{cols}_s{seed}", rows=rows, cols=cols,
                 shortcuts=shortcuts, seed=seed)


def knn(npts: int, k: int, seed: int, return_points: bool = False):
    """Symmetrised exact kNN graph of uniform points in the unit square."""
    lib = _load()
    c = _CSR()
    xy = np.zeros((npts, 2), dtype=np.float32) if return_points else None
    ptr = xy.ctypes.data if xy is not None else None
    _check(lib.gg_knn(npts, k, seed, ctypes.byref(c), ptr), "knn")
    g = _take(c, False, f"knn_{npts}_k{k}_s{seed}", npts=npts, k=k, seed=seed)
    return (g, xy) if return_points else g


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19,
         permute: bool = True) -> Graph:
    """Symmetrised, deduplicated R-MAT graph with permuted ids."""
    cs = _CSR()
    _check(_load().gg_rmat(scale, edge_factor, a, b, c, seed, int(permute), ctypes.byref(cs)), "rmat")
    return _take(cs, False, f"rmat_{scale}_{edge_factor}_s{seed}", scale=scale, seed=seed)


def random_graph(n: int, draws: int, directed: bool, seed: int, keep_raw: bool = False) -> Graph:
    """Uniform random arcs; keep_raw keeps self-loops and duplicate arcs."""
    c = _CSR()
    _check(_load().gg_random(n, draws, int(directed), int(keep_raw), seed, ctypes.byref(c)), "random")
    return _take(c, directed, f"random_{n}_{draws}_s{seed}")


def from_arcs(n: int, src, dst, symmetrize: bool = False, clean: bool = True,
              directed: bool = True) -> Graph:
    s = np.ascontiguousarray(src, dtype=np.uint32)
    d = np.ascontiguousarray(dst, dtype=np.uint32)
    c = _CSR()
    _check(_load().gg_from_arcs(n, len(s), s.ctypes.data, d.ctypes.data, int(symmetrize),
                                int(clean), ctypes.byref(c)), "from_arcs")
    return _take(c, directed and not symmetrize, "arcs")


def read_adj(path: str, directed: bool = True) -> Graph:
    """Read a graph in the PBBS "AdjacencyGraph" text format (header, n, m,
    n offsets, m targets).  Arcs are taken as given; `directed=False` marks a
    file that stores both directions of every edge."""
    c = _CSR()
    _check(_load().gg_read_adj(os.fsencode(path), ctypes.byref(c)), f"read_adj({path})")
    return _take(c, directed, os.path.basename(path), path=path)


def write_adj(g: Graph, path: str) -> None:
    """Write g in the PBBS "AdjacencyGraph" text format."""
    off = np.ascontiguousarray(g.offsets, dtype=np.uint32)
    idx = np.ascontiguousarray(g.indices, dtype=np.uint32)
    _check(_load().gg_write_adj(os.fsencode(path), g.n, g.m, off.ctypes.data, idx.ctypes.data),
           f"write_adj({path})")


def edge_weights(g: Graph, lo: int, hi: int, seed: int) -> np.ndarray:
    """Seeded uint32 weights in [lo, hi] (lo >= 1), one per arc of g, drawn per
    unordered vertex pair so that both arcs of an undirected edge agree."""
    out = np.empty(max(g.m, 1), dtype=np.uint32)
    off = np.ascontiguousarray(g.offsets, dtype=np.uint32)
    idx = np.ascontiguousarray(g.indices, dtype=np.uint32)
    _check(_load().gg_edge_weights(g.n, off.ctypes.data, idx.ctypes.data, lo, hi, seed,
                                   out.ctypes.data), "edge_weights")
    return out[:g.m]


def read_gbbs_bin(path: str, directed: bool = True) -> Graph:
    """Read a graph in the GBBS binary layout: 64-bit header words n, m and
    the file size, n + 1 64-bit offsets, m 32-bit targets (little-endian).
    Arcs are taken as given; `directed=False` marks a file that stores both
    directions of every edge."""
    c = _CSR()
    _check(_load().gg_read_gbbs_bin(os.fsencode(path), ctypes.byref(c)), f"read_gbbs_bin({path})")
    return _take(c, directed, os.path.basename(path), path=path)


def write_gbbs_bin(g: Graph, path: str) -> None:
    """Write g in the GBBS binary layout (see read_gbbs_bin)."""
    off = np.ascontiguousarray(g.offsets, dtype=np.uint32)
    idx = np.ascontiguousarray(g.indices, dtype=np.uint32)
    _check(_load().gg_write_gbbs_bin(os.fsencode(path), g.n, g.m, off.ctypes.data, idx.ctypes.data),
           f"write_gbbs_bin({path})")


def pick_sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct uniform sources with out-degree > 0."""
    out = np.zeros(k, dtype=np.uint32)
    _check(_load().gg_pick_sources(g.n, g.offsets.ctypes.data, k, seed, out.ctypes.data),
           "pick_sources")
    return out


def rand(seed: int, stream: int, i: int) -> int:
    return int(_load().gg_rand(seed, stream, i))


def num_threads() -> int:
    return int(_load().gg_num_threads())


# ------------------------------------------------------------------ workloads
# The benchmark configurations (sizes and seeds).

def grid_1000() -> Graph:
    """1000 x 1000 undirected 4-neighbour grid, source 0 (REC-like)."""
    return grid(1000, 1000)


def knn_10m(npts: int = 10_000_000) -> Graph:
    """10M uniform points, k = 5, symmetrised (GL5/CH5-like), seed 2."""
    return knn(npts, 5, 2)


def rmat_24(scale: int = 24) -> Graph:
    """R-MAT scale 24, edge factor 16, a/b/c = .57/.19/.19, seed 3."""
    return rmat(scale, 16, 3)


def dgrid_4000(side: int = 4000) -> Graph:
    """4000 x 4000 directed grid, p_both = .5, 0.01 % shortcuts, seed 4."""
    return dgrid(side, side, 4)


def knn_30m_k3(npts: int = 30_000_000) -> Graph:
    """Held-out kNN graph: 30M points, k = 3, seed 5."""
    return knn(npts, 3, 5)


def strip_20m(length: int = 20_000_000) -> Graph:
    """1 x 20M strip (a path)."""
    return strip(length)


def strip_200k(length: int = 200_000) -> Graph:
    """1 x 200k strip (a path): a small chain for per-hop latency profiles."""
    return strip(length)
