"""Generator checks (no GPU): structure, determinism and exact kNN."""
import os
import numpy as np
import pytest

import graphgen as gg


def _canonical(g):
    off = g.offsets.astype(np.int64)
    for v in range(g.n):
        row = g.indices[off[v]:off[v + 1]]
        assert np.all(np.diff(row.astype(np.int64)) > 0), "sorted, no duplicates"
        assert not np.any(row == v), "no self-loops"


def _symmetric(g):
    u = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    fwd = set(zip(u.tolist(), g.indices.astype(np.int64).tolist()))
    assert all((b, a) in fwd for a, b in fwd)


def test_grid_structure():
    g = gg.grid(4, 6)
    assert g.n == 24 and g.m == 2 * (4 * 5 + 3 * 6)
    _canonical(g)
    _symmetric(g)
    deg = g.degrees().reshape(4, 6)
    assert deg[0, 0] == 2 and deg[0, 3] == 3 and deg[2, 3] == 4
    s = gg.strip(10)
    assert s.m == 18 and s.indices[:3].tolist() == [1, 0, 2]


def test_dgrid_counts():
    rows, cols = 30, 20
    E = rows * (cols - 1) + (rows - 1) * cols
    both = gg.dgrid(rows, cols, 1, p_both=1.0, shortcuts=0)
    one = gg.dgrid(rows, cols, 1, p_both=0.0, shortcuts=0)
    assert both.m == 2 * E and one.m == E
    h = gg.dgrid(rows, cols, 1)
    assert h.meta["shortcuts"] == round(1e-4 * gg.dgrid(rows, cols, 1, shortcuts=0).m)
    g = gg.dgrid(rows, cols, 1, shortcuts=25)
    base = gg.dgrid(rows, cols, 1, shortcuts=0)
    assert g.m == base.m + 25
    _canonical(g)
    # roughly half the edges kept both ways
    mid = gg.dgrid(200, 200, 3, shortcuts=0)
    E2 = 2 * 200 * 199
    assert abs(mid.m / E2 - 1.5) < 0.01


def test_knn_exact_small():
    npts, k = 400, 5
    g, xy = gg.knn(npts, k, 7, return_points=True)
    _canonical(g)
    _symmetric(g)
    P = xy.astype(np.float64)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(d2, np.inf)
    adj = [set(g.indices[g.offsets[v]:g.offsets[v + 1]].tolist()) for v in range(npts)]
    for i in range(npts):
        order = np.lexsort((np.arange(npts), d2[i]))[:k]
        for j in order:
            assert j in adj[i] and i in adj[j]
    # every arc is some point's kNN arc
    for i in range(npts):
        for j in adj[i]:
            ki = set(np.lexsort((np.arange(npts), d2[i]))[:k].tolist())
            kj = set(np.lexsort((np.arange(npts), d2[j]))[:k].tolist())
            assert j in ki or i in kj


def test_rmat_structure_and_determinism():
    a = gg.rmat(12, 8, 5)
    b = gg.rmat(12, 8, 5)
    c = gg.rmat(12, 8, 6)
    assert np.array_equal(a.indices, b.indices) and np.array_equal(a.offsets, b.offsets)
    assert not (a.m == c.m and np.array_equal(a.indices, c.indices))
    _canonical(a)
    _symmetric(a)
    deg = a.degrees()
    assert deg.max() > 20 * deg[deg > 0].mean()  # skewed


def test_pick_sources():
    g = gg.dgrid(50, 50, 2)
    s = gg.pick_sources(g, 64, 9)
    assert len(set(s.tolist())) == 64
    assert np.all(g.degrees()[s] > 0)
    assert np.array_equal(s, gg.pick_sources(g, 64, 9))


def test_rand_is_counter_based():
    assert gg.rand(1, 2, 3) == gg.rand(1, 2, 3)
    assert len({gg.rand(1, 2, i) for i in range(1000)}) == 1000


def test_adjacency_graph_file_round_trip(tmp_path):
    """PBBS AdjacencyGraph text files: write then read gives the same CSR,
    a hand-written file parses to the expected arcs, and malformed files
    (wrong header, decreasing offsets, a target >= n, truncation) are
    rejected."""
    g = gg.dgrid(20, 30, 5, shortcuts=7)
    p = str(tmp_path / "g.adj")
    gg.write_adj(g, p)
    h = gg.read_adj(p)
    assert (h.n, h.m) == (g.n, g.m)
    assert np.array_equal(h.offsets, g.offsets) and np.array_equal(h.indices, g.indices)
    q = tmp_path / "tiny.adj"
    q.write_text("AdjacencyGraph\n3\n4\n0\n2\n3\n1\n2\n2\n0\n")
    t = gg.read_adj(str(q))
    assert t.offsets.tolist() == [0, 2, 3, 4] and t.indices.tolist() == [1, 2, 2, 0]
    for bad in ("WeightedAdjacencyGraph\n1\n0\n0\n", "AdjacencyGraph\n3\n2\n0\n2\n1\n0\n1\n",
                "AdjacencyGraph\n2\n1\n0\n1\n5\n", "AdjacencyGraph\n3\n4\n0\n2\n"):
        b = tmp_path / "bad.adj"
        b.write_text(bad)
        with pytest.raises(RuntimeError):
            gg.read_adj(str(b))


def test_gbbs_binary_file_round_trip(tmp_path):
    """GBBS binary graph files (64-bit n, m, byte size; n + 1 64-bit offsets;
    m 32-bit targets): write then read gives the same CSR, a file assembled
    byte by byte here parses to the expected arcs, and malformed files (wrong
    size word, truncation, decreasing offsets, a target >= n, offsets not
    ending at m) are rejected."""
    g = gg.dgrid(20, 30, 5, shortcuts=7)
    p = str(tmp_path / "g.bin")
    gg.write_gbbs_bin(g, p)
    h = gg.read_gbbs_bin(p)
    assert (h.n, h.m) == (g.n, g.m)
    assert np.array_equal(h.offsets, g.offsets) and np.array_equal(h.indices, g.indices)
    assert os.path.getsize(p) == 24 + 8 * (g.n + 1) + 4 * g.m

    def blob(n, m, size, offs, tgts):
        return (np.array([n, m, size], dtype="<u8").tobytes() + np.array(offs, dtype="<u8").tobytes()
                + np.array(tgts, dtype="<u4").tobytes())
    good = blob(3, 4, 24 + 32 + 16, [0, 2, 3, 4], [1, 2, 2, 0])
    q = tmp_path / "tiny.bin"
    q.write_bytes(good)
    t = gg.read_gbbs_bin(str(q))
    assert t.offsets.tolist() == [0, 2, 3, 4] and t.indices.tolist() == [1, 2, 2, 0]
    bads = [blob(3, 4, 99, [0, 2, 3, 4], [1, 2, 2, 0]),     # size word wrong
            good[:-4],                                        # truncated
            blob(3, 4, 72, [0, 3, 2, 4], [1, 2, 2, 0]),      # decreasing offsets
            blob(3, 4, 72, [0, 2, 3, 4], [1, 7, 2, 0]),      # target >= n
            blob(3, 4, 72, [0, 2, 3, 3], [1, 2, 2, 0])]      # offsets[n] != m
    for i, b in enumerate(bads):
        f = tmp_path / f"bad{i}.bin"
        f.write_bytes(b)
        with pytest.raises(RuntimeError):
            gg.read_gbbs_bin(str(f))
