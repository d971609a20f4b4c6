"""Pins of the CPU oracle's weighted shortest paths (no GPU).

oracle.sssp is Dijkstra's algorithm (the sequential counterpart of the
paper's parallel SSSP, Sec. 2.2); it is pinned by what the mathematics fixes,
never by itself:
  * unit weights reduce it to BFS hop distances (oracle.bfs, itself pinned);
  * closed forms: a weighted path (prefix sums of the weights) and a grid
    with one weight on horizontal and another on vertical arcs (weighted
    Manhattan distance, from a corner and from an interior source);
  * brute force: the weighted Floyd-Warshall rows on tiny seeded graphs
    with zero weights, self-loops and duplicate arcs;
  * a hand-derived fixture where the fewest-hop route is not the shortest;
  * at medium size, the arc inequality dist[w] <= dist[u] + w(u, w) and a
    tight predecessor for every reached vertex.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

INF64 = np.uint64(oracle.INF64)


def _grid_weights(rows, cols, g, wh, wv):
    """Weight wh on horizontal arcs (ids differ by 1), wv on vertical ones."""
    u = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    w = g.indices.astype(np.int64)
    return np.where(np.abs(u - w) == 1, wh, wv).astype(np.uint32)


@pytest.mark.parametrize("make", [lambda: gg.knn(3000, 5, 1), lambda: gg.rmat(10, 8, 2),
                                  lambda: gg.dgrid(30, 40, 3, shortcuts=5)])
def test_unit_weights_are_bfs(make):
    g = make()
    ones = np.ones(g.m, dtype=np.uint32)
    for s in (0, g.n // 3, g.n - 1):
        d = oracle.sssp(g, ones, s)
        b = oracle.bfs(g, s).astype(np.uint64)
        b[b == np.uint64(oracle.INF)] = INF64
        assert np.array_equal(d, b), s


def test_weighted_path_prefix_sums():
    g = gg.strip(200)
    rng = np.random.default_rng(5)
    step = rng.integers(1, 1000, size=199).astype(np.uint64)   # weight of edge (i, i+1)
    u = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    w = g.indices.astype(np.int64)
    wts = step[np.minimum(u, w)].astype(np.uint32)
    d = oracle.sssp(g, wts, 0)
    assert np.array_equal(d, np.concatenate([[0], np.cumsum(step)]).astype(np.uint64))
    d = oracle.sssp(g, wts, 100)
    pre = np.concatenate([[0], np.cumsum(step)]).astype(np.int64)
    assert np.array_equal(d, np.abs(pre - pre[100]).astype(np.uint64))


@pytest.mark.parametrize("wh,wv", [(1, 1), (3, 7), (1000, 1)])
def test_weighted_grid_manhattan(wh, wv):
    rows, cols = 37, 53
    g = gg.grid(rows, cols)
    wts = _grid_weights(rows, cols, g, wh, wv)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    for r0, c0 in ((0, 0), (20, 11)):
        want = (np.abs(r - r0) * wv + np.abs(c - c0) * wh).astype(np.uint64).reshape(-1)
        assert np.array_equal(oracle.sssp(g, wts, r0 * cols + c0), want), (r0, c0)


def test_tiny_graphs_match_weighted_floyd_warshall():
    rng = np.random.default_rng(11)
    for t in range(40):
        n = int(rng.integers(2, 40))
        draws = int(rng.integers(0, 4 * n))
        g = gg.random_graph(n, draws, directed=bool(t % 2), seed=100 + t, keep_raw=True)
        wts = rng.integers(0, 51, size=g.m).astype(np.uint32)    # zero weights included
        D = oracle.floyd_warshall_w(g, wts)
        for s in range(n):
            assert np.array_equal(oracle.sssp(g, wts, s), D[s]), (t, s)


def test_fewest_hops_is_not_shortest():
    # 0 -> 1 (10); 0 -> 2 (1); 2 -> 3 (1); 3 -> 1 (1); 1 -> 4 (1); 5 isolated
    src = np.array([0, 0, 2, 3, 1], dtype=np.uint32)
    dst = np.array([1, 2, 3, 1, 4], dtype=np.uint32)
    g = gg.from_arcs(6, src, dst, clean=False, directed=True)
    order = np.lexsort((dst, src))
    wsorted = np.array([10, 1, 1, 1, 1], dtype=np.uint32)[order]
    d = oracle.sssp(g, wsorted, 0)
    assert d.tolist() == [0, 3, 1, 2, 4, oracle.INF64]


def test_invariants_at_medium_size():
    g = gg.knn(50_000, 5, 4)
    wts = gg.edge_weights(g, 1, 1000, 9)
    d = oracle.sssp(g, wts, 0)
    assert d[0] == 0
    u = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    w = g.indices.astype(np.int64)
    du, dw = d[u], d[w]
    fin = du != INF64
    assert np.all(dw[fin] <= du[fin] + wts[fin])
    tight = np.zeros(g.n, dtype=bool)
    np.logical_or.at(tight, w[fin], dw[fin] == du[fin] + wts[fin])
    reached = d != INF64
    reached[0] = False
    assert np.all(tight[reached])


def test_edge_weights_are_symmetric_and_seeded():
    g = gg.knn(2000, 4, 3)
    a = gg.edge_weights(g, 5, 9, 1)
    assert a.min() >= 5 and a.max() <= 9
    assert np.array_equal(a, gg.edge_weights(g, 5, 9, 1))
    assert not np.array_equal(a, gg.edge_weights(g, 5, 9, 2))
    u = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    key = {(int(x), int(y)): int(c) for x, y, c in zip(u, g.indices, a)}
    assert all(key[(y, x)] == c for (x, y), c in key.items())
