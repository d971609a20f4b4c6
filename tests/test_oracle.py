"""Pins for the CPU oracle (runs without a GPU).

The oracle is checked against things other than itself:
  * closed forms of hop distance (Sec. 2.2 defines BFS output as the hop
    distance from the source): grids (r + c), paths |i - j|, cycles,
    stars, complete and complete-bipartite graphs, the directed grid with
    every arc in both directions (Manhattan distance), hypercubes (Hamming
    distance), and hand-derived golden fixtures in tests/golden/;
  * brute force: Floyd-Warshall hop distances and the Warshall transitive
    closure on tiny seeded graphs from the same generator code paths as the
    benchmark graphs, including raw inputs with self-loops and duplicate
    arcs;
  * reachability semantics (Sec. 2.1): forward masks are the closure rows
    of the sources, backward masks its columns; on an undirected graph bit j
    is set iff the BFS distance from source j is finite; a directed path
    reaches exactly the later vertices;
  * full-size invariants that any exact hop-distance array satisfies.
A planted error in the queue BFS (a dropped +1, a wrong offset index, a
reversed arc) or in the reachability (wrong direction, wrong bit) fails at
least one of these.
"""
import json
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

INF = oracle.INF
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _undirected(n, edges):
    s = [a for a, b in edges] + [b for a, b in edges]
    d = [b for a, b in edges] + [a for a, b in edges]
    return gg.from_arcs(n, s, d, directed=False)


def test_grid_closed_form():
    for rows, cols in [(1, 1), (1, 7), (5, 1), (7, 9), (31, 17), (100, 100)]:
        g = gg.grid(rows, cols)
        d = oracle.bfs(g, 0).reshape(rows, cols)
        r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
        assert np.array_equal(d, (r + c).astype(np.uint32))


def test_grid_interior_source():
    rows, cols, sr, sc = 23, 41, 11, 7
    g = gg.grid(rows, cols)
    d = oracle.bfs(g, sr * cols + sc).reshape(rows, cols)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    assert np.array_equal(d, (np.abs(r - sr) + np.abs(c - sc)).astype(np.uint32))


def test_path_and_strip():
    n = 1000
    g = gg.strip(n)
    for s in [0, 1, 500, n - 1]:
        assert np.array_equal(oracle.bfs(g, s), np.abs(np.arange(n) - s).astype(np.uint32))


def test_cycle():
    n = 101
    g = _undirected(n, [(i, (i + 1) % n) for i in range(n)])
    for s in [0, 37]:
        i = np.arange(n)
        k = np.abs(i - s)
        assert np.array_equal(oracle.bfs(g, s), np.minimum(k, n - k).astype(np.uint32))


def test_star_complete_bipartite():
    n = 50
    star = _undirected(n, [(0, i) for i in range(1, n)])
    assert oracle.bfs(star, 0).tolist() == [0] + [1] * (n - 1)
    assert oracle.bfs(star, 5).tolist() == [1] + [2] * 4 + [0] + [2] * (n - 6)
    k = 12
    kn = _undirected(k, [(i, j) for i in range(k) for j in range(i + 1, k)])
    assert oracle.bfs(kn, 3).tolist() == [1, 1, 1, 0] + [1] * (k - 4)
    a, b = 5, 7
    kab = _undirected(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    d = oracle.bfs(kab, 0)
    assert d.tolist() == [0] + [2] * (a - 1) + [1] * b


def test_hypercube_hamming():
    dim = 10
    n = 1 << dim
    edges = [(v, v ^ (1 << b)) for v in range(n) for b in range(dim) if v < v ^ (1 << b)]
    g = _undirected(n, edges)
    for s in [0, 5, 1023]:
        want = np.array([bin(v ^ s).count("1") for v in range(n)], dtype=np.uint32)
        assert np.array_equal(oracle.bfs(g, s), want)


def test_directed_grid_both_ways_is_manhattan():
    rows, cols = 40, 30
    g = gg.dgrid(rows, cols, seed=9, p_both=1.0, shortcuts=0)
    s = 17 * cols + 4
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    want = (np.abs(r - 17) + np.abs(c - 4)).astype(np.uint32).reshape(-1)
    assert np.array_equal(oracle.bfs(g, s), want)


def test_directed_path_reach():
    n = 200
    g = gg.from_arcs(n, np.arange(n - 1), np.arange(1, n))
    d = oracle.bfs(g, 50)
    assert np.all(d[:50] == INF)
    assert np.array_equal(d[50:], np.arange(n - 50, dtype=np.uint32))
    srcs = np.array([0, 50, 199, 120], dtype=np.uint32)
    fwd = oracle.reach(g, srcs)
    bwd = oracle.reach(g, srcs, backward=True)
    for v in range(n):
        want_f = sum(1 << j for j, s in enumerate(srcs) if v >= s)
        want_b = sum(1 << j for j, s in enumerate(srcs) if v <= s)
        assert int(fwd[v]) == want_f and int(bwd[v]) == want_b


def test_disconnected_union():
    a = gg.grid(10, 10)
    # two copies of the grid side by side, no arcs between them
    off = np.concatenate([a.offsets[:-1], a.offsets + a.m]).astype(np.uint32)
    idx = np.concatenate([a.indices, a.indices + a.n]).astype(np.uint32)
    g = gg.Graph(2 * a.n, 2 * a.m, off, idx, False)
    d = oracle.bfs(g, 0)
    assert np.all(d[a.n:] == INF) and np.array_equal(d[:a.n], oracle.bfs(a, 0))
    assert oracle.reached_edges(g, d) == (a.n, a.m)


def test_golden_fixtures():
    with open(os.path.join(GOLDEN, "hop_distances.json")) as f:
        cases = json.load(f)["cases"]
    assert len(cases) >= 3
    for case in cases:
        n = case["n"]
        arcs = case["arcs"]
        g = gg.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs],
                         symmetrize=not case["directed"], clean=False,
                         directed=case["directed"])
        for s, want in case["dist"].items():
            got = oracle.bfs(g, int(s)).astype(np.int64)
            want = np.array([INF if w is None else w for w in want], dtype=np.int64)
            assert np.array_equal(got, want), case["name"]


def _tiny_graphs():
    out = []
    for seed in range(6):
        for n, draws in [(1, 3), (2, 1), (9, 12), (24, 30), (48, 60), (64, 300)]:
            out.append(gg.random_graph(n, draws, directed=True, seed=seed, keep_raw=True))
            out.append(gg.random_graph(n, draws, directed=False, seed=seed, keep_raw=True))
    out.append(gg.knn(64, 3, 11))
    out.append(gg.knn(50, 5, 12))
    out.append(gg.rmat(5, 4, 13))
    out.append(gg.rmat(6, 2, 14))
    out.append(gg.dgrid(6, 6, 15))
    out.append(gg.dgrid(7, 5, 16, shortcuts=3))
    out.append(gg.grid(6, 9))
    return out


@pytest.mark.parametrize("g", _tiny_graphs(), ids=lambda g: g.name)
def test_bfs_equals_floyd_warshall(g):
    D = oracle.floyd_warshall(g)
    for s in range(g.n):
        assert np.array_equal(oracle.bfs(g, s), D[s])


@pytest.mark.parametrize("g", _tiny_graphs(), ids=lambda g: g.name)
def test_reach_equals_warshall(g):
    R = oracle.warshall(g)
    rng = np.random.default_rng(g.n)
    k = min(64, g.n)
    srcs = rng.integers(0, g.n, size=k).astype(np.uint32)  # duplicates allowed
    fwd = oracle.reach(g, srcs)
    bwd = oracle.reach(g, srcs, backward=True)
    for j, s in enumerate(srcs):
        bit = np.uint64(1) << np.uint64(j)
        assert np.array_equal((fwd & bit) != 0, R[s, :])
        assert np.array_equal((bwd & bit) != 0, R[:, s])


def test_bfs_multi_is_per_source_bfs():
    g = gg.knn(500, 4, 3)
    srcs = gg.pick_sources(g, 7, 1)
    D = oracle.bfs_multi(g, srcs)
    for j, s in enumerate(srcs):
        assert np.array_equal(D[j], oracle.bfs(g, s))


def test_transpose_is_reverse():
    g = gg.dgrid(9, 8, 3, shortcuts=4)
    toff, tidx = oracle.transpose(g)
    fwd = {(u, int(w)) for u in range(g.n) for w in g.indices[g.offsets[u]:g.offsets[u + 1]]}
    rev = {(int(w), u) for u in range(g.n) for w in tidx[toff[u]:toff[u + 1]]}
    assert fwd == rev and toff[-1] == g.m


def check_bfs_invariants(g, src, dist, undirected):
    """Properties every exact hop-distance array has (any size)."""
    off = g.offsets.astype(np.int64)
    idx = g.indices.astype(np.int64)
    deg = np.diff(off)
    u = np.repeat(np.arange(g.n), deg)
    du = dist[u].astype(np.int64)
    dv = dist[idx].astype(np.int64)
    assert dist[src] == 0
    reached_u = du != INF
    # every arc: dist[v] <= dist[u] + 1
    assert np.all(dv[reached_u] <= du[reached_u] + 1)
    # every reached v != src has a predecessor at dist - 1
    has_pred = np.zeros(g.n, dtype=bool)
    ok = reached_u & (dv == du + 1)
    has_pred[idx[ok]] = True
    reached = dist != INF
    reached[src] = False
    assert np.all(has_pred[reached])
    if undirected:
        both = reached_u & (dv != INF)
        assert np.all(np.abs(du[both] - dv[both]) <= 1)


def test_invariants_knn_and_dgrid():
    g = gg.knn(200_000, 5, 2)
    d = oracle.bfs(g, 0)
    check_bfs_invariants(g, 0, d, True)
    h = gg.dgrid(300, 300, 4)
    src = int(gg.pick_sources(h, 1, 5)[0])
    check_bfs_invariants(h, src, oracle.bfs(h, src), False)


def test_reached_edges_counts():
    g = gg.knn(10_000, 3, 7)
    d = oracle.bfs(g, 0)
    reached = d != INF
    assert oracle.reached_edges(g, d) == (int(reached.sum()), int(g.degrees()[reached].sum()))


def test_parallel_oracle_helper_matches_serial_oracle():
    """The test helper that splits multi-source oracle questions into chunks
    run on several cores returns exactly what one serial call returns."""
    import _oracle_par as par
    g = gg.dgrid(40, 50, 9)
    srcs = gg.pick_sources(g, 20, 3)
    for back in (False, True):
        assert np.array_equal(par.reach(g, srcs, backward=back, chunk=8),
                              oracle.reach(g, srcs, backward=back))
    rows = par.bfs_rows(g, srcs[:5])
    for s in srcs[:5]:
        assert np.array_equal(rows[int(s)], oracle.bfs(g, int(s)))
