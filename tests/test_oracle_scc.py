"""Pins for the oracle's strongly connected components (no GPU).

An SCC is a maximal vertex set in which every vertex reaches every other
(Sec. 2).  The oracle (Tarjan's algorithm, the paper's sequential SCC
baseline) is checked against things other than itself:
  * brute force: u and v share a label iff each reaches the other in the
    Warshall transitive closure, on tiny seeded graphs from the same
    generator code paths as the benchmark graphs (self-loops and duplicate
    arcs included), and every label is the smallest id of its class;
  * closed forms: a directed cycle is one component, a directed path (and
    any DAG) has only singletons, a symmetric graph's components are its
    connected components (BFS from the smallest vertex), and a long path
    closed into a cycle by one arc (depth 200k: no recursion limit) is one
    component;
  * the definition at medium size: for 64 sampled roots r on a directed
    grid with shortcuts, the vertices labelled like r are exactly those that
    r reaches and that reach r (the independent reachability oracle);
  * the condensation is acyclic (Kahn's topological sort of the quotient
    graph consumes every component).
A planted error (a low-link taken from a finished component, a wrong stack
pop boundary, a label other than the minimum, an arc direction flipped)
fails at least one of these.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle


def _tiny():
    out = []
    for seed in range(5):
        for n, draws in [(1, 3), (2, 2), (9, 14), (24, 40), (48, 70), (64, 160)]:
            out.append(gg.random_graph(n, draws, directed=True, seed=seed, keep_raw=True))
    out.append(gg.dgrid(6, 6, 15))
    out.append(gg.dgrid(7, 5, 16, shortcuts=3))
    out.append(gg.rmat(5, 4, 13))
    return out


@pytest.mark.parametrize("g", _tiny(), ids=lambda g: g.name)
def test_scc_equals_mutual_reachability(g):
    R = oracle.warshall(g).astype(bool)
    np.fill_diagonal(R, True)
    mutual = R & R.T
    lab = oracle.scc(g)
    assert np.array_equal(lab[:, None] == lab[None, :], mutual)
    for v in range(g.n):
        assert lab[v] == np.flatnonzero(mutual[v]).min()


def test_cycle_path_dag():
    n = 50
    cyc = gg.from_arcs(n, np.arange(n), (np.arange(n) + 1) % n, directed=True)
    assert np.all(oracle.scc(cyc) == 0)
    path = gg.from_arcs(n, np.arange(n - 1), np.arange(1, n), directed=True)
    assert np.array_equal(oracle.scc(path), np.arange(n))
    rng = np.random.default_rng(3)
    a = rng.integers(0, n, 400)
    b = rng.integers(0, n, 400)
    keep = a != b
    dag = gg.from_arcs(n, np.minimum(a, b)[keep], np.maximum(a, b)[keep], directed=True)
    assert np.array_equal(oracle.scc(dag), np.arange(n))


def test_symmetric_graph_components():
    g = gg.random_graph(3000, 2600, directed=False, seed=9)
    lab = oracle.scc(g)
    want = np.full(g.n, -1, dtype=np.int64)
    for v in range(g.n):
        if want[v] < 0:
            d = oracle.bfs(g, v)
            want[d != oracle.INF] = v  # v is the smallest id of its component
    assert np.array_equal(lab, want.astype(np.uint32))


def test_deep_cycle_no_recursion():
    n = 200_000
    src = np.arange(n)
    dst = (np.arange(n) + 1) % n
    lab = oracle.scc(gg.from_arcs(n, src, dst, directed=True))
    assert np.all(lab == 0)
    lab = oracle.scc(gg.from_arcs(n, src[:-1], dst[:-1], directed=True))
    assert np.array_equal(lab, np.arange(n))


def test_definition_on_dgrid_with_shortcuts():
    g = gg.dgrid(60, 70, 21, shortcuts=6)
    lab = oracle.scc(g)
    roots = gg.pick_sources(g, 64, 2)
    fwd = oracle.reach(g, roots)
    bwd = oracle.reach(g, roots, backward=True)
    for j, r in enumerate(roots):
        bit = np.uint64(1) << np.uint64(j)
        both = ((fwd & bit) != 0) & ((bwd & bit) != 0)
        assert np.array_equal(both, lab == lab[r]), int(r)


def test_condensation_is_acyclic():
    g = gg.dgrid(80, 90, 22, shortcuts=10)
    lab = oracle.scc(g)
    u = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    w = g.indices.astype(np.int64)
    cross = lab[u] != lab[w]
    comps = np.unique(lab)
    cid = {int(c): i for i, c in enumerate(comps)}
    a = np.array([cid[int(x)] for x in lab[u][cross]], dtype=np.int64)
    b = np.array([cid[int(x)] for x in lab[w][cross]], dtype=np.int64)
    pairs = np.unique(np.stack([a, b], 1), axis=0) if len(a) else np.zeros((0, 2), np.int64)
    indeg = np.bincount(pairs[:, 1], minlength=len(comps))
    out = [[] for _ in comps]
    for x, y in pairs:
        out[x].append(y)
    stack = [i for i in range(len(comps)) if indeg[i] == 0]
    seen = 0
    while stack:
        x = stack.pop()
        seen += 1
        for y in out[x]:
            indeg[y] -= 1
            if indeg[y] == 0:
                stack.append(y)
    assert seen == len(comps)
