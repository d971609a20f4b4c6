"""GPU parity of pg_sssp (weighted shortest paths, Sec. 2.2) against the
oracle's Dijkstra, bit-exact (integer distances).

Cases span tiny graphs with zero weights, self-loops and duplicate arcs,
medium graphs of every generator family, closed forms (weighted path and
grid), every step width from 1 to "one step covers the whole graph" and
every local-search budget (the result may not depend on them), a host
output buffer, argument errors, and a host-chosen barrier stall that must
time out and leave the context usable.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _run(pg, G, s, **kw):
    st = pg.Stats()
    d = G.sssp(s, cfg=pg.default_config(**kw), stats=st)
    return pg.to_uint64(d), st


def test_tiny_graphs_vs_oracle(pg):
    rng = np.random.default_rng(3)
    for t in range(24):
        n = int(rng.integers(2, 60))
        g = gg.random_graph(n, int(rng.integers(0, 5 * n)), directed=bool(t % 2), seed=500 + t,
                            keep_raw=True)
        w = rng.integers(0, 40, size=g.m).astype(np.uint32)
        G = pg.Graph.from_graphgen(g)
        G.set_weights(w)
        for s in (0, n - 1):
            got, _ = _run(pg, G, s, delta=int(rng.integers(1, 60)), tau=int(rng.integers(1, 8)))
            assert np.array_equal(got, oracle.sssp(g, w, s)), (t, s)
        G.free()


MEDIUM = [
    ("knn", lambda: gg.knn(60_000, 5, 7), 1, 1000),
    ("rmat", lambda: gg.rmat(14, 8, 5), 1, 100),
    ("dgrid", lambda: gg.dgrid(120, 130, 4, shortcuts=20), 1, 50),
    ("grid_unit", lambda: gg.grid(300, 251), 1, 1),
]


@pytest.mark.parametrize("name,make,lo,hi", MEDIUM, ids=[m[0] for m in MEDIUM])
def test_medium_vs_oracle_every_schedule(pg, name, make, lo, hi):
    g = make()
    w = gg.edge_weights(g, lo, hi, 11)
    G = pg.Graph.from_graphgen(g)
    G.set_weights(w)
    srcs = [0, int(gg.pick_sources(g, 1, 3)[0])]
    for s in srcs:
        want = oracle.sssp(g, w, s)
        for delta in (1, hi, 8 * hi, 0, 1 << 31):
            for tau in (1, 16, 64):
                got, st = _run(pg, G, s, delta=delta, tau=tau)
                bad = np.flatnonzero(got != want)
                assert len(bad) == 0, (name, s, delta, tau, len(bad))
    if hi == 1:  # unit weights: the hop distances
        b = oracle.bfs(g, 0).astype(np.uint64)
        b[b == np.uint64(oracle.INF)] = np.uint64(oracle.INF64)
        assert np.array_equal(_run(pg, G, 0)[0], b)


def test_weighted_grid_closed_form(pg):
    rows, cols = 200, 300
    g = gg.grid(rows, cols)
    u = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.offsets.astype(np.int64)))
    w = np.where(np.abs(u - g.indices.astype(np.int64)) == 1, 3, 7).astype(np.uint32)
    G = pg.Graph.from_graphgen(g)
    G.set_weights(w)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    s = 120 * cols + 41
    want = (np.abs(r - 120) * 7 + np.abs(c - 41) * 3).astype(np.uint64).reshape(-1)
    got, _ = _run(pg, G, s)
    assert np.array_equal(got, want)


def test_weighted_path_prefix_sums(pg):
    g = gg.strip(5000)
    rng = np.random.default_rng(9)
    step = rng.integers(1, 1000, size=4999).astype(np.uint64)
    u = np.repeat(np.arange(g.n), np.diff(g.offsets.astype(np.int64)))
    w = step[np.minimum(u, g.indices.astype(np.int64))].astype(np.uint32)
    G = pg.Graph.from_graphgen(g)
    G.set_weights(w)
    got, st = _run(pg, G, 0, tau=64)
    assert np.array_equal(got, np.concatenate([[0], np.cumsum(step)]).astype(np.uint64))


def test_host_output_and_errors(pg):
    g = gg.knn(8000, 4, 2)
    w = gg.edge_weights(g, 1, 9, 4)
    G = pg.Graph.from_graphgen(g)
    with pytest.raises(pg.PgError) as e:
        G.sssp(0)                                 # no weights yet
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        G.set_weights(w[:-1])
    G.set_weights(w)
    h = np.empty(g.n, dtype=np.uint64)
    G.sssp(5, out=h)
    assert np.array_equal(h, oracle.sssp(g, w, 5))
    with pytest.raises(pg.PgError) as e:
        G.sssp(g.n)
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    w2 = gg.edge_weights(g, 100, 200, 5)        # replacing the weights
    G.set_weights(w2)
    assert np.array_equal(_run(pg, G, 5)[0], oracle.sssp(g, w2, 5))


def test_sssp_barrier_timeout_is_reported_and_recoverable(pg):
    g = gg.dgrid(40, 40, 5)
    w = gg.edge_weights(g, 1, 20, 1)
    G = pg.Graph.from_graphgen(g)
    G.set_weights(w)
    with pytest.raises(pg.PgError) as e:
        G.sssp(0, cfg=pg.default_config(test_stall_block=1, timeout_ms=300))
    assert e.value.status == pg.PG_ERR_TIMEOUT
    assert np.array_equal(_run(pg, G, 0)[0], oracle.sssp(g, w, 0))
