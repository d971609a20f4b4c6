"""SCC through the C ABI (pg_scc) against the oracle's Tarjan labels (GPU).

Labels are canonical (the smallest vertex id of each component), so the
comparison is element by element: tiny seeded directed graphs with
self-loops and duplicate arcs, directed grids with shortcuts, a directed
cycle and path (closed forms: one component / all singletons), undirected
kNN graphs (components), and several search configurations (tau 1 / 16 /
64, a 32-entry local queue that overflows into the bags, 64-thread CTAs).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _labels(pg, G, **kw):
    cfg = pg.default_config(**kw) if kw else None
    st = pg.Stats()
    lab, it = G.scc(cfg=cfg, stats=st)
    return pg.to_uint32(lab), it, st


def _tiny():
    out = []
    for seed in range(4):
        for n, draws in [(1, 2), (2, 3), (9, 14), (40, 70), (64, 150), (300, 420)]:
            out.append(gg.random_graph(n, draws, directed=True, seed=seed, keep_raw=True))
    return out


@pytest.mark.parametrize("g", _tiny(), ids=lambda g: g.name)
def test_tiny_vs_tarjan(pg, g):
    G = pg.Graph.from_graphgen(g)
    want = oracle.scc(g)
    for kw in ({}, {"tau": 1}, {"tau": 64, "local_queue": 32, "threads_per_block": 64}):
        got, _, _ = _labels(pg, G, **kw)
        assert np.array_equal(got, want), kw


@pytest.mark.parametrize("rows,cols,seed,sc", [(40, 50, 3, 0), (120, 130, 4, 20), (300, 200, 7, 60)])
def test_dgrid_vs_tarjan(pg, rows, cols, seed, sc):
    g = gg.dgrid(rows, cols, seed, shortcuts=sc)
    G = pg.Graph.from_graphgen(g)
    want = oracle.scc(g)
    for kw in ({}, {"tau": 4, "seed": 5}):
        got, it, st = _labels(pg, G, **kw)
        assert np.array_equal(got, want), kw
        assert it >= 1 and st.kernel_ms > 0


def test_cycle_and_path_closed_forms(pg):
    n = 50_000
    cyc = gg.from_arcs(n, np.arange(n), (np.arange(n) + 1) % n, directed=True)
    got, _, _ = _labels(pg, pg.Graph.from_graphgen(cyc))
    assert np.all(got == 0)
    path = gg.from_arcs(n, np.arange(n - 1), np.arange(1, n), directed=True)
    got, _, _ = _labels(pg, pg.Graph.from_graphgen(path))
    assert np.array_equal(got, np.arange(n, dtype=np.uint32))


def test_undirected_components(pg):
    g = gg.knn(40_000, 2, 31)
    G = pg.Graph.from_graphgen(g, ell=True)
    got, _, _ = _labels(pg, G)
    assert np.array_equal(got, oracle.scc(g))


def test_host_output_and_missing_transpose(pg):
    g = gg.dgrid(30, 30, 9, shortcuts=4)
    G = pg.Graph.from_graphgen(g)
    want = oracle.scc(g)
    out = np.empty(g.n, dtype=np.uint32)
    G.scc(out=out)
    assert np.array_equal(out, want)
    lab, _ = G.scc()
    assert np.array_equal(pg.to_uint32(lab), want)
    H = pg.Graph.upload(g.offsets, g.indices, directed=True, transpose=False)
    with pytest.raises(pg.PgError) as e:
        H.scc()
    assert e.value.status == pg.PG_ERR_UNSUPPORTED


def test_scc_barrier_timeout_is_reported_and_recoverable(pg):
    """The SCC search kernel with one CTA that never arrives at the grid
    barrier (a host-chosen stall): PG_ERR_TIMEOUT after timeout_ms, then an
    exact SCC in the same context."""
    g = gg.dgrid(40, 40, 5)
    G = pg.Graph.from_graphgen(g)
    with pytest.raises(pg.PgError) as e:
        G.scc(cfg=pg.default_config(test_stall_block=1, timeout_ms=300))
    assert e.value.status == pg.PG_ERR_TIMEOUT
    lab, _ = G.scc()
    assert np.array_equal(pg.to_uint32(lab), oracle.scc(g))
