"""Parity at the benchmark configurations' full sizes (GPU).

Launch configurations are the ones bench.py times: padded rows uploaded,
library defaults (CTA-cooperative local search), and the learned schedule
when trained weights are present.  Where the oracle can compute the whole
output in seconds it is compared element by element; otherwise sampled
outputs are compared and every output is checked against properties that
hold at any size:
  * C1 grid 1000 x 1000: closed form dist(r, c) = r + c and the oracle;
  * C2 kNN 10M (k = 5): the oracle, every vertex;
  * C3 R-MAT 24: batched 64-source BFS against the oracle on 8 rows
    (rows 0 and 17 and six seeded others), single-source BFS with
    direction optimisation on rows 0 and 17 against the oracle, and on two
    more rows the arc inequality dist[w] <= dist[u] + 1;
  * C4 directed grid 4000 x 4000: 64-source forward and backward masks,
    every bit of every vertex against the oracle (one oracle search per
    source and direction, run on several host cores);
  * C5 held-out kNN 30M (k = 3): the oracle; 1 x 20M strip: dist = index;
  * SCC of the C4 grid against the oracle's Tarjan labels, every vertex.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

import _oracle_par as par

pytestmark = pytest.mark.gpu


def _forms(pg, G):
    forms = {"default": pg.default_config(), "warp_tau8": pg.default_config(tau=8, vgc_mode=1)}
    w = pg.trained_weights()
    if w is not None:
        G.set_schedule_weights(w)
        forms["learned"] = pg.default_config(schedule=pg.PG_SCHED_LEARNED)
    return forms


def test_c1_grid_1000(pg):
    g = gg.grid_1000()
    G = pg.Graph.from_graphgen(g, ell=True)
    r, c = np.meshgrid(np.arange(1000), np.arange(1000), indexing="ij")
    want = (r + c).astype(np.uint32).reshape(-1)
    assert np.array_equal(want, oracle.bfs(g, 0))
    for name, cfg in _forms(pg, G).items():
        assert np.array_equal(pg.to_uint32(G.bfs(0, cfg=cfg)), want), name


def test_c2_knn_10m(pg):
    g = gg.knn_10m()
    G = pg.Graph.from_graphgen(g, ell=True)
    want = oracle.bfs(g, 0)
    for name, cfg in _forms(pg, G).items():
        d = pg.to_uint32(G.bfs(0, cfg=cfg))
        bad = np.flatnonzero(d != want)
        assert len(bad) == 0, (name, len(bad), int(bad[0]))
    n_r, m_r = G.count_reached(G.bfs(0))
    assert (n_r, m_r) == oracle.reached_edges(g, want)


def test_c3_rmat_24(pg):
    g = gg.rmat_24()
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 3)
    D = pg.to_uint32(G.bfs_multi(srcs, cfg=pg.default_config(direction=pg.PG_DIR_AUTO)))
    rng = np.random.default_rng(0)
    rows = sorted({0, 17, *(int(j) for j in rng.choice(64, size=6, replace=False))})
    want = par.bfs_rows(g, [srcs[j] for j in rows])
    for j in rows:
        assert np.array_equal(D[j], want[int(srcs[j])]), int(j)
    # single-source BFS with push/pull switching against the oracle
    for j in (0, 17):
        d = pg.to_uint32(G.bfs(int(srcs[j]), cfg=pg.default_config(tau=1, direction=pg.PG_DIR_AUTO)))
        assert np.array_equal(d, want[int(srcs[j])]), int(j)
    # two more rows: source at 0 and no arc shortens any distance (520M arcs each)
    u = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.offsets.astype(np.int64)))
    for j in (5, 41):
        row = D[j]
        assert row[srcs[j]] == 0
        ru = row[u]
        ok = ru != np.uint32(0xFFFFFFFF)
        assert np.all(row[g.indices[ok]] <= ru[ok] + np.uint32(1))


def test_c4_dgrid_4000_reach(pg):
    """All 64 forward and all 64 backward bits of every vertex against the
    oracle (128 oracle searches, several host cores)."""
    g = gg.dgrid_4000()
    G = pg.Graph.from_graphgen(g, ell=True)
    srcs = gg.pick_sources(g, 64, 4)
    fwd, bwd = G.reach_multi(srcs, pg.PG_FWD | pg.PG_BWD)
    f, b = pg.to_uint64(fwd), pg.to_uint64(bwd)
    want_f = par.reach(g, srcs)
    bad = np.flatnonzero(f != want_f)
    assert len(bad) == 0, ("fwd", len(bad), int(bad[0]))
    want_b = par.reach(g, srcs, backward=True)
    bad = np.flatnonzero(b != want_b)
    assert len(bad) == 0, ("bwd", len(bad), int(bad[0]))


def test_c5_heldout_knn_30m_k3(pg):
    g = gg.knn_30m_k3()
    G = pg.Graph.from_graphgen(g, ell=True)
    want = oracle.bfs(g, 0)
    for name, cfg in _forms(pg, G).items():
        if name == "warp_tau8":
            continue
        d = pg.to_uint32(G.bfs(0, cfg=cfg))
        assert np.array_equal(d, want), name


def test_c5_strip_20m(pg):
    g = gg.strip_20m()
    G = pg.Graph.from_graphgen(g)
    d = pg.to_uint32(G.bfs(0, cfg=pg.default_config(tau=64, timeout_ms=20000)))
    assert np.array_equal(d, np.arange(g.n, dtype=np.uint32))


def test_c4_dgrid_4000_scc(pg):
    """SCC of the full directed grid with shortcuts, element by element."""
    g = gg.dgrid_4000()
    G = pg.Graph.from_graphgen(g, ell=True)
    lab, it = G.scc()
    assert np.array_equal(pg.to_uint32(lab), oracle.scc(g))
    assert it >= 1
