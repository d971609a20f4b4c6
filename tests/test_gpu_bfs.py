"""GPU parity tests for pg_bfs: CUDA path vs the oracle, bit-exact.

Hop distances are integers, so every comparison is exact equality.  Cases
span several tiles and ragged tails (sizes not multiples of 32 or of the
task chunk), hubs (high-degree splitting), pull rounds, every schedule
action, host-memory outputs and the error paths.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
INF = 0xFFFFFFFF


def _bfs(pg, G, src, **kw):
    cfg = pg.default_config(**kw)
    st = pg.Stats()
    d = pg.to_uint32(G.bfs(src, cfg=cfg, stats=st))
    return d, st


def _first_diff(a, b):
    i = np.flatnonzero(a != b)
    return None if len(i) == 0 else (int(i[0]), int(a[i[0]]), int(b[i[0]]), len(i))


@pytest.mark.parametrize("tau", [1, 2, 16, 64])
def test_grid_closed_form(pg, tau):
    rows, cols = 97, 131
    G = pg.Graph.from_graphgen(gg.grid(rows, cols))
    d, st = _bfs(pg, G, 0, tau=tau)
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    assert np.array_equal(d.reshape(rows, cols), (r + c).astype(np.uint32))
    assert st.rounds >= 1


def test_path_cycle_star(pg):
    n = 5001
    P = pg.Graph.from_graphgen(gg.strip(n))
    for tau in (1, 64):
        d, _ = _bfs(pg, P, 1234, tau=tau)
        assert np.array_equal(d, np.abs(np.arange(n) - 1234).astype(np.uint32))
    s = np.arange(n)
    cyc = gg.from_arcs(n, np.concatenate([s, (s + 1) % n]), np.concatenate([(s + 1) % n, s]),
                       directed=False)
    C = pg.Graph.from_graphgen(cyc)
    d, _ = _bfs(pg, C, 7, tau=8)
    k = np.abs(s - 7)
    assert np.array_equal(d, np.minimum(k, n - k).astype(np.uint32))
    star = gg.from_arcs(n, np.concatenate([np.zeros(n - 1), s[1:]]),
                        np.concatenate([s[1:], np.zeros(n - 1)]), directed=False)
    S = pg.Graph.from_graphgen(star)
    d, _ = _bfs(pg, S, 3, tau=4, hub_degree=64)   # vertex 0 is a hub
    want = np.full(n, 2, dtype=np.uint32)
    want[0], want[3] = 1, 0
    assert np.array_equal(d, want)


def _tiny():
    out = []
    for seed in range(4):
        for n, draws in [(1, 2), (9, 12), (64, 300), (200, 900)]:
            out.append(gg.random_graph(n, draws, directed=True, seed=seed, keep_raw=True))
            out.append(gg.random_graph(n, draws, directed=False, seed=seed, keep_raw=True))
    return out


@pytest.mark.parametrize("ell", [True, False])
def test_tiny_graphs_all_sources(pg, ell):
    for g in _tiny():
        G = pg.Graph.from_graphgen(g, ell=ell)
        D = oracle.floyd_warshall(g) if g.n <= 64 else None
        for s in range(0, g.n, max(1, g.n // 9)):
            want = oracle.bfs(g, s)
            if D is not None:
                assert np.array_equal(want, D[s])
            for tau in (1, 8):
                d, _ = _bfs(pg, G, s, tau=tau, chunk=5)
                assert _first_diff(d, want) is None, (g.name, s, tau)
        G.free()


@pytest.mark.parametrize("name,make,directed", [
    ("knn", lambda: gg.knn(150_001, 5, 2), False),
    ("knn_k3", lambda: gg.knn(120_000, 3, 5), False),
    ("rmat", lambda: gg.rmat(16, 16, 3), False),
    ("dgrid", lambda: gg.dgrid(301, 277, 4), True),
])
@pytest.mark.parametrize("ell", [True, False])
def test_medium_vs_oracle(pg, name, make, directed, ell):
    g = make()
    G = pg.Graph.from_graphgen(g, ell=ell)
    srcs = gg.pick_sources(g, 3, 7)
    for s in srcs:
        want = oracle.bfs(g, s)
        for kw in ({"tau": 1}, {"tau": 4, "chunk": 8}, {"tau": 32, "local_queue": 128},
                   {"tau": 16, "hub_degree": 64}, {"tau": 1, "direction": 1},
                   {"tau": 8, "direction": 1, "threads_per_block": 256, "blocks_per_sm": 1},
                   {"tau": 64, "chunk": 2, "local_queue": 32}):
            d, st = _bfs(pg, G, int(s), **kw)
            assert _first_diff(d, want) is None, (name, int(s), kw, _first_diff(d, want))


@pytest.mark.parametrize("make", [lambda: gg.knn(60_000, 4, 9), lambda: gg.rmat(14, 8, 2)])
def test_schedule_independence_fuzz(pg, make):
    """Any per-round action sequence gives the same exact distances."""
    g = make()
    G = pg.Graph.from_graphgen(g)
    want = oracle.bfs(g, 5)
    rng = np.random.default_rng(0)
    for trial in range(12):
        script = rng.integers(0, pg.PG_NUM_ACTIONS, size=int(rng.integers(1, 40))).astype(np.uint8)
        cfg = pg.default_config(schedule=pg.PG_SCHED_SCRIPT, script_len=len(script),
                                chunk=int(rng.integers(1, 33)))
        cfg.script = script.ctypes.data
        d = pg.to_uint32(G.bfs(5, cfg=cfg))
        assert _first_diff(d, want) is None, (trial, script.tolist())
    for seed in range(6):
        d, _ = _bfs(pg, G, 5, schedule=pg.PG_SCHED_RANDOM, seed=seed)
        assert _first_diff(d, want) is None, seed


def test_pull_directed_with_transpose(pg):
    g = gg.dgrid(150, 170, 11)
    G = pg.Graph.from_graphgen(g)
    s = int(gg.pick_sources(g, 1, 3)[0])
    want = oracle.bfs(g, s)
    script = np.array([0, 7, 7, 3, 7, 0, 5], dtype=np.uint8)
    cfg = pg.default_config(schedule=pg.PG_SCHED_SCRIPT, script_len=len(script))
    cfg.script = script.ctypes.data
    st = pg.Stats()
    d = pg.to_uint32(G.bfs(s, cfg=cfg, stats=st))
    assert _first_diff(d, want) is None
    assert st.pull_rounds > 0


def test_unreachable_and_isolated(pg):
    a = gg.grid(10, 12)
    off = np.concatenate([a.offsets[:-1], a.offsets + a.m]).astype(np.uint32)
    idx = np.concatenate([a.indices, a.indices + a.n]).astype(np.uint32)
    # plus one isolated vertex at the end
    off = np.concatenate([off, [off[-1]]]).astype(np.uint32)
    g = gg.Graph(2 * a.n + 1, 2 * a.m, off, idx, False)
    G = pg.Graph.from_graphgen(g)
    d, _ = _bfs(pg, G, 0, tau=4)
    assert np.array_equal(d, oracle.bfs(g, 0))
    d, st = _bfs(pg, G, g.n - 1)
    assert d[-1] == 0 and np.all(d[:-1] == INF)
    one = gg.Graph(1, 0, np.zeros(2, dtype=np.uint32), np.zeros(0, dtype=np.uint32), False)
    O = pg.Graph.from_graphgen(one)
    d, _ = _bfs(pg, O, 0)
    assert d.tolist() == [0]


def test_host_output_and_count(pg):
    import torch
    g = gg.knn(30_000, 5, 3)
    G = pg.Graph.from_graphgen(g)
    out = np.empty(g.n, dtype=np.uint32)
    G.bfs_host(0, out)
    want = oracle.bfs(g, 0)
    assert np.array_equal(out, want)
    d = G.bfs(0)
    assert G.count_reached(d) == oracle.reached_edges(g, want)
    torch.cuda.synchronize()


def test_errors(pg):
    g = gg.grid(5, 5)
    G = pg.Graph.from_graphgen(g)
    with pytest.raises(pg.PgError) as e:
        G.bfs(25)
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    bad = g.indices.copy()
    bad[3] = 99
    with pytest.raises(pg.PgError) as e:
        pg.Graph.upload(g.offsets, bad)
    assert e.value.status == pg.PG_ERR_INVALID_GRAPH
    off = g.offsets.copy()
    off[-1] -= 1
    with pytest.raises(pg.PgError) as e:
        pg.Graph.upload(off, g.indices)
    assert e.value.status == pg.PG_ERR_INVALID_GRAPH
    with pytest.raises(pg.PgError) as e:
        G.bfs(0, cfg=pg.default_config(local_queue=100))
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    dg = gg.dgrid(5, 5, 1)
    d_nt = pg.Graph.upload(dg.offsets, dg.indices, directed=True, transpose=False)
    with pytest.raises(pg.PgError) as e:
        d_nt.reach_multi([0], pg.PG_BWD)
    assert e.value.status == pg.PG_ERR_UNSUPPORTED
    with pytest.raises(pg.PgError) as e:
        G.reach_multi(np.zeros(65, dtype=np.uint32))
    assert e.value.status == pg.PG_ERR_INVALID_ARG


def test_barrier_timeout_is_reported_and_recoverable(pg):
    """A CTA that never arrives: the others give up after timeout_ms."""
    g = gg.grid(50, 50)
    G = pg.Graph.from_graphgen(g)
    with pytest.raises(pg.PgError) as e:
        G.bfs(0, cfg=pg.default_config(test_stall_block=1, timeout_ms=300))
    assert e.value.status == pg.PG_ERR_TIMEOUT
    d, _ = _bfs(pg, G, 0)   # context still usable
    assert np.array_equal(d, oracle.bfs(g, 0))


def test_upload_from_device_tensors(pg):
    import torch
    g = gg.knn(10_000, 6, 1)
    off = torch.from_numpy(g.offsets.view(np.int32)).cuda()
    idx = torch.from_numpy(g.indices.view(np.int32)).cuda()
    G = pg.Graph.upload(off, idx)
    d, _ = _bfs(pg, G, 17)
    assert np.array_equal(d, oracle.bfs(g, 17))


def test_upload_free_cycles_reuse_pool_memory(pg):
    """Graphs of different sizes uploaded and freed in turn (their buffers
    are recycled through the device memory pool) keep giving exact results,
    including host-output calls that stage through a pooled buffer."""
    graphs = [gg.knn(30_000, 5, 3), gg.dgrid(90, 110, 2, shortcuts=5), gg.knn(8_000, 3, 4)]
    want = [oracle.bfs(g, 1) for g in graphs]
    for cycle in range(4):
        for g, w in zip(graphs, want):
            G = pg.Graph.from_graphgen(g, ell=(cycle % 2 == 0))
            d, _ = _bfs(pg, G, 1)
            assert np.array_equal(d, w), (cycle, g.name)
            h = np.empty(g.n, dtype=np.uint32)
            G.bfs_host(1, h)
            assert np.array_equal(h, w), (cycle, g.name)
            G.free()


def test_batched_bfs_barrier_timeout_is_reported_and_recoverable(pg):
    """pg_bfs_multi's persistent kernel with one CTA that never arrives at the
    grid barrier (a host-chosen stall): the others give up after timeout_ms,
    the call returns PG_ERR_TIMEOUT and the next call in the same context is
    exact."""
    g = gg.dgrid(40, 40, 5)
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 8, 2)
    with pytest.raises(pg.PgError) as e:
        G.bfs_multi(srcs, cfg=pg.default_config(test_stall_block=1, timeout_ms=300))
    assert e.value.status == pg.PG_ERR_TIMEOUT
    D = pg.to_uint32(G.bfs_multi(srcs))
    assert np.array_equal(D, oracle.bfs_multi(g, srcs))


MULTI_FRONTIER = [
    ("knn", lambda: gg.knn(150_001, 5, 2), False),
    ("rmat", lambda: gg.rmat(16, 16, 3), False),
    ("dgrid", lambda: gg.dgrid(301, 277, 4), True),
    ("grid", lambda: gg.grid(400, 311), False),
]


@pytest.mark.parametrize("name,make,directed", MULTI_FRONTIER, ids=[m[0] for m in MULTI_FRONTIER])
@pytest.mark.parametrize("ell", [True, False])
def test_multi_frontier_buckets_vs_oracle(pg, name, make, directed, ell):
    """The multiple-frontier local search (PG_VGC_BUCKETS: phases at depths
    1, 2, 4, ... < tau with a grid barrier between them) gives the oracle's
    distances for every tau, with hubs split and with a small CTA queue
    (rounds whose frontier exceeds the CTAs' buffers run unphased)."""
    g = make()
    G = pg.Graph.from_graphgen(g, ell=ell)
    for s in gg.pick_sources(g, 2, 13):
        want = oracle.bfs(g, int(s))
        for kw in ({"tau": 2}, {"tau": 8}, {"tau": 16}, {"tau": 64}, {"tau": 64, "cta_queue": 64},
                   {"tau": 16, "hub_degree": 64}, {"tau": 32, "direction": 1}):
            d, st = _bfs(pg, G, int(s), vgc_mode=pg.PG_VGC_BUCKETS, **kw)
            assert _first_diff(d, want) is None, (name, int(s), kw, _first_diff(d, want))


def test_multi_frontier_schedules_and_reach(pg):
    """Scripted and random per-round actions with the multiple-frontier
    search; tiny graphs from every source; reachability masks."""
    g = gg.knn(60_000, 4, 9)
    G = pg.Graph.from_graphgen(g, ell=True)
    want = oracle.bfs(g, 5)
    rng = np.random.default_rng(4)
    for trial in range(8):
        script = rng.integers(0, pg.PG_NUM_ACTIONS, size=int(rng.integers(1, 40))).astype(np.uint8)
        cfg = pg.default_config(schedule=pg.PG_SCHED_SCRIPT, script_len=len(script),
                                vgc_mode=pg.PG_VGC_BUCKETS)
        cfg.script = script.ctypes.data
        assert _first_diff(pg.to_uint32(G.bfs(5, cfg=cfg)), want) is None, (trial, script.tolist())
    for seed in range(4):
        d, _ = _bfs(pg, G, 5, schedule=pg.PG_SCHED_RANDOM, seed=seed, vgc_mode=pg.PG_VGC_BUCKETS)
        assert _first_diff(d, want) is None, seed
    for t in _tiny():
        T = pg.Graph.from_graphgen(t)
        for s in range(0, t.n, max(1, t.n // 5)):
            d, _ = _bfs(pg, T, s, tau=8, vgc_mode=pg.PG_VGC_BUCKETS)
            assert _first_diff(d, oracle.bfs(t, s)) is None, (t.name, s)
        T.free()
    h = gg.dgrid(90, 110, 6, shortcuts=9)
    H = pg.Graph.from_graphgen(h, ell=True)
    srcs = gg.pick_sources(h, 64, 2)
    f, b = H.reach_multi(srcs, pg.PG_FWD | pg.PG_BWD,
                         cfg=pg.default_config(tau=16, vgc_mode=pg.PG_VGC_BUCKETS))
    assert np.array_equal(pg.to_uint64(f), oracle.reach(h, srcs))
    assert np.array_equal(pg.to_uint64(b), oracle.reach(h, srcs, backward=True))
    w = pg.trained_weights()
    if w is not None:
        G.set_schedule_weights(w)
        d, _ = _bfs(pg, G, 5, schedule=pg.PG_SCHED_LEARNED, vgc_mode=pg.PG_VGC_BUCKETS)
        assert _first_diff(d, want) is None
