"""GPU parity tests for pg_reach_multi and pg_bfs_multi (bit-exact).

Reachability masks: bit j of fwd[v] = v reachable from sources[j]; bit j of
bwd[v] = sources[j] reachable from v (Sec. 2.1).  Batched BFS must equal k
independent queue BFS runs (Sec. 2.2).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _reach(pg, G, srcs, direction, **kw):
    fwd, bwd = G.reach_multi(srcs, direction, cfg=pg.default_config(**kw))
    return (pg.to_uint64(fwd) if fwd is not None else None,
            pg.to_uint64(bwd) if bwd is not None else None)


def test_tiny_vs_warshall(pg):
    for seed in range(5):
        for n, draws, directed in [(1, 1, True), (30, 40, True), (64, 200, True), (50, 60, False)]:
            g = gg.random_graph(n, draws, directed=directed, seed=seed, keep_raw=True)
            G = pg.Graph.from_graphgen(g)
            R = oracle.warshall(g)
            rng = np.random.default_rng(seed)
            k = int(rng.integers(1, 65))
            srcs = rng.integers(0, n, size=k).astype(np.uint32)   # duplicates allowed
            for tau in (1, 8):
                f, b = _reach(pg, G, srcs, pg.PG_FWD | pg.PG_BWD, tau=tau)
                for j, s in enumerate(srcs):
                    bit = np.uint64(1) << np.uint64(j)
                    assert np.array_equal((f & bit) != 0, R[s, :]), (seed, n, j)
                    assert np.array_equal((b & bit) != 0, R[:, s]), (seed, n, j)
                hi = ~np.uint64(0) << np.uint64(k) if k < 64 else np.uint64(0)
                assert not np.any(f & hi) and not np.any(b & hi)


@pytest.mark.parametrize("ell", [True, False])
@pytest.mark.parametrize("tau,kw", [(1, {}), (16, {}), (64, {"chunk": 4}),
                                     (8, {"hub_degree": 32, "local_queue": 64})])
def test_dgrid_fwd_bwd(pg, tau, kw, ell):
    g = gg.dgrid(211, 199, 4)
    G = pg.Graph.from_graphgen(g, ell=ell)
    srcs = gg.pick_sources(g, 64, 2)
    f, b = _reach(pg, G, srcs, pg.PG_FWD | pg.PG_BWD, tau=tau, **kw)
    assert np.array_equal(f, oracle.reach(g, srcs))
    assert np.array_equal(b, oracle.reach(g, srcs, backward=True))
    f1, _ = _reach(pg, G, srcs[:5], pg.PG_FWD, tau=tau)
    assert np.array_equal(f1, oracle.reach(g, srcs[:5]))
    _, b1 = _reach(pg, G, srcs[:1], pg.PG_BWD, tau=tau)
    assert np.array_equal(b1, oracle.reach(g, srcs[:1], backward=True))


def test_undirected_reach_is_finite_distance(pg):
    g = gg.knn(40_000, 2, 6)   # k = 2 leaves many components
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 3)
    f, b = _reach(pg, G, srcs, pg.PG_FWD | pg.PG_BWD, tau=16)
    assert np.array_equal(f, b)
    D = oracle.bfs_multi(g, srcs)
    for j in range(64):
        assert np.array_equal(((f >> np.uint64(j)) & np.uint64(1)) == 1, D[j] != oracle.INF)


def test_rmat_hubs(pg):
    g = gg.rmat(15, 16, 8)
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 4)
    f, _ = _reach(pg, G, srcs, pg.PG_FWD, tau=4, hub_degree=128)
    assert np.array_equal(f, oracle.reach(g, srcs))


@pytest.mark.parametrize("make,k", [(lambda: gg.rmat(15, 16, 3), 64), (lambda: gg.knn(50_000, 5, 2), 17),
                                    (lambda: gg.dgrid(120, 130, 4), 64), (lambda: gg.grid(33, 70), 1)])
def test_bfs_multi_vs_oracle(pg, make, k):
    g = make()
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, k, 5)
    want = oracle.bfs_multi(g, srcs)
    for direction in (0, 1):
        st = pg.Stats()
        D = pg.to_uint32(G.bfs_multi(srcs, cfg=pg.default_config(direction=direction), stats=st))
        assert np.array_equal(D, want), direction


def test_bfs_multi_output_alignment(pg):
    """The decode pass writes four vertices per 16-byte store when n is a
    multiple of 4 and the output starts on a 16-byte boundary, else one per
    4-byte store: an output 4 bytes past an aligned start takes the second
    path; distances up to ~100 exercise the directly written codes (>= 31);
    a short output is refused before anything launches."""
    import torch
    g = gg.knn(20_000, 5, 3)
    assert g.n % 4 == 0
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 9, 2)
    want = oracle.bfs_multi(g, srcs)
    assert want[want != oracle.INF].max() >= 31
    buf = torch.empty(9 * g.n + 4, dtype=torch.int32, device="cuda")
    for off in (0, 1):
        D = buf[off:off + 9 * g.n].view(9, g.n)
        G.bfs_multi(srcs, out=D)
        assert np.array_equal(pg.to_uint32(D), want), off
    with pytest.raises(ValueError):
        G.bfs_multi(srcs, out=buf[:9 * g.n - 1])


def test_bfs_multi_duplicate_sources(pg):
    g = gg.knn(5000, 4, 1)
    G = pg.Graph.from_graphgen(g)
    srcs = np.array([3, 3, 9, 3], dtype=np.uint32)
    D = pg.to_uint32(G.bfs_multi(srcs))
    assert np.array_equal(D, oracle.bfs_multi(g, srcs))


def _heavy_directed():
    """Directed graph with hubs far above the chunk size in both directions."""
    rng = np.random.default_rng(12)
    n = 20_000
    src = [rng.integers(0, n, 60_000)]
    dst = [rng.integers(0, n, 60_000)]
    src.append(np.full(5000, 7)); dst.append(rng.integers(0, n, 5000))        # out-hub
    src.append(rng.integers(0, n, 3000)); dst.append(np.full(3000, 11))       # in-hub
    src.append(np.arange(0, 900)); dst.append(np.arange(1, 901))              # a chain
    return gg.from_arcs(n, np.concatenate(src), np.concatenate(dst), directed=True)


def test_bfs_multi_heavy_directed(pg):
    """Chunked high-degree vertices, top-down and bottom-up, on a directed graph."""
    g = _heavy_directed()
    G = pg.Graph.from_graphgen(g)
    srcs = np.concatenate([[7, 11, 0], gg.pick_sources(g, 61, 6)]).astype(np.uint32)
    want = oracle.bfs_multi(g, srcs)
    for direction in (0, 1):
        D = pg.to_uint32(G.bfs_multi(srcs, cfg=pg.default_config(direction=direction)))
        assert np.array_equal(D, want), direction
    # replacing the transpose rebuilds the in-edge chunk lists
    toff, tidx = oracle.transpose(g)
    G.set_transpose(toff, tidx)
    D = pg.to_uint32(G.bfs_multi(srcs, cfg=pg.default_config(direction=1)))
    assert np.array_equal(D, want)


def _ell_width(deg):
    """The library's padded-row width rule: the smallest of 4 / 8 / 16 that
    all but 0.1% of the vertices fit (0: no padded rows)."""
    tol = len(deg) // 1000
    for w in (4, 8, 16):
        if int((deg > w).sum()) <= tol:
            return w
    return 0


def test_padded_rows_of_different_widths(pg):
    """Forward rows 4 wide, reverse rows 8 wide: slot-parallel waves group
    lanes by the wider row and each direction uses its own width."""
    rng = np.random.default_rng(21)
    n = 50_000
    src = np.repeat(np.arange(n), 2)
    dst = rng.integers(0, n, 2 * n)
    g = gg.from_arcs(n, src, dst, directed=True)
    toff, _ = oracle.transpose(g)
    assert _ell_width(np.diff(g.offsets.astype(np.int64))) == 4
    assert _ell_width(np.diff(toff.astype(np.int64))) == 8
    G = pg.Graph.from_graphgen(g, ell=True)
    srcs = gg.pick_sources(g, 64, 8)
    want_f, want_b = oracle.reach(g, srcs), oracle.reach(g, srcs, backward=True)
    for tau in (1, 4, 16, 64):
        f, b = _reach(pg, G, srcs, pg.PG_FWD | pg.PG_BWD, tau=tau)
        assert np.array_equal(f, want_f), tau
        assert np.array_equal(b, want_b), tau
    for s_ in srcs[:4]:
        d = pg.to_uint32(G.bfs(int(s_), cfg=pg.default_config(tau=16)))
        assert np.array_equal(d, oracle.bfs(g, int(s_)))


@pytest.mark.parametrize("alpha,beta", [(2, 2), (1000, 2), (1, 1000), (3, 50)])
@pytest.mark.parametrize("make", [lambda: gg.rmat(16, 16, 21), lambda: gg.knn(60_000, 5, 22),
                                  lambda: _heavy_directed()])
def test_bfs_multi_direction_switching(pg, make, alpha, beta):
    """Batched BFS with push/pull thresholds that switch direction often:
    top-down rounds that follow bottom-up rounds see visit words left over
    from older rounds (hubs included), and bottom-up rounds that follow
    top-down rounds resume from the unfinished list; every row must equal the
    oracle's BFS."""
    g = make()
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 9)
    st = pg.Stats()
    D = pg.to_uint32(G.bfs_multi(srcs, cfg=pg.default_config(direction=pg.PG_DIR_AUTO, alpha=alpha,
                                                              beta=beta), stats=st))
    assert np.array_equal(D, oracle.bfs_multi(g, srcs)), (st.rounds, st.pull_rounds)


def test_autotuned_configurations_are_exact(pg):
    """pg_autotune picks a launch shape and tau by timing; whatever it picks,
    the tuned configuration's output must equal the oracle's: BFS (kind 0)
    on a kNN graph with padded rows, forward + backward reachability (kind
    1) on a directed grid."""
    g = gg.knn(300_000, 5, 12)
    G = pg.Graph.from_graphgen(g, ell=True)
    cfg = G.autotune([0], kind=0, trials=1)
    assert cfg.tau >= 1 and cfg.threads_per_block in (0, 256, 512)
    d = pg.to_uint32(G.bfs(0, cfg=cfg))
    assert np.array_equal(d, oracle.bfs(g, 0)), (cfg.tau, cfg.vgc_mode, cfg.chunk)
    h = gg.dgrid(400, 500, 7, shortcuts=20)
    H = pg.Graph.from_graphgen(h, ell=True)
    srcs = gg.pick_sources(h, 64, 8)
    both = pg.PG_FWD | pg.PG_BWD
    tuned = H.autotune(srcs, kind=1, direction=both, trials=1)
    f, b = H.reach_multi(srcs, both, cfg=tuned)
    assert np.array_equal(pg.to_uint64(f), oracle.reach(h, srcs)), (tuned.tau, tuned.vgc_mode)
    assert np.array_equal(pg.to_uint64(b), oracle.reach(h, srcs, backward=True))


def test_autotuned_batched_bfs_is_exact(pg):
    """Kind 2 tunes the batched BFS's chunk length, alpha and CTAs per SM; the
    tuned configuration and chunk lengths different from the default
    (rebuilt chunk lists) give the oracle's rows."""
    g = gg.rmat(15, 16, 31)
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 3)
    want = oracle.bfs_multi(g, srcs)
    tuned = G.autotune(srcs, kind=2, trials=1, cfg=pg.default_config(direction=pg.PG_DIR_AUTO))
    assert tuned.hub_degree in (256, 512, 1024, 2048, 4096)
    assert np.array_equal(pg.to_uint32(G.bfs_multi(srcs, cfg=tuned)), want)
    for clen in (32, 100, 4096):
        D = G.bfs_multi(srcs, cfg=pg.default_config(direction=pg.PG_DIR_AUTO, hub_degree=clen))
        assert np.array_equal(pg.to_uint32(D), want), clen
