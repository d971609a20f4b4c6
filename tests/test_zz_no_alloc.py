"""The allocation-free BFS entry point (pg_bfs_noalloc) against the oracle
and against pg_bfs.

pg_bfs_noalloc serves callers that cannot allocate device memory at call
time (a framework memory pool that owns the device, a loop where
cudaMalloc's implicit synchronisation is not allowed): it works on the
caller's device CSR and output and keeps its scratch in a fixed array
compiled into the library.  Its distances must equal the oracle's and
pg_bfs's bit for bit (hop distances are integers), on two calls in a row,
since every call reuses the same scratch; one case fills the scratch to its
stated maximum (n = 2^20 vertices).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


@pytest.mark.parametrize("make,srcs", [
    (lambda: gg.knn(80_000, 5, 3), [0, 17]),
    (lambda: gg.dgrid(150, 170, 2), [5, 999]),
    (lambda: gg.grid(300, 251), [0, 75299]),
    (lambda: gg.rmat(14, 8, 6), [1, 2]),
])
def test_noalloc_matches_pg_bfs_on_consecutive_calls(pg, make, srcs):
    import torch
    g = make()
    G = pg.Graph.from_graphgen(g)
    off, idx = _dev(g.offsets), _dev(g.indices)
    for s in srcs:
        s = int(s) % g.n
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        pg.bfs_noalloc(off, idx, s, out, cfg=pg.default_config(tau=8))
        got = pg.to_uint32(out)
        assert np.array_equal(got, oracle.bfs(g, s)), (g.name, s)
        want = pg.to_uint32(G.bfs(s, cfg=pg.default_config(tau=8)))
        assert np.array_equal(got, want), (g.name, s)
    torch.cuda.synchronize()


def test_noalloc_at_the_maximum_size(pg):
    """n = PG_NOALLOC_MAX_N (a 1024 x 1024 grid) uses the whole bag and round-
    tag extent of the fixed scratch; two calls in a row, closed form
    dist(r, c) = |r - r0| + |c - c0| and the oracle."""
    import torch
    g = gg.grid(1024, 1024)
    assert g.n == pg.NOALLOC_MAX_N
    off, idx = _dev(g.offsets), _dev(g.indices)
    r, c = np.meshgrid(np.arange(1024), np.arange(1024), indexing="ij")
    for s in (0, 1024 * 700 + 300):
        out = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
        pg.bfs_noalloc(off, idx, s, out)
        got = pg.to_uint32(out)
        r0, c0 = divmod(s, 1024)
        want = (np.abs(r - r0) + np.abs(c - c0)).astype(np.uint32).reshape(-1)
        assert np.array_equal(got, want), s
        assert np.array_equal(got, oracle.bfs(g, s)), s


def test_noalloc_rejects_what_it_cannot_hold(pg):
    import torch
    n = pg.NOALLOC_MAX_N + 1
    off = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    idx = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(pg.PgError) as e:
        pg.bfs_noalloc(off, idx[:0], 0, out)
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    g = gg.grid(10, 10)
    with pytest.raises(pg.PgError) as e:
        pg.bfs_noalloc(_dev(g.offsets), _dev(g.indices), 100, torch.empty(100, dtype=torch.int32, device="cuda"))
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    bad = g.indices.copy()
    bad[0] = 500
    with pytest.raises(pg.PgError) as e:
        pg.bfs_noalloc(_dev(g.offsets), _dev(bad), 0, torch.empty(100, dtype=torch.int32, device="cuda"))
    assert e.value.status == pg.PG_ERR_INVALID_GRAPH
