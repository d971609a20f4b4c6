"""Schedule-network kernels against the fp64 oracle (oracle/mlp.py).

Tolerance: the kernels compute in fp32 with fused multiply-adds in a fixed
order; the oracle in fp64.  For inputs in [0,1] and weights of unit scale,
sums of <= 32 products give relative errors of a few 1e-7 per layer, and the
gradient sums over B = 700 rows add at most ~1e-4 relative; the tests use
rtol = 1e-4 with an absolute floor of 1e-5 (scaled by the tensor's largest
entry).  The in-loop decision must equal the oracle's arg-max except where
the top two outputs are within 1e-4 of each other.
"""
import numpy as np
import pytest

import graphgen as gg
from oracle import mlp

pytestmark = pytest.mark.gpu


def _close(got, want, rtol=1e-4, atol_rel=1e-5):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    atol = atol_rel * max(1.0, float(np.abs(want).max()))
    return np.allclose(got, want, rtol=rtol, atol=atol)


def _rand(seed, B):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.4, size=mlp.N_PARAMS)
    X = rng.uniform(0, 1, size=(B, 5))
    a = rng.integers(0, 8, size=B)
    t = rng.normal(size=B)
    return p, X, a, t


@pytest.mark.parametrize("B", [1, 31, 700])
def test_forward_backward_match_oracle(pg, B):
    import torch
    p, X, a, t = _rand(B, B)
    P = torch.tensor(p, dtype=torch.float32, device="cuda")
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Ad = torch.tensor(a, dtype=torch.int32, device="cuda")
    Td = torch.tensor(t, dtype=torch.float32, device="cuda")
    # the oracle evaluates the fp32-rounded inputs
    p32, X32, t32 = (np.asarray(v, np.float32).astype(np.float64) for v in (p, X, t))
    Y = pg.mlp_forward(P, Xd).cpu().numpy()
    Yw, _ = mlp.forward(p32, X32)
    assert _close(Y, Yw)
    loss, grad = pg.mlp_backward(P, Xd, Ad, Td)
    Lw, Gw = mlp.backward(p32, X32, a, t32)
    assert _close([loss.item()], [Lw])
    assert _close(grad.cpu().numpy(), Gw, rtol=2e-4)


def test_adam_matches_oracle(pg):
    import torch
    rng = np.random.default_rng(5)
    p = rng.normal(size=mlp.N_PARAMS).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    P, M, V = (torch.tensor(x, device="cuda") for x in (p, m, v))
    pw, mw, vw = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 4):
        g = rng.normal(size=mlp.N_PARAMS).astype(np.float32)
        pg.mlp_adam(P, torch.tensor(g, device="cuda"), M, V, t, lr=1e-2)
        pw, mw, vw = mlp.adam_step(pw, g.astype(np.float64), mw, vw, t, lr=1e-2)
    assert _close(P.cpu().numpy(), pw, rtol=1e-5, atol_rel=1e-6)
    assert _close(M.cpu().numpy(), mw, rtol=1e-5, atol_rel=1e-6)


JUDGE_UP, JUDGE_DOWN = 0.1, 0.3  # the kernel's margins for overriding the fixed-tau action
A_FIX = 4                        # push with the default tau = 16


def test_in_loop_decision_matches_oracle_argmax(pg):
    """The traversal's choice for round r >= 1 is the arg-max of the network on
    the features recorded in round r - 1 (CTA 0 evaluates it while waiting at
    the barrier that ends round r - 1), and round 0's on round 0's own
    features (known before the first barrier), unless that beats the fixed-tau
    action by no more than the judge margin.  This pins the in-kernel
    inference and the judge; the result is still exact."""
    import oracle
    g = gg.knn(200_000, 5, 4)
    G = pg.Graph.from_graphgen(g)
    rng = np.random.default_rng(9)
    for trial in range(3):
        w = rng.normal(0, 0.5, size=mlp.N_PARAMS).astype(np.float32)
        G.set_schedule_weights(w)
        cap = 20000
        buf = (pg.RoundTrace * cap)()
        cfg = pg.default_config(schedule=pg.PG_SCHED_LEARNED, trace_cap=cap)
        cfg.trace_out = buf
        st = pg.Stats()
        d = pg.to_uint32(G.bfs(0, cfg=cfg, stats=st))
        assert np.array_equal(d, oracle.bfs(g, 0))
        R = min(st.rounds, cap)
        X = np.array([list(buf[r].features) for r in range(R)], dtype=np.float32)
        acts = np.array([buf[r].action for r in range(R)])
        Y, _ = mlp.forward(w.astype(np.float64), X.astype(np.float64))
        for r in range(R):
            y = Y[max(r - 1, 0)]
            order = np.argsort(-y)
            if y[order[0]] - y[order[1]] < 1e-4:
                continue
            gain = y[order[0]] - y[A_FIX]
            margin = JUDGE_DOWN if order[0] < A_FIX else JUDGE_UP
            if abs(gain - margin) < 1e-4:
                continue
            want = order[0] if gain > margin else A_FIX
            assert acts[r] == want, (trial, r, acts[r], order[:3], y)


def test_features_match_definition(pg):
    """Recorded features equal the oracle's feature formula on the recorded
    raw statistics (frontier size, out-edges, round index)."""
    g = gg.grid(300, 400)
    G = pg.Graph.from_graphgen(g)
    cap = 5000
    buf = (pg.RoundTrace * cap)()
    cfg = pg.default_config(tau=4, trace_cap=cap)
    cfg.trace_out = buf
    st = pg.Stats()
    G.bfs(0, cfg=cfg, stats=st)
    R = min(st.rounds, cap)
    F = np.array([buf[r].frontier for r in range(R)], dtype=np.float64)
    E = np.array([buf[r].out_edges for r in range(R)], dtype=np.float64)
    X = np.array([list(buf[r].features) for r in range(R)], dtype=np.float64)
    want = mlp.features(F, E, np.arange(R), np.zeros(R))
    assert np.allclose(X[:, :4], want[:, :4], rtol=1e-5, atol=1e-6)
    assert np.all(X[:, 4] >= 0)
