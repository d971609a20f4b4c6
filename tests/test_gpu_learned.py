"""What the trained schedule network gains over the method without it (GPU).

The committed network (trained on other seeds and sizes by the library's own
MLP kernels) runs inside the persistent traversal and picks tau or a pull
round every round; the method without it is the plain fixed-tau schedule
(tau = 16, the library default).  On held-out graphs both must give the
oracle's distances; the network must be clearly faster where tau = 16 is the
wrong choice (a wide grid wants tau = 64, a path-like strip wants tau = 64,
an R-MAT graph wants plain rounds and a pull), and must not lose more than a
little where tau = 16 is already the best fixed value (kNN).  Times are the
library's kernel events, best of 3 after a warm-up.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


def _best_ms(pg, G, cfg, reps=3):
    st = pg.Stats()
    G.bfs(0, cfg=cfg, stats=st)
    ts = []
    for _ in range(reps):
        out = G.bfs(0, cfg=cfg, stats=st)
        ts.append(st.kernel_ms)
    return min(ts), out


# (graph, minimum speed-up of learned over plain tau = 16)
CASES = [
    ("grid_1100x900_heldout", lambda: gg.grid(1100, 900), 1.10),
    ("strip_1x200000", lambda: gg.strip(200_000), 1.10),
    ("rmat_18_heldout", lambda: gg.rmat(18, 16, 903), 1.10),
    ("knn_2m_k3_heldout", lambda: gg.knn(2_000_000, 3, 902), 0.90),
]


@pytest.mark.parametrize("name,make,min_speedup", CASES, ids=[c[0] for c in CASES])
def test_learned_schedule_gain(pg, name, make, min_speedup):
    w = pg.trained_weights()
    assert w is not None, "trained weights missing from the package"
    g = make()
    G = pg.Graph.from_graphgen(g, ell=True)
    G.set_schedule_weights(w)
    want = oracle.bfs(g, 0)
    t_plain, d_plain = _best_ms(pg, G, pg.default_config())
    t_learn, d_learn = _best_ms(pg, G, pg.default_config(schedule=pg.PG_SCHED_LEARNED))
    assert np.array_equal(pg.to_uint32(d_plain), want)
    assert np.array_equal(pg.to_uint32(d_learn), want)
    speedup = t_plain / t_learn
    print(f"{name}: plain tau=16 {t_plain:.3f} ms, learned {t_learn:.3f} ms, speed-up {speedup:.2f}x")
    assert speedup >= min_speedup, (name, t_plain, t_learn)
