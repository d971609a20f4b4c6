"""Run independent oracle calls on several host cores (test helper).

The oracle itself stays serial and unchanged: this helper only splits a
multi-source question into independent single-purpose oracle calls (one
chunk of sources each) and runs them in threads.  ctypes releases the GIL
for the duration of a foreign call, so the chunks run in parallel.  No
process is forked (the GPU context of the test process stays untouched).
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle


def workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def reach(g, srcs, backward: bool = False, chunk: int = 8) -> np.ndarray:
    """oracle.reach over all sources, computed chunk by chunk in parallel;
    bit j of the result belongs to srcs[j], as in oracle.reach."""
    srcs = np.asarray(srcs, dtype=np.uint32)
    parts = [(i, srcs[i:i + chunk]) for i in range(0, len(srcs), chunk)]
    out = np.zeros(g.n, dtype=np.uint64)
    with cf.ThreadPoolExecutor(max_workers=min(workers(), len(parts))) as ex:
        futs = {ex.submit(oracle.reach, g, s, backward): i for i, s in parts}
        for f in cf.as_completed(futs):
            out |= f.result() << np.uint64(futs[f])
    return out


def bfs_rows(g, srcs) -> dict:
    """{source: oracle.bfs(g, source)} for every distinct source, in parallel."""
    uniq = sorted({int(s) for s in srcs})
    with cf.ThreadPoolExecutor(max_workers=min(workers(), len(uniq))) as ex:
        res = list(ex.map(lambda s: oracle.bfs(g, s), uniq))
    return dict(zip(uniq, res))
