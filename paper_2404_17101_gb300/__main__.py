"""Command line: run one traversal on a graph file or a named workload.

    python -m paper_2404_17101_gb300 bfs   --input g.adj [--directed] [--source 0] [--tau 16]
                                           [--learned] [--out dist.u32]
    python -m paper_2404_17101_gb300 reach --input g.adj --sources 0,5,9 [--directed] [--out masks.u64]
    python -m paper_2404_17101_gb300 scc   --input g.adj [--directed] [--out labels.u32]
    python -m paper_2404_17101_gb300 bfs64 --input g.adj [--sources ...] [--out dist.u32]
    python -m paper_2404_17101_gb300 sssp  --input g.adj [--weights w.u32 | --wmax 1000 --wseed 1]
                                           [--source 0] [--delta 0] [--out dist.u64]

`--input` reads the PBBS "AdjacencyGraph" text format, or the GBBS binary
layout when the file name ends in `.bin`; `--workload` takes a
named generator of the graphgen module instead (e.g. knn_10m, grid_1000).
One JSON line with the device time (kernel events), rounds and, for BFS, the
traversed edges and GTEPS is printed; `--out` writes the result as raw
little-endian integers (uint32 distances / labels, uint64 masks: forward, then
backward; bfs64: 64 x n distances, source-major; sssp: uint64 distances).
sssp reads one uint32 weight per arc (CSR order) from --weights, or draws
seeded weights in 1..wmax per undirected edge.  Without --sources, reach
and bfs64 take 64 seeded sources of out-degree > 0.  Needs a CUDA GPU; there
is no CPU fallback.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _args(argv):
    ap = argparse.ArgumentParser(prog="python -m paper_2404_17101_gb300",
                                 description="Exact BFS, reachability and SCC on one GB300.")
    ap.add_argument("op", choices=["bfs", "reach", "scc", "bfs64", "sssp"])
    src = ap.add_mutually_exclusive_group(required=True)
    src.add_argument("--input", help="graph file: PBBS AdjacencyGraph text, or GBBS binary (*.bin)")
    src.add_argument("--workload", help="named graphgen generator, e.g. knn_10m, grid_1000, dgrid_4000")
    ap.add_argument("--directed", action="store_true", help="arcs as given (else the file is symmetric)")
    ap.add_argument("--source", type=int, default=0, help="bfs: source vertex")
    ap.add_argument("--sources", default="", help="reach / bfs64: comma-separated sources (at most 64)")
    ap.add_argument("--backward", action="store_true", help="reach: also the backward masks")
    ap.add_argument("--tau", type=int, default=0, help="VGC hop window (0 = library default)")
    ap.add_argument("--learned", action="store_true", help="bfs: learned per-round schedule")
    ap.add_argument("--no-ell", action="store_true", help="no padded rows (CSR only)")
    ap.add_argument("--weights", help="sssp: raw little-endian uint32 weight per arc (CSR order)")
    ap.add_argument("--wmax", type=int, default=1000, help="sssp: seeded weights in 1..wmax")
    ap.add_argument("--wseed", type=int, default=1, help="sssp: seed of the weights")
    ap.add_argument("--delta", type=int, default=0, help="sssp: step width (0 = automatic)")
    ap.add_argument("--out", help="write the result as raw little-endian integers")
    return ap.parse_args(argv)


def main(argv=None) -> int:
    a = _args(argv)
    import torch
    if not torch.cuda.is_available():
        print("error: needs a CUDA GPU (there is no CPU fallback)", file=sys.stderr)
        return 2
    import graphgen as gg
    import paper_2404_17101_gb300 as pg
    if a.input:
        reader = gg.read_gbbs_bin if a.input.endswith(".bin") else gg.read_adj
        g = reader(a.input, directed=a.directed)
    else:
        if not hasattr(gg, a.workload):
            print(f"error: unknown workload {a.workload!r}", file=sys.stderr)
            return 2
        g = getattr(gg, a.workload)()
    G = pg.Graph.from_graphgen(g, ell=not a.no_ell)
    kw = {"tau": a.tau} if a.tau else {}
    st = pg.Stats()
    rec = {"op": a.op, "graph": g.name, "n": g.n, "m": g.m}
    if a.op == "bfs":
        if a.learned:
            G.set_schedule_weights(pg.trained_weights())
            kw["schedule"] = pg.PG_SCHED_LEARNED
        d = G.bfs(a.source, cfg=pg.default_config(**kw), stats=st)
        n_r, m_r = G.count_reached(d)
        rec.update(source=a.source, reached=n_r, traversed_edges=m_r,
                   gteps=m_r / st.kernel_ms / 1e6 if st.kernel_ms else None)
        out = pg.to_uint32(d)
    elif a.op in ("reach", "bfs64"):
        srcs = np.array([int(x) for x in a.sources.split(",") if x], dtype=np.uint32)
        if len(srcs) == 0:
            srcs = gg.pick_sources(g, min(64, g.n), 3)
    if a.op == "bfs64":
        D = G.bfs_multi(srcs, cfg=pg.default_config(direction=pg.PG_DIR_AUTO, **kw), stats=st)
        out = pg.to_uint32(D).reshape(-1)
        rec.update(sources=len(srcs), pull_rounds=st.pull_rounds)
    elif a.op == "reach":
        direction = pg.PG_FWD | (pg.PG_BWD if a.backward else 0)
        f, b = G.reach_multi(srcs, direction, cfg=pg.default_config(**kw), stats=st)
        out = pg.to_uint64(f) if b is None else np.concatenate([pg.to_uint64(f), pg.to_uint64(b)])
        rec.update(sources=len(srcs))
    elif a.op == "scc":
        lab, it = G.scc(cfg=pg.default_config(**kw), stats=st)
        out = pg.to_uint32(lab)
        rec.update(components=int(len(np.unique(out))), iterations=it)
    elif a.op == "sssp":
        if a.weights:
            w = np.fromfile(a.weights, dtype="<u4")
            if len(w) != g.m:
                print(f"error: {len(w)} weights for {g.m} arcs", file=sys.stderr)
                return 2
        else:
            w = gg.edge_weights(g, 1, a.wmax, a.wseed)
        G.set_weights(w)
        d = G.sssp(a.source, cfg=pg.default_config(delta=a.delta, **kw), stats=st)
        out = pg.to_uint64(d)
        rec.update(source=a.source, reached=int((out != np.uint64(0xFFFFFFFFFFFFFFFF)).sum()),
                   expansions=st.expansions)
    rec.update(ms=st.kernel_ms, rounds=st.rounds)
    if a.out:
        out.astype(out.dtype.newbyteorder("<")).tofile(a.out)
        rec["out"] = a.out
    print(json.dumps(rec))
    G.free()
    return 0


if __name__ == "__main__":
    sys.exit(main())
