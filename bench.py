#!/usr/bin/env python
"""Benchmark: exact BFS throughput (GTEPS) and HBM-roofline fraction on one GB300.

Workload (default): single-source BFS from vertex 0 on the kNN graph of
10,000,000 seeded uniform points in the unit square, k = 5, symmetrised
(59.6M directed CSR arcs) -- the stand-in for the paper's large-diameter kNN
inputs (GL5 / CH5, Table 1).  One step = one pg_bfs call (in-kernel init,
every traversal round, result in HBM).  Two forms are timed on the same
graph: the plain fixed-tau traversal (tau and launch shape from the
autotuner) and the learned per-round schedule (when trained weights exist).

Printed: ONE JSON line (rank 0).  `value` is the headline form's GTEPS
(learned if available, else plain) summed over all ranks (replicas: every
rank runs the same workload on its own GPU, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFS GTEPS and % of HBM roofline, learned/batched vs plain on one GB300, exact dist"
FALLBACK_HBM_GBS = 6800.0
WORKLOADS = {
    # name -> (graphgen factory name, source, description)
    "knn_10m": ("knn_10m", 0, "kNN graph, 10M uniform points in the unit square, k=5, seed 2, "
                              "symmetrised; BFS from vertex 0"),
    "grid_1000": ("grid_1000", 0, "1000x1000 undirected 4-neighbour grid; BFS from vertex 0"),
    "knn_30m_k3": ("knn_30m_k3", 0, "held-out kNN graph, 30M points, k=3, seed 5; BFS from 0"),
    "strip_20m": ("strip_20m", 0, "1 x 20M strip (path); BFS from vertex 0"),
    "strip_200k": ("strip_200k", 0, "1 x 200k strip (path, per-hop latency profile); BFS from vertex 0"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="knn_10m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--configs", action="store_true",
                    help="instead of the headline line: one JSON line per benchmark configuration")
    ap.add_argument("--with-strip", action="store_true", help="--configs: include the 1 x 20M strip")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other configurations' forms (C1, C3, C4, C5) in the headline line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_throughput(local_total_ms, world, units_per_step, steps, dist=None, device=None):
    """Whole-job throughput of N independent replicas (weak scaling): every
    rank ran `steps` steps of `units_per_step` units; the job took as long
    as the slowest rank.  Returns (units per ms summed over ranks, max ms).
    The only collective is this one all-reduce of the timing, outside the
    timed region."""
    import torch
    t = torch.tensor([float(local_total_ms)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tmax = float(t.item())
    return world * units_per_step * steps / tmax, tmax


def algorithmic_bytes(n, n_r, m_r):
    """Bytes an ideal traversal must touch: offsets of reached vertices,
    their adjacency lists, and one write of every distance."""
    return 4 * (n_r + 1) + 4 * m_r + 4 * n


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("pg_traverse.cu", "pg_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2404_17101_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", f"traffic_{workload}.json")
    try:
        with open(p) as f:
            d = json.load(f)
        if d.get("kernel_source_sha256_16") == kernel_source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median SM clock under load, the largest max clock and the throttle
    reasons seen Active, from `nvidia-smi --query-gpu=<ClockSampler.Q>
    --format=csv,noheader,nounits` lines; None when no line parses."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_bfs(g, src, budget_s=12.0):
    """The oracle (serial queue BFS, one core) on the same workload."""
    import oracle
    t0 = time.perf_counter()
    d = oracle.bfs(g, src)
    t1 = time.perf_counter() - t0
    reps = max(1, min(20, int(budget_s / max(t1, 1e-3)) - 1))
    ts = [t1]
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.bfs(g, src)
        ts.append(time.perf_counter() - t0)
    n_r, m_r = oracle.reached_edges(g, d)
    return d, n_r, m_r, ts


def eccentricity(out):
    """Largest finite distance in a device int32 view of uint32 distances."""
    import torch
    d = out.to(torch.int64) & 0xFFFFFFFF
    fin = d[d != 0xFFFFFFFF]
    return int(fin.max().item()) if fin.numel() else 0


def latency_floor(pg, gg, rounds, levels, kernel_ms):
    """The round-latency floor of a traversal with `rounds` rounds over
    `levels` dependent BFS levels: rounds x t_barrier + levels x t_hop.
    t_barrier: an empty persistent loop of grid barriers (pg_probe_barrier);
    t_hop: the per-level cost of a one-vertex-per-level chain, measured as
    a BFS on a 1 x 20,000 strip (tau = 64) minus its barriers."""
    t_bar = pg.probe_barrier(20000)
    strip = gg.strip(20000)
    S = pg.Graph.from_graphgen(strip, ell=True)
    cfg = pg.default_config(tau=64)
    st = pg.Stats()
    for _ in range(2):
        S.bfs(0, cfg=cfg, stats=st)
    ts = []
    for _ in range(3):
        S.bfs(0, cfg=cfg, stats=st)
        ts.append(st.kernel_ms)
    S.free()
    t_hop = (min(ts) * 1e3 - st.rounds * t_bar) / (strip.n - 1)
    floor_ms = (rounds * t_bar + levels * t_hop) / 1e3
    return {"t_barrier_us": t_bar, "t_hop_us": t_hop, "rounds": rounds, "levels": levels,
            "floor_ms": floor_ms, "frac_latency": floor_ms / kernel_ms,
            "how": "t_barrier: pg_probe_barrier, 20000 empty grid barriers of the traversal's "
                   "launch shape; t_hop: BFS on a 1x20000 strip at tau 64, minus its rounds' "
                   "barriers, per level"}


def learned_on(pg, cfg):
    """The learned per-round schedule on top of `cfg`: same launch shape, and
    cfg's tau is the fixed action the network falls back to."""
    c = pg.Config.from_buffer_copy(cfg)
    c.schedule = pg.PG_SCHED_LEARNED
    return c


def other_configs(pg, gg, peak, steps, warm, with_oracle):
    """Timed forms of the other benchmark configurations (one GPU):
    C3 (R-MAT 24, 64 single-source BFS vs one 64-source batch), C4 (directed
    4000^2 grid, 64-source forward + backward reachability batch vs single
    launches, default and autotuned), C1 (grid 1000^2) and C5 (held-out kNN
    30M, k = 3): plain tau = 16 vs the best fixed tau vs the learned
    schedule.  Device times are kernel events (min of `steps` after `warm`
    warm-ups, L2 flushed between runs).  With `with_oracle` the CPU leg runs
    the oracle on a bounded sample (sampled rows / bits) of every form's
    output and reports whether they are equal, and the oracle's time."""
    import numpy as np
    import torch
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")
    w = pg.trained_weights()
    res = {}

    def best(call, reps=steps, wu=warm):
        st = pg.Stats()
        for _ in range(wu):
            call(st)
        ts = []
        for i in range(reps):
            flush.fill_(i)
            call(st)
            ts.append(st.kernel_ms)
        return min(ts), st

    # ---- C3: 64 single-source BFS vs one 64-source batch
    t0 = time.perf_counter()
    g = gg.rmat_24()
    t_gen = time.perf_counter() - t0
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 3)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    c1 = pg.default_config(tau=1, direction=pg.PG_DIR_AUTO)
    single, m_tot, rows = 0.0, 0, {}
    keep = (0, 17)
    for j, s_ in enumerate(srcs):
        ms, _ = best(lambda st: G.bfs(int(s_), out=out, cfg=c1, stats=st), 1, 1 if j == 0 else 0)
        single += ms
        m_tot += G.count_reached(out)[1]
        if j in keep:
            rows[j] = pg.to_uint32(out)
    D = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
    cb = pg.default_config(direction=pg.PG_DIR_AUTO)
    ms_b, st_b = best(lambda st: G.bfs_multi(srcs, cfg=cb, stats=st, out=D))
    B3 = 4 * (g.n + 1) + 4 * g.m + 4 * 64 * g.n
    c3 = {"n": g.n, "m": g.m, "k": 64, "traversed_edges_sum": m_tot, "generate_s": t_gen,
          "single_x64": {"ms": single, "gteps": m_tot / single / 1e6,
                         "form": "64 pg_bfs calls, tau 1, push/pull (Beamer)"},
          "batch64": {"ms": ms_b, "gteps": m_tot / ms_b / 1e6, "rounds": st_b.rounds,
                      "pull_rounds": st_b.pull_rounds,
                      "roofline": {"bound": "hbm", "algorithmic_bytes": B3,
                                   "achieved": B3 / (ms_b * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                                   "frac": B3 / (ms_b * 1e-3) / 1e9 / peak,
                                   "bytes": "4(n+1) + 4m + 4kn"}},
          "batch_speedup": single / ms_b}
    if with_oracle:
        import oracle
        Dh = {j: pg.to_uint32(D[j]) for j in keep}
        t0 = time.perf_counter()
        want = {j: oracle.bfs(g, int(srcs[j])) for j in keep}
        t_or = (time.perf_counter() - t0) / len(keep)
        c3["exact_vs_oracle"] = {
            "rows": list(keep),
            "batch": all(np.array_equal(Dh[j], want[j]) for j in keep),
            "single": all(np.array_equal(rows[j], want[j]) for j in keep)}
        c3["cpu_oracle"] = {"ms": 64 * t_or * 1e3, "gteps": m_tot / (64 * t_or) / 1e9, "cores": 1,
                            "sample": f"{len(keep)} sources timed, times 32"}
    res["C3 rmat_24"] = c3
    del G, D, rows
    torch.cuda.empty_cache()

    # ---- C4: 64-source forward + backward reachability in one launch
    g = gg.dgrid_4000()
    G = pg.Graph.from_graphgen(g, ell=True)
    srcs = gg.pick_sources(g, 64, 4)
    both = pg.PG_FWD | pg.PG_BWD
    ms_d, st_d = best(lambda st: G.reach_multi(srcs, both, cfg=pg.default_config(), stats=st))
    t0 = time.perf_counter()
    tuned = G.autotune(srcs, kind=1, direction=both, trials=2)
    t_tune = time.perf_counter() - t0
    fw_bw = {}

    def run_tuned(st):
        fw_bw["r"] = G.reach_multi(srcs, both, cfg=tuned, stats=st)
    ms_t, st_t = best(run_tuned)
    fw, bw = fw_bw["r"]
    single = 0.0
    for s_ in srcs[:8]:
        ms, _ = best(lambda st: G.reach_multi([int(s_)], both, cfg=pg.default_config(), stats=st), 1, 1)
        single += ms
    single *= 8
    f, b = pg.to_uint64(fw), pg.to_uint64(bw)
    deg = np.diff(g.offsets.astype(np.int64))
    tdeg = np.bincount(g.indices, minlength=g.n).astype(np.int64)
    nr_f, nr_b = int(np.count_nonzero(f)), int(np.count_nonzero(b))
    mr_f, mr_b = int(deg[f != 0].sum()), int(tdeg[b != 0].sum())
    B4 = (4 * (nr_f + 1) + 4 * mr_f + 8 * g.n) + (4 * (nr_b + 1) + 4 * mr_b + 8 * g.n)
    c4 = {"n": g.n, "m": g.m, "k": 64,
          "batch64_default": {"ms": ms_d, "rounds": st_d.rounds},
          "batch64_tuned": {"ms": ms_t, "rounds": st_t.rounds, "tau": int(tuned.tau),
                            "chunk": int(tuned.chunk), "local_queue": int(tuned.local_queue),
                            "cta_queue": int(tuned.cta_queue), "vgc_mode": int(tuned.vgc_mode),
                            "blocks_per_sm": int(tuned.blocks_per_sm), "autotune_s": t_tune,
                            "roofline": {"bound": "hbm", "algorithmic_bytes": B4,
                                         "achieved": B4 / (ms_t * 1e-3) / 1e9, "peak": peak,
                                         "unit": "GB/s", "frac": B4 / (ms_t * 1e-3) / 1e9 / peak,
                                         "bytes": "per direction 4(n_r+1) + 4 m_r + 8n"}},
          "single_x64": {"ms": single, "sample": "8 sources timed, times 8"},
          "batch_speedup": single / ms_t}
    if with_oracle:
        import oracle
        sample = np.array([3, 40], dtype=np.int64)
        t0 = time.perf_counter()
        wf = oracle.reach(g, srcs[sample])
        t_or = (time.perf_counter() - t0) / len(sample)
        wb = oracle.reach(g, srcs[sample], backward=True)
        ok = True
        for i, j in enumerate(sample):
            bit, bi = np.uint64(1) << np.uint64(j), np.uint64(1) << np.uint64(i)
            ok &= bool(np.array_equal((f & bit) != 0, (wf & bi) != 0))
            ok &= bool(np.array_equal((b & bit) != 0, (wb & bi) != 0))
        c4["exact_vs_oracle"] = {"bits": sample.tolist(), "fwd_and_bwd": ok}
        c4["cpu_oracle"] = {"ms": 128 * t_or * 1e3, "cores": 1,
                            "sample": "2 sources, forward, timed; times 128"}
    res["C4 dgrid_4000"] = c4
    del G
    torch.cuda.empty_cache()

    # ---- next row f3: weighted shortest paths on the C2 graph (seeded
    # weights 1..1000 per undirected edge), stepping framework with VGC
    g = gg.knn_10m()
    wts = gg.edge_weights(g, 1, 1000, 2)
    G = pg.Graph.from_graphgen(g)
    G.set_weights(wts)
    dsp = torch.empty(g.n, dtype=torch.int64, device="cuda")
    ms_s, st_s = best(lambda st: G.sssp(0, out=dsp, stats=st))
    Bs = 4 * (g.n + 1) + 8 * g.m + 8 * g.n
    ss = {"n": g.n, "m": g.m, "weights": "seeded uniform 1..1000 per undirected edge",
          "ms": ms_s, "rounds": st_s.rounds, "expansions_per_vertex": st_s.expansions / g.n,
          "gteps": g.m / ms_s / 1e6,
          "roofline": {"bound": "hbm", "algorithmic_bytes": Bs, "achieved": Bs / (ms_s * 1e-3) / 1e9,
                       "peak": peak, "unit": "GB/s", "frac": Bs / (ms_s * 1e-3) / 1e9 / peak,
                       "bytes": "4(n+1) + 4m indices + 4m weights + 8n distances"}}
    if with_oracle:
        import oracle
        t0 = time.perf_counter()
        want = oracle.sssp(g, wts, 0)
        t_or = time.perf_counter() - t0
        ss["exact_vs_oracle"] = bool(np.array_equal(pg.to_uint64(dsp), want))
        ss["cpu_oracle"] = {"ms": t_or * 1e3, "cores": 1, "sample": "full workload, one Dijkstra run"}
    res["f3 sssp knn_10m"] = ss
    del G, dsp, wts
    torch.cuda.empty_cache()

    # ---- C1 and C5 held-out kNN: fixed tau 16 / 32 / 64, the autotuned
    # configuration, and the learned schedule on top of it
    for name, make in (("C1 grid_1000", gg.grid_1000), ("C5 knn_30m_k3", gg.knn_30m_k3)):
        g = make()
        G = pg.Graph.from_graphgen(g, ell=True)
        forms = {"plain_tau16": pg.default_config(), "plain_tau32": pg.default_config(tau=32),
                 "plain_tau64": pg.default_config(tau=64),
                 "plain_tuned": G.autotune([0], kind=0, trials=1, cfg=pg.default_config())}
        if w is not None:
            G.set_schedule_weights(w)
            forms["learned"] = learned_on(pg, forms["plain_tuned"])
        outs, fr = {}, {}
        for f_, cfg in forms.items():
            o = torch.empty(g.n, dtype=torch.int32, device="cuda")
            ms, st = best(lambda st: G.bfs(0, out=o, cfg=cfg, stats=st))
            outs[f_] = o
            fr[f_] = {"ms": ms, "rounds": st.rounds}
        n_r, m_r = G.count_reached(outs["plain_tau16"])
        for f_ in fr:
            fr[f_]["gteps"] = m_r / fr[f_]["ms"] / 1e6
        Bc = algorithmic_bytes(g.n, n_r, m_r)
        entry = {"n": g.n, "m": g.m, "traversed_edges": m_r, "forms": fr,
                 "algorithmic_bytes": Bc}
        if with_oracle:
            import oracle
            t0 = time.perf_counter()
            want = oracle.bfs(g, 0)
            t_or = time.perf_counter() - t0
            entry["exact_vs_oracle"] = {f_: bool(np.array_equal(pg.to_uint32(o), want))
                                        for f_, o in outs.items()}
            entry["cpu_oracle"] = {"ms": t_or * 1e3, "gteps": m_r / t_or / 1e9, "cores": 1,
                                   "sample": "full workload, one run"}
        res[name] = entry
        del G, outs
        torch.cuda.empty_cache()
    return res


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    oracle.build()
    gg.build()
    fac, src, desc = WORKLOADS[args.workload]
    g = getattr(gg, fac)()
    d = oracle.bfs(g, src)
    n_r, m_r = oracle.reached_edges(g, d)
    for _ in range(args.warmup):
        oracle.bfs(g, src)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.bfs(g, src)
        ts.append(time.perf_counter() - t0)
    mean = sum(ts) / len(ts)
    value = m_r / mean / 1e9
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m,
                   "source": src, "reached_vertices": n_r, "traversed_edges": m_r},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"full workload, {args.steps} timed serial queue-BFS runs"},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_configs(args):
    """One JSON line per benchmark configuration (rank 0, one GPU): every
    form's device time (CUDA events, min of `steps` after `warmup`), the
    forms' outputs compared with each other, and the oracle on one host core
    over a bounded sample (the CPU-baseline leg)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import graphgen as gg
    import oracle
    import paper_2404_17101_gb300 as pg
    torch.cuda.set_device(0)
    oracle.build()
    w = pg.trained_weights()
    steps, warm = max(1, args.steps), max(1, args.warmup)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")

    def best(call, reps=steps, wu=warm):
        st = pg.Stats()
        for _ in range(wu):
            call(st)
        ts, res = [], None
        for i in range(reps):
            flush.fill_(i)
            res = call(st)
            ts.append(st.kernel_ms)
        return min(ts), st, res

    def cpu(fn, budget_s=8.0):
        t0 = time.perf_counter(); fn(); t = time.perf_counter() - t0
        reps = max(0, min(4, int(budget_s / max(t, 1e-3)) - 1))
        ts = [t]
        for _ in range(reps):
            t0 = time.perf_counter(); fn(); ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    def emit(d):
        print(json.dumps(d), flush=True)

    def bfs_forms(name, g, extra=None):
        G = pg.Graph.from_graphgen(g, ell=True)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        forms = {"tau16": pg.default_config(), "tau32": pg.default_config(tau=32),
                 "tau64": pg.default_config(tau=64)}
        if not name.startswith("strip"):
            forms["tuned"] = G.autotune([0], kind=0, trials=1, cfg=pg.default_config())
        if w is not None:
            G.set_schedule_weights(w)
            forms["learned"] = learned_on(pg, forms.get("tuned", forms["tau64"]))
        if extra:
            forms.update(extra)
        res, ref = {}, None
        for f, cfg in forms.items():
            cfg.timeout_ms = 30000
            reps, wu = (1, 1) if name.startswith("strip") else (steps, warm)
            ms, st, _ = best(lambda st: G.bfs(0, out=out, cfg=cfg, stats=st), reps, wu)
            d = pg.to_uint32(out)
            same = True if ref is None else bool(np.array_equal(d, ref))
            ref = d if ref is None else ref
            res[f] = {"ms": ms, "rounds": st.rounds, "same_as_first": same}
        n_r, m_r = G.count_reached(out)
        for f in res:
            res[f]["gteps"] = m_r / res[f]["ms"] / 1e6
        t_or = cpu(lambda: oracle.bfs(g, 0))
        emit({"config": name, "kind": "bfs", "n": g.n, "m": g.m, "traversed_edges": m_r, "forms": res,
              "cpu_oracle": {"ms": t_or * 1e3, "gteps": m_r / t_or / 1e9, "cores": 1}})
        G.free()

    bfs_forms("C1 grid_1000", gg.grid_1000())
    bfs_forms("C2 knn_10m", gg.knn_10m())

    # C3: 64 single-source BFS (direction-optimising, plain rounds) vs one batch
    g = gg.rmat_24()
    G = pg.Graph.from_graphgen(g)
    srcs = gg.pick_sources(g, 64, 3)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    c1 = pg.default_config(tau=1, direction=pg.PG_DIR_AUTO)
    single, m_tot = 0.0, 0
    for s_ in srcs:
        ms, _, _ = best(lambda st: G.bfs(int(s_), out=out, cfg=c1, stats=st), 1, 1)
        single += ms
        m_tot += G.count_reached(out)[1]
    D = torch.empty((64, g.n), dtype=torch.int32, device="cuda")
    cb = pg.default_config(direction=pg.PG_DIR_AUTO)
    ms_b, st_b, _ = best(lambda st: G.bfs_multi(srcs, cfg=cb, stats=st, out=D))
    row_ok = bool(np.array_equal(pg.to_uint32(D[17]), pg.to_uint32(G.bfs(int(srcs[17]), cfg=c1))))
    t_or = cpu(lambda: oracle.bfs(g, int(srcs[0])))
    emit({"config": "C3 rmat_24", "kind": "bfs x64", "n": g.n, "m": g.m, "traversed_edges_sum": m_tot,
          "forms": {"single_x64": {"ms": single, "gteps": m_tot / single / 1e6},
                    "batch64": {"ms": ms_b, "gteps": m_tot / ms_b / 1e6, "rounds": st_b.rounds,
                                "pull_rounds": st_b.pull_rounds, "row_equals_single": row_ok}},
          "cpu_oracle": {"ms": 64 * t_or * 1e3, "gteps": m_tot / (64 * t_or) / 1e9, "cores": 1,
                         "sample": "one source timed, times 64"}})
    del G, D
    torch.cuda.empty_cache()

    # C4: 64-source forward + backward reachability in one launch vs 64
    # single-source launches; then SCC of the same graph
    g = gg.dgrid_4000()
    G = pg.Graph.from_graphgen(g, ell=True)
    srcs = gg.pick_sources(g, 64, 4)
    both = pg.PG_FWD | pg.PG_BWD
    ms_d, st_d, _ = best(lambda st: G.reach_multi(srcs, both, cfg=pg.default_config(), stats=st))
    tuned = G.autotune(srcs, kind=1, direction=both, trials=2)
    ms_t, st_t, (fw, bw) = best(lambda st: G.reach_multi(srcs, both, cfg=tuned, stats=st))
    single = 0.0
    for s_ in srcs[:8]:
        ms, _, _ = best(lambda st: G.reach_multi([int(s_)], both, cfg=pg.default_config(), stats=st), 1, 1)
        single += ms
    single *= 8
    ms_s, st_s, (lab, it) = best(lambda st: G.scc(cfg=pg.default_config(tau=64), stats=st))
    ms_s1, _, _ = best(lambda st: G.scc(cfg=pg.default_config(tau=1), stats=st))
    t_or = cpu(lambda: oracle.reach(g, srcs[:1]), budget_s=4.0)
    t_scc = cpu(lambda: oracle.scc(g), budget_s=4.0)
    emit({"config": "C4 dgrid_4000", "kind": "reach fwd+bwd x64, scc", "n": g.n, "m": g.m,
          "forms": {"batch64_default": {"ms": ms_d, "rounds": st_d.rounds},
                    "batch64_tuned": {"ms": ms_t, "rounds": st_t.rounds,
                                      "tau": int(tuned.tau), "chunk": int(tuned.chunk)},
                    "single_x64": {"ms": single, "sample": "8 sources timed, times 8"},
                    "scc_tau64": {"ms": ms_s, "iterations": it, "rounds": st_s.rounds},
                    "scc_tau1": {"ms": ms_s1}},
          "cpu_oracle": {"reach_ms": 128 * t_or * 1e3, "scc_ms": t_scc * 1e3, "cores": 1,
                         "sample": "one source, one direction timed, times 128; Tarjan once"}})
    del G
    torch.cuda.empty_cache()

    bfs_forms("C5 knn_30m_k3", gg.knn_30m_k3())
    if args.with_strip:
        bfs_forms("C5 strip_20m", gg.strip_20m())


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.configs:
        run_configs(args)
        return
    rank, world, local = dist_env()
    import numpy as np
    import torch

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    import graphgen as gg
    import paper_2404_17101_gb300 as pg

    fac, src, desc = WORKLOADS[args.workload]
    g = getattr(gg, fac)()
    G = pg.Graph.from_graphgen(g, ell=True)
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")

    # --- forms: the plain fixed-tau traversal (library defaults), the same
    # with tau and launch shape picked by the autotuner for this graph, and
    # the learned per-round schedule (when trained weights exist) on top of
    # the tuned configuration: the network's fallback action is the tuned tau
    plain_cfg = pg.default_config()
    forms = {"plain": plain_cfg}
    tuned = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        forms["plain_tuned"] = G.autotune([src], kind=0, trials=3, cfg=pg.default_config())
        tuned = time.perf_counter() - t0
    w = pg.trained_weights()
    if w is not None:
        G.set_schedule_weights(w)
        forms["learned"] = learned_on(pg, forms.get("plain_tuned", plain_cfg))

    G.bfs(src, out=out, cfg=plain_cfg)
    n_r, m_r = G.count_reached(out)
    levels = eccentricity(out)
    B = algorithmic_bytes(g.n, n_r, m_r)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device="cuda")  # 256 MB > L2

    def timed(cfg, steps, warmup, sampler=None):
        st = pg.Stats()
        for _ in range(warmup):
            G.bfs(src, out=out, cfg=cfg, stats=st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if sampler:
            sampler.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        kms, rounds, exps = [], [], []
        for i in range(steps):
            flush.fill_(i)                      # L2 flush between steps, outside the events
            ev[i][0].record()
            G.bfs(src, out=out, cfg=cfg, stats=st)
            ev[i][1].record()
            kms.append(st.kernel_ms)
            rounds.append(st.rounds)
            exps.append(st.expansions)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop() if sampler else None
        ms = [a.elapsed_time(b) for a, b in ev]
        _, tmax = replica_throughput(sum(ms), world, 1, 1, dist, device="cuda")
        return {"ms": ms, "total_ms_max": tmax, "kernel_ms": kms,
                "rounds": rounds, "expansions": exps, "clocks": clocks}

    results = {}
    for name, cfg in forms.items():
        sampler = ClockSampler(local) if name == ("learned" if "learned" in forms else "plain") else None
        results[name] = timed(cfg, args.steps, args.warmup, sampler)
    head = "learned" if "learned" in forms else "plain"
    R = results[head]
    ms_per_step = R["total_ms_max"] / args.steps
    value = world * m_r * args.steps / (R["total_ms_max"] * 1e6)  # GTEPS over all replicas
    peak, peak_kind = measured_peak()
    kmean = statistics.mean(R["kernel_ms"])
    achieved = B / (kmean * 1e-3) / 1e9
    traffic = profiled_traffic(args.workload)

    # exactness on this run's output, checked against the oracle in the CPU leg
    cpu = None
    exact = None
    if rank == 0 and not args.no_cpu_baseline:
        d_or, nr_o, mr_o, ts = cpu_baseline_bfs(g, src)
        exact = bool(np.array_equal(pg.to_uint32(out), d_or))
        med = statistics.median(ts)
        cpu = {"value": mr_o / med / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"full workload (n={g.n}, m={g.m}), {len(ts)} serial queue-BFS runs, "
                         f"median {med*1e3:.1f} ms"}

    # end to end through the C ABI with host buffers: upload from pinned host
    # memory, BFS, distances back into pinned host memory, free
    e2e = None
    if not args.no_e2e:
        off_h = torch.from_numpy(g.offsets.view(np.int32)).pin_memory()
        idx_h = torch.from_numpy(g.indices.view(np.int32)).pin_memory()
        dist_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
        lib = pg.load()
        import ctypes
        cfg = forms[head]
        ts = []
        nsteps = max(1, min(args.steps, 5))
        for i in range(nsteps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = ctypes.c_void_p()
            pg._check(lib.pg_graph_upload(ctypes.c_void_p(off_h.data_ptr()),
                                          ctypes.c_void_p(idx_h.data_ptr()), g.n, g.m, pg.PG_ELL,
                                          pg._stream_ptr(), ctypes.byref(h)))
            if head == "learned":
                pg._check(lib.pg_set_schedule_weights(h, ctypes.c_void_p(w.ctypes.data), w.size))
            pg._check(lib.pg_bfs(h, src, ctypes.c_void_p(dist_h.data_ptr()), ctypes.byref(cfg), None,
                                 pg._stream_ptr()))
            pg._check(lib.pg_graph_free(h))
            t1 = time.perf_counter()
            if i > 0:
                ts.append(t1 - t0)
        emean = sum(ts) / len(ts)
        e2e = {"value": world * m_r / emean / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": 4 * (g.n + 1) + 4 * g.m,
               "d2h_bytes_per_step": 4 * g.n, "steps": nsteps,
               "ms_per_step": emean * 1e3}

    floor = latency_floor(pg, gg, int(round(statistics.mean(R["rounds"]))), levels, kmean)
    extra = None
    if world == 1 and not args.no_extra:
        extra = other_configs(pg, gg, peak, steps=3, warm=2, with_oracle=not args.no_cpu_baseline)

    if rank == 0:
        def summary(r):
            return {"gteps": m_r * len(r["ms"]) / (sum(r["ms"]) * 1e6),
                    "ms_per_step": sum(r["ms"]) / len(r["ms"]),
                    "kernel_ms_mean": statistics.mean(r["kernel_ms"]),
                    "rounds_mean": statistics.mean(r["rounds"]),
                    "expansions_per_reached": statistics.mean(r["expansions"]) / max(n_r, 1)}
        cfgd = lambda c: {f: int(getattr(c, f)) for f in ("schedule", "tau", "chunk", "local_queue",
                                                          "threads_per_block", "blocks_per_sm")}
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": g.n, "m": g.m,
                       "source": src, "reached_vertices": n_r, "traversed_edges": m_r,
                       "headline_form": head, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}", "forms": {k: cfgd(c) for k, c in forms.items()},
                       "autotune_s": tuned},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": "pg_traverse_kernel<BFS>", "algorithmic_bytes": B,
                         "kernel_ms_mean": kmean, "latency_floor": floor},
            "gteps_graph500": value / 2,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": R["clocks"],
            "exact_vs_oracle": exact,
            "forms": {k: summary(v) for k, v in results.items()},
            "other_configs": extra,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
