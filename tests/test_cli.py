"""The command line (python -m paper_2404_17101_gb300): argument handling on
the CPU, and BFS / reachability / SCC on a PBBS adjacency file against the
oracle on the GPU."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import graphgen as gg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args):
    return subprocess.run([sys.executable, "-m", "paper_2404_17101_gb300", *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=600)


def test_help_and_bad_arguments():
    r = _run(["--help"])
    assert r.returncode == 0 and "bfs" in r.stdout and "scc" in r.stdout
    r = _run(["bfs"])                      # neither --input nor --workload
    assert r.returncode == 2
    r = _run(["walk", "--workload", "grid_1000"])
    assert r.returncode == 2


@pytest.mark.gpu
def test_bfs_reach_scc_on_a_file(tmp_path):
    g = gg.dgrid(50, 60, 3, shortcuts=6)
    p = str(tmp_path / "g.adj")
    gg.write_adj(g, p)
    out = str(tmp_path / "d.u32")
    r = _run(["bfs", "--input", p, "--directed", "--source", "7", "--out", out])
    assert r.returncode == 0, r.stderr
    rec = json.loads(r.stdout.strip().splitlines()[-1])
    want = oracle.bfs(g, 7)
    assert np.array_equal(np.fromfile(out, dtype="<u4"), want)
    assert rec["reached"] == int((want != oracle.INF).sum())
    out = str(tmp_path / "m.u64")
    r = _run(["reach", "--input", p, "--directed", "--sources", "0,9,100", "--backward", "--out", out])
    assert r.returncode == 0, r.stderr
    m = np.fromfile(out, dtype="<u8")
    srcs = np.array([0, 9, 100], dtype=np.uint32)
    assert np.array_equal(m[:g.n], oracle.reach(g, srcs))
    assert np.array_equal(m[g.n:], oracle.reach(g, srcs, backward=True))
    out = str(tmp_path / "l.u32")
    r = _run(["scc", "--input", p, "--directed", "--out", out])
    assert r.returncode == 0, r.stderr
    assert np.array_equal(np.fromfile(out, dtype="<u4"), oracle.scc(g))
    out = str(tmp_path / "D.u32")
    r = _run(["bfs64", "--input", p, "--directed", "--sources", "3,77,1000", "--out", out])
    assert r.returncode == 0, r.stderr
    D = np.fromfile(out, dtype="<u4").reshape(3, g.n)
    assert np.array_equal(D, oracle.bfs_multi(g, np.array([3, 77, 1000], dtype=np.uint32)))


@pytest.mark.gpu
def test_bfs_on_a_gbbs_binary_file(tmp_path):
    """The same command line on a GBBS binary file (*.bin) against the oracle."""
    g = gg.dgrid(40, 70, 8, shortcuts=4)
    p = str(tmp_path / "g.bin")
    gg.write_gbbs_bin(g, p)
    out = str(tmp_path / "d.u32")
    r = _run(["bfs", "--input", p, "--directed", "--source", "11", "--out", out])
    assert r.returncode == 0, r.stderr
    assert np.array_equal(np.fromfile(out, dtype="<u4"), oracle.bfs(g, 11))


@pytest.mark.gpu
def test_sssp_from_the_command_line(tmp_path):
    """sssp with a weight file and with seeded weights, against Dijkstra."""
    g = gg.knn(20_000, 4, 6)
    p = str(tmp_path / "g.bin")
    gg.write_gbbs_bin(g, p)
    w = gg.edge_weights(g, 1, 50, 3)
    wp = str(tmp_path / "w.u32")
    w.astype("<u4").tofile(wp)
    out = str(tmp_path / "d.u64")
    r = _run(["sssp", "--input", p, "--weights", wp, "--source", "9", "--out", out])
    assert r.returncode == 0, r.stderr
    assert np.array_equal(np.fromfile(out, dtype="<u8"), oracle.sssp(g, w, 9))
    r = _run(["sssp", "--input", p, "--wmax", "700", "--wseed", "5", "--out", out])
    assert r.returncode == 0, r.stderr
    assert np.array_equal(np.fromfile(out, dtype="<u8"), oracle.sssp(g, gg.edge_weights(g, 1, 700, 5), 0))
