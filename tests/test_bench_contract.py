"""bench.py's reference arm (the oracle, timed on the host) prints one JSON line
with the keys the benchmark contract requires (no GPU needed)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "grid_1000",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "GTEPS" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["config"]["workload"] == "grid_1000"


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_reads_nvidia_smi_lines():
    """The clocks record that decides whether a run is kept: median SM clock,
    the largest max clock, and only the reasons reported Active."""
    b = _bench()
    row = "0, {sm}, 2070, 900.5, 0x{mask}, {hw}, Not Active, Not Active, {pc}"
    lines = [row.format(sm=2070, mask="0", hw="Not Active", pc="Not Active"),
             row.format(sm=1980, mask="4", hw="Not Active", pc="Active"),
             row.format(sm=2055, mask="0", hw="Not Active", pc="Not Active"),
             "0, [N/A], 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active",
             "short line"]
    c = b.summarise_clocks(lines)
    assert c["sm_mhz"] == 2055 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    lines.append(row.format(sm=1500, mask="8", hw="Active", pc="Not Active"))
    assert b.summarise_clocks(lines)["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert b.summarise_clocks(["garbage"]) is None


def test_algorithmic_bytes_of_one_bfs():
    """4 (n_r + 1) offsets + 4 m_r indices + 4 n distance writes, on the C2
    numbers quoted beside the headline (n = 10^7, n_r = 9,999,609, m_r =
    59,569,914)."""
    b = _bench()
    assert b.algorithmic_bytes(10_000_000, 9_999_609, 59_569_914) == 318_278_096


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs and prints the reference arm; another
    rank exits 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2",
                        "--workload", "grid_1000", "--steps", "2", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr
    assert not [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
