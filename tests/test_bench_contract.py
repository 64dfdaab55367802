"""bench.py's JSON-line contract, checked on the CPU through its reference arm
(the FP64 oracle timed on the host cores): one line carrying every key of
the contract, the same workload string as the GPU arm, zero copy bytes, and
the replica helpers' whole-job arithmetic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from workload.standin import spec_for  # noqa: E402


def _reference_line(cfg):
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", cfg, "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_reference_arm_line_c0():
    d = _reference_line("C0")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC
    assert d["unit"] == "evals/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    # the same workload string as the GPU arm prints for this configuration
    assert d["config"]["workload"] == bench.workload_name(spec_for("C0"))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    # value is queries per second of the timed steps
    n = int(cb["sample"].split()[0])
    assert abs(d["value"] - n / (d["ms_per_step"] / 1e3)) <= 1e-3 * d["value"] + 1.0


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--config", "C0", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]


def test_workload_names_carry_the_sizes():
    c4 = bench.workload_name(spec_for("C4"))
    assert c4.startswith("C4:")
    for part in ("1 det x 4 modes", "N=8000+5", "rank 80", "M=2048", "K=656", "Q=1000000"):
        assert part in c4, (part, c4)
    c1 = bench.workload_name(spec_for("C1"))
    for part in ("3 det x 4 modes", "N=1500+5", "rank 20", "M=512", "K=528", "Q=65536"):
        assert part in c1, (part, c1)


def test_job_rate_is_all_ranks_units_over_the_slowest_rank():
    assert bench._job_rate(1000, 1, 2.0) == 500000.0
    assert bench._job_rate(1000, 4, 2.0) == 2000000.0
    assert bench._rank_seed(4000, 0) != bench._rank_seed(4000, 1)
    # one process, no process group: the max over ranks is the value itself
    assert bench._max_over_ranks(3.25) == 3.25
