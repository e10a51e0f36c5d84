"""Host logic of bench.py (no GPU): the defaults keep every timed chunk a graph replay and
the reductions on chunk boundaries, the algorithmic bytes per update are one read and one
write of the stored value plus the local-energy read and write per cell, and the reference
arm (the oracle on the host) prints the native arm's workload config with the bench line's
keys."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(monkeypatch):
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_defaults_keep_chunks_whole(bench):
    a = bench.parse()
    assert a.graph > 0 and a.graph % 6 == 0          # energy-plane roles return every 6
    assert a.reduce_every % a.graph == 0             # reductions fall between replays
    assert a.profile_every >= 1 and a.graph % a.profile_every == 0
    assert a.gpus == 1 and a.warmup >= 3


def test_algorithmic_bytes(bench):
    # 8 B (float32) or 4 B (bfloat16) per site-direction plus 8 B per cell over Q
    assert bench.bytes_per_update("fp32", 64) == 8.125
    assert bench.bytes_per_update("bf16", 128) == 4.0625


@pytest.mark.parametrize("workload", ["pulses", "film"])
def test_reference_arm_line(bench, workload):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", workload, "--nx", "64", "--q", "16", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, cwd=ROOT,
                         timeout=600, check=True)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    a = bench.parse()
    a.workload, a.nx, a.q = workload, 64, 16
    want = dict(bench.workload_config(a, bench.workload(a)), parallelism="replicas x1")
    assert line["config"] == json.loads(json.dumps(want))


def test_cpu_baseline_one_thread_and_all_cores(bench):
    """The host baseline reports the oracle on one thread and on one spawned process per
    core, the core count and the CPU model."""
    import workloads as W
    cfg = W.pulses_c2(seed=2, n=48, q=16, npulse=2)
    cb = bench.cpu_baseline(cfg, seconds=0.3, window=32)
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] > 0 and cb["value_one_thread"] > 0
    assert "cpu_model" in cb and "32x32" in cb["sample"]
