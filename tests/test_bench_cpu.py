"""bench.py on the CPU: the reference arm's JSON line (the FP64 oracle timed
on a bounded sample), and the helpers behind the GPU line's roofline object
(algorithmic flops from the work counters; the DRAM traffic record, used only
while the pair-kernel sources are the ones it was captured on)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in j, k
    assert j["steps"] == 2 and j["warmup"] == 3 and j["n_gpus"] == 1
    assert j["value"] > 0 and j["higher_is_better"] is True
    assert j["config"]["workload"].startswith("batched")
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"]
    assert cb["unit"] == j["unit"] and cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_algorithmic_flops():
    counts = np.zeros(20, np.int64)
    for k in bench.FLOPS_PER_PATH:
        counts[k] = 10 + k
    want = sum(bench.FLOPS_PER_PATH[k] * (10 + k) for k in bench.FLOPS_PER_PATH)
    counts[15] = 7
    assert bench.algorithmic_flops(counts, False, split=False) == want
    assert bench.algorithmic_flops(counts, True, split=False) == \
        want + (bench.TWO_SUM_EXTRA + bench.REFINE_PER_TERM) * counts[2]
    assert bench.algorithmic_flops(counts, False) == want + bench.SPLIT_EXPAND * 7


def test_traffic_record_follows_the_source():
    rec = json.load(open(os.path.join(ROOT, "profiles", "pair_kernel_traffic.json")))
    entry = rec["batched/fp32c"]
    assert entry["bytes_per_launch"] == entry["dram_read_bytes"] + entry["dram_write_bytes"]
    got = bench.ncu_traffic("batched", "fp32c")
    if entry["source_hash"] == bench.pair_source_hash():
        assert got == entry["bytes_per_launch"]
    else:
        assert got is None
    # any other workload or precision has no record
    assert bench.ncu_traffic("cubes", "fp32c") is None
    assert bench.ncu_traffic("batched", "fp64") is None


def test_reduce_over_ranks_single():
    assert bench.reduce_over_ranks(None, 12.5, 1000, "cpu") == (12.5, 1000)


@pytest.mark.parametrize("flag", ["--energy-drift", "--workload", "--decomp"])
def test_cli_flags_exist(flag):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r.returncode == 0 and flag in r.stdout


def test_options_parse(monkeypatch):
    """The bench's options for profiling and for the library's parameters:
    the defaults keep the driver's contract (N = 1, autotuned execution), and
    --set takes NAME=VALUE pairs that main() hands to dem_set_param."""
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.execution == "auto" and a.set == [] and a.profile_evals == 0
    monkeypatch.setattr(sys, "argv", ["bench.py", "--execution", "graph", "--set", "split_slice=131072",
                                      "--set", "skin=0.3", "--profile-evals", "2"])
    a = bench.parse()
    assert a.execution == "graph" and a.profile_evals == 2
    assert [kv.split("=", 1) for kv in a.set] == [["split_slice", "131072"], ["skin", "0.3"]]
    monkeypatch.setattr(sys, "argv", ["bench.py", "--execution", "fast"])
    with pytest.raises(SystemExit):
        bench.parse()
