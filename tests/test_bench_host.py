"""The bench's host-side logic, without a GPU: the reference arm (the CPU
oracle) prints the one JSON line of the bench contract, both arms describe
the same workload, and the DRAM traffic records are used only while the
kernel source they were taken on is unchanged."""
import argparse
import hashlib
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--size", "32", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "DOF/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["dofs"] == 31 * 31


def test_both_arms_share_the_workload_description():
    a = argparse.Namespace(size=1024, rho=3.0, contrast=1e4, level_tol=0.05, refine_tol=1e-9)
    c = bench.bench_config(a, 1046529)
    assert c["dofs"] == 1046529 and "1024x1024" in c["workload"]
    assert c == bench.bench_config(a, 1046529)


def test_traffic_records_follow_the_kernel_source(tmp_path, monkeypatch):
    recs = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    name, rec = next(iter(recs.items()))
    src = os.path.join(ROOT, rec["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if sha != rec["source_sha"]:
        pytest.skip("the committed record predates the current source")
    # a copy of the tree holding the record and its source
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / os.path.dirname(rec["source"]))
    shutil.copy(src, tmp_path / rec["source"])
    json.dump({name: rec}, open(tmp_path / "profiles" / "ncu_traffic.json", "w"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    mixed = rec.get("precision", "f32") == "f32"
    assert bench.ncu_traffic(name, mixed) == rec["bytes_per_launch"]
    assert bench.ncu_traffic(name, not mixed) is None     # the other precision
    with open(tmp_path / rec["source"], "a") as f:        # the kernel source changes
        f.write("\n// edited\n")
    assert bench.ncu_traffic(name, mixed) is None
