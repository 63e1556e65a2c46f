"""bench.py's host-side pieces, on the CPU: the reference arm's JSON line (the
oracle timed on the host cores) and the lookup of a kernel's recorded DRAM
traffic, which must fall back to null once the kernel's source changes."""
import hashlib
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900, check=True)
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("c3_sphere_m5")


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    src = tmp_path / "paper_1503_00707_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "k_x.cu").write_text("kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    rec = {"k_x_case": {"bytes_per_launch": 123.0, "source_sha": sha}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._profiled_traffic("k_x.cu", "k_x_case") == 123.0
    assert bench._profiled_traffic("k_x.cu", "another_case") is None
    (src / "k_x.cu").write_text("kernel v2\n")
    assert bench._profiled_traffic("k_x.cu", "k_x_case") is None

