"""The benchmark's host-side parts on the CPU.

* the reference arm (`bench.py --impl reference`, the FP64 oracle on all
  host threads, on a bounded sample of the config-2 recipe) prints one line
  carrying the keys
  the benchmark contract names, with one value in value, cpu_baseline and
  e2e;
* the recorded ncu DRAM traffic of the fused push is reported only while the
  kernel sources hash to the recorded digest, and is null once they change.
"""
import hashlib
import json
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300, check=True)
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["metric"] == "particle-steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    import bench
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == bench.host_threads()
    assert abs(d["ms_per_step"] - 1e3 * (1 << 20) / d["value"]) <= 1e-6 * d["ms_per_step"]


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "push_fixed_traffic.json")))
    for f in rec["source_files"] + ["profiles/push_fixed_traffic.json"]:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, f), dst)
    # the digest of the copied sources, so the check does not depend on the
    # committed record being current
    m = hashlib.sha256()
    for f in rec["source_files"]:
        m.update((tmp_path / f).read_bytes())
    rec["source_sha256"] = m.hexdigest()
    (tmp_path / "profiles" / "push_fixed_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    first = rec["launches"][0]
    assert bench.recorded_traffic() == first["bytes_per_launch_c2"]
    assert bench.recorded_traffic(first["variant"], first["unroll"]) == first["bytes_per_launch_c2"]
    assert bench.recorded_traffic(1, 1) is None               # no capture of that shape
    with open(tmp_path / rec["source_files"][0], "a") as fh:
        fh.write("\n// changed\n")
    assert bench.recorded_traffic() is None
