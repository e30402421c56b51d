"""Host logic of bench.py (no GPU).

* The reference arm times the FP64 oracle on the host cores and prints the
  benchmark's JSON line with the arm's own fields; ranks other than 0 print
  nothing.
* The roofline's DRAM-traffic figure comes from a record in profiles/ that is
  tied to a hash of the line-kernel sources: a record is used only while the
  sources it was measured on are unchanged.
"""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run_reference(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_json_line():
    out = _run_reference()
    lines = [ln for ln in out.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "Gunknowns/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"] == bench.CONFIG
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    assert _run_reference({"RANK": "1", "WORLD_SIZE": "2"}).strip() == ""


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    for rel in bench.KERNEL_SOURCES:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, rel), dst)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_traffic_record_used_only_for_its_sources(fake_root):
    h = bench.kernel_source_hash()
    (fake_root / "profiles" / "k.md").write_text(
        "# summary\n\ntraffic-record: kernel=line_kernel_refine_yz size=512 source=%s bytes=2143441000\n"
        "traffic-record: kernel=line_kernel_refine_yz size=256 source=%s bytes=268000000\n" % (h, h))
    assert bench.traffic_record("line_kernel_refine_yz", 512) == 2143441000.0
    assert bench.traffic_record("line_kernel_refine_yz", 256) == 268000000.0
    assert bench.traffic_record("line_kernel_refine_yz", 128) is None
    assert bench.traffic_record("other_kernel", 512) is None
    # any change to a line-kernel source makes the record stale
    src = fake_root / bench.KERNEL_SOURCES[0]
    src.write_text(src.read_text() + "\n")
    assert bench.kernel_source_hash() != h
    assert bench.traffic_record("line_kernel_refine_yz", 512) is None


def test_traffic_record_absent_profiles(fake_root):
    shutil.rmtree(fake_root / "profiles")
    assert bench.traffic_record("line_kernel_refine_yz", 512) is None
