"""Host logic of bench.py (CPU): the roofline's byte counts, the lookup of
the committed ncu traffic by kernel-source hash, the peak bandwidth's
fallback, the clock-record parsing, and the reference arm (the FP64 oracle
on the host cores) on a tiny box, including its rank-0-only rule."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_method_and_layout_bytes():
    # the method's bytes per cell and step: populations (or C and deviations)
    # read and written once, plus the link mask and relaxation rate
    assert bench.bytes_per_cell("fp16dev") == 38  # 2 * (4 + 6 * 2) + 2 + 4
    assert bench.bytes_per_cell("fp32") == 62     # 2 * 7 * 4 + 2 + 4
    assert bench.bytes_per_cell("fp32pop") == 62
    assert bench.bytes_per_cell("fp16dev", "d3q19") == 88   # 2 * (4 + 18 * 2) + 8
    assert bench.bytes_per_cell("fp32", "d3q19") == 160     # 2 * 19 * 4 + 8
    assert bench.bytes_per_cell("fp32pop", "d3q19") == 160
    # what the layouts move: C as a double-float (FP16 low word, or a second f32)
    assert bench.layout_bytes_per_cell("fp16dev") == 42
    assert bench.layout_bytes_per_cell("fp32") == 70
    assert bench.layout_bytes_per_cell("fp32pop") == 62
    assert bench.layout_bytes_per_cell("fp16dev", "d3q19") == 96
    assert bench.layout_bytes_per_cell("fp32", "d3q19") == 168


def test_traffic_lookup_by_source_hash(tmp_path, monkeypatch):
    sha = bench.kernel_src_sha256(bench.KERNEL_SRCS)
    rec = {"fp16dev": {"dram_bytes_per_cell": 39.0, "case": "a capture", "src_sha256": sha},
           "fp32": {"dram_bytes_per_cell": 62.0, "case": "an older capture", "src_sha256": "0" * 64}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(p))
    assert bench.measured_traffic("fp16dev", 1000) == (39.0 * 1000, "a capture")
    assert bench.measured_traffic("fp32", 1000) == (None, "kernel changed since the capture")
    assert bench.measured_traffic("fp32pop", 1000) == (None, "no capture")
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(tmp_path / "missing.json"))
    assert bench.measured_traffic("fp16dev", 1000) == (None, "no capture")


def test_source_hash_covers_the_kernel_files(tmp_path):
    a, b = tmp_path / "a.cu", tmp_path / "b.cuh"
    a.write_text("kernel A")
    b.write_text("header B")
    h1 = bench.kernel_src_sha256([str(a), str(b)])
    b.write_text("header B changed")
    h2 = bench.kernel_src_sha256([str(a), str(b)])
    assert h2 != h1
    # comments and layout are not the kernel: editing them keeps the key
    b.write_text("header   B /* a note */ changed // another note\n")
    assert bench.kernel_src_sha256([str(a), str(b)]) == h2
    a.write_text("kernel A // x\n/* y\n z */")
    assert bench.kernel_src_sha256([str(a), str(b)]) == h2


def test_peak_bandwidth_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak_gbs() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6685.8, "bf16_tflops": 1900.0}))
    assert bench.measured_peak_gbs() == (6685.8, "measured")


def test_clock_record_parsing():
    c = bench.ClockSampler(0)
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
    c.lines = ["2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
               "2070, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
               "garbled line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append("1500, 2070, 800.0, 0x8, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]


def _reference(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    env.setdefault("OMP_NUM_THREADS", "2")
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--shape", "6", "8", "16",
                           "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_reference_arm_line():
    r = _reference()
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "MLUPS (D3Q7 fused collide-stream step, all box cells)"
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["shape_zyx"] == [6, 8, 16]


def test_reference_arm_other_ranks_exit_quietly():
    r = _reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_warmup_floor():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "--warmup must be >= 3" in r.stderr
