"""The benchmark's host-side logic on the CPU: the reference arm's JSON line, the workload
description, the roofline traffic lookup (used only while the kernel sources are unchanged) and
the Taylor-Green relaxation time."""
import json
import math
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("D3Q27 CM-LBM F32 decaying Taylor-Green vortex 256^3")


def test_workload_description():
    c = bench.workload_config(256, "f32", 1)
    assert c["cells"] == 256 ** 3 and c["parallelism"] == "single GPU" and ">>" in c["l2"]
    h = bench.workload_config(512, "bf16", 2, "hit")
    assert "forced isotropic turbulence 512^3" in h["workload"] and h["parallelism"] == "replicas"


def test_tgv_relaxation_time_from_reynolds_number():
    # nu = u0 L' / Re with L' = n / (2 pi), tau = 3 nu + 1/2
    assert math.isclose(bench.tgv_tau(256), 3 * 0.05 * (256 / (2 * math.pi)) / 1600 + 0.5)
    assert abs(bench.tgv_tau(256) - 0.503820) < 1e-6


def test_traffic_lookup_needs_the_current_kernel_sources(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    f.write_text(f"# comment\nsource_hash = {bench.kernel_source_hash()}\nk_test = 212.5\n")
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    assert bench.measured_traffic("k_test") == 212.5
    assert bench.measured_traffic("k_missing") is None
    f.write_text("source_hash = 0000000000000000\nk_test = 212.5\n")
    assert bench.measured_traffic("k_test") is None
