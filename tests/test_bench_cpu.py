"""Host logic of bench.py (no GPU): the clock and throttle-reason summary
taken from nvidia-smi samples, the source hash that keeps ncu counters from
outliving the kernel they were taken on, and the JSON line of the reference
arm (the FP64 oracle timed on the host cores)."""
import json
import os
import shutil
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def test_clock_summary_median_max_and_reasons(monkeypatch):
    rows = [
        "0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1385.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbled line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeProc("\n".join(rows)))
    s = bench.ClockSampler(0)
    s.start()
    r = s.stop()
    assert r["sm_mhz"] == 2010.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    rows[0] = rows[0].replace("Not Active, Not Active, Not Active, Not Active",
                              "Not Active, Active, Not Active, Not Active")
    monkeypatch.setattr(bench.subprocess, "Popen", lambda *a, **k: _FakeProc("\n".join(rows)))
    s.start()
    assert s.stop()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_nvidia_smi(monkeypatch):
    def boom(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(bench.subprocess, "Popen", boom)
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}


def _tree(tmp_path):
    src = os.path.join(ROOT, "paper_1210_1833_gb300", "csrc")
    dst = tmp_path / "paper_1210_1833_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "*.o", "__pycache__"))
    return dst


def test_kernel_hash_follows_code_not_comments(tmp_path, monkeypatch):
    dst = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._kernel_hash()
    p = dst / "plan.cpp"
    src = p.read_text()
    p.write_text("// a new comment line\n" + src.replace("\n", "\n\n", 3) + "/* trailing */\n")
    assert bench._kernel_hash() == h0
    p.write_text(src.replace("1.0001", "1.0002", 1))
    assert bench._kernel_hash() != h0


def test_counters_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    dst = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"kernel_source_hash": bench._kernel_hash(), "per_launch_bytes": 123,
                 "fp32_ops_per_candidate": 10.0, "summary": "x.md"}}
    (tmp_path / "profiles" / "counters.json").write_text(json.dumps(rec))
    assert bench.traffic_record("k") == 123
    c = bench.counted_record("k", 1e12, 40.0)
    assert c["i_pair"] == 10.0 and c["frac"] == pytest.approx(0.25)
    p = dst / "count_kernel.cuh"
    p.write_text(p.read_text() + "\nstatic const int kChanged = 1;\n")
    assert bench.traffic_record("k") is None and bench.counted_record("k", 1e12, 40.0) is None


def test_recheck_fractions():
    st = {"candidate_pairs": 4000, "rechecked_pairs": 40, "fp64_pairs": 2}
    assert bench._recheck(st) == {"rechecked_fraction": 0.01, "fp64_fraction": 0.0005}
    assert bench._recheck({"candidate_pairs": 0, "rechecked_pairs": 0, "fp64_pairs": 0}) == {
        "rechecked_fraction": 0.0, "fp64_fraction": 0.0}


def test_a_failing_row_does_not_lose_the_others(monkeypatch):
    class _Torch:
        class cuda:
            @staticmethod
            def current_stream(dev):
                return None
    monkeypatch.setitem(sys.modules, "torch", _Torch)

    def row(name):
        return lambda ctx, dev, timed: {name: {"ok": True}}

    def boom(ctx, dev, timed):
        raise RuntimeError("no device")
    for n in ("batched", "monopole", "density", "pixel", "angular"):
        monkeypatch.setattr(bench, "_row_" + n, row(n))
    monkeypatch.setattr(bench, "_row_weighted", boom)
    out = bench.run_extras(None, 0)
    assert set(out) == {"batched", "weighted", "monopole", "density", "pixel", "angular"}
    assert out["weighted"] == {"error": "RuntimeError: no device"}
    assert bench.run_extras(None, 0, which="angular") == {"angular": {"ok": True}}
    assert bench.run_extras(None, 0, which="pixel") == {"pixel": {"ok": True}}


def test_total_pairs_closed_form():
    assert bench.total_pairs(4, 3) == 6 + 12 + 3
    assert bench.total_pairs(500000, 2000000) == (
        500000 * 499999 // 2 + 500000 * 2000000 + 2000000 * 1999999 // 2)


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "randoms" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] == "c2_rmu_lightcone"
