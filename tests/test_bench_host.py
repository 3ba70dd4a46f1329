"""CPU tests of the benchmark's host logic: roofline bookkeeping from a profile, the
source-hash gate on committed DRAM counters, the clock-sample parsing, and the JSON
line of the reference arm (the CPU oracle on a bounded sample)."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _prof():
    # two FFT passes and two block kernels; gram has the largest share of time
    return {
        "zin_c64": {"launches": 10, "total_ms": 0.5, "bytes": 1.5e9, "flops": 1e9},
        "xy_c64": {"launches": 10, "total_ms": 0.7, "bytes": 1.9e9, "flops": 2e9},
        "gram_c64": {"launches": 4, "total_ms": 2.0, "bytes": 0.8e9, "flops": 40e9},
        "xy_c128": {"launches": 1, "total_ms": 1.0, "bytes": 0.4e9, "flops": 0.5e9},
    }


def test_kernel_table_orders_by_time_and_shares_sum_to_one():
    t = bench.kernel_table(_prof())
    assert list(t) == ["gram_c64", "xy_c128", "xy_c64", "zin_c64"]
    assert abs(sum(v["share"] for v in t.values()) - 1.0) < 1e-3
    assert t["gram_c64"]["launches"] == 4
    assert abs(t["zin_c64"]["GBps"] - 1.5e9 / 0.5 / 1e6) < 1e-6


def test_bound_of_each_kind(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6746.0, "measured"))
    P = _prof()
    ridge32 = bench.FP32_PEAK_TFLOPS * 1e12 / 6746e9          # about 11.9 flop per byte
    assert bench._bound("zin_c64", P["zin_c64"])[:1] == ("hbm",)
    assert bench._bound("xy_c64", P["xy_c64"])[2] == "GB/s"
    # 50 flop per byte: above the FP32 ridge
    assert bench._bound("gram_c64", P["gram_c64"])[:3] == ("alu", bench.FP32_PEAK_TFLOPS, "TFLOP/s")
    # the same kind below the ridge is HBM bound
    low = {"flops": 0.5 * ridge32 * 1e9, "bytes": 1e9}
    assert bench._bound("gram_c64", low)[:2] == ("hbm", 6746.0)
    # double-float update: 8 flops per complex multiply-add over its bytes, against the FP32 ridge
    df = {"flops": 5.7 * 1e9, "bytes": 1e9}
    assert bench._bound("combine_df_c128", df)[:1] == ("hbm",)
    assert bench._bound("combine_df_c128", {"flops": 2 * ridge32 * 1e9, "bytes": 1e9})[:2] == \
        ("alu", bench.FP32_PEAK_TFLOPS)
    # complex128 FFT pass: above the (low) FP64 ridge
    assert bench._bound("xy_c128", P["xy_c128"])[:2] == ("alu", bench.FP64_PEAK_TFLOPS)
    # 152 SMs x 128 lanes x 2 flops x 2.07 GHz
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.54784)


def test_roofline_takes_dominant_kernel(monkeypatch):
    monkeypatch.setattr(bench, "traffic_for", lambda name, model_bytes=None: None)
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6746.0, "measured"))
    r = bench.roofline(_prof())
    assert r["kernel"] == "gram_c64" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(40e9 / 2.0e-3 / 1e12)          # flops per second
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP32_PEAK_TFLOPS)
    assert r["avg_launch_ms"] == pytest.approx(0.5)
    assert r["share_of_kernel_time"] == pytest.approx(2.0 / 4.2)
    assert bench.roofline({}) is None


def test_apply_roofline_counts_complex64_passes_only(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: (6746.0, "measured"))
    a = bench.apply_roofline(_prof())
    assert a["bound"] == "hbm" and a["peak"] == 6746.0
    assert a["achieved"] == pytest.approx((1.5e9 + 1.9e9) / 1.2e-3 / 1e9)
    assert a["frac"] == pytest.approx(a["achieved"] / 6746.0)


def test_traffic_only_for_matching_sources(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    d = {"source_hash": "abc", "kernels": {"gram_c64": {"dram_bytes_per_launch": 1.25e8},
                                          "xy_c64": {"dram_bytes_per_launch": 1.3e8,
                                                     "model_bytes_per_launch": 2.0e8}}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(d))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.traffic_for("gram_c64") == 1.25e8
    assert bench.traffic_for("zin_c64") is None
    # scaled to the bench's average launch by the ratio of the pass-model bytes
    assert bench.traffic_for("xy_c64", 1.0e8) == pytest.approx(0.65e8)
    assert bench.traffic_for("xy_c64") == 1.3e8
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.traffic_for("gram_c64") is None


def test_kernel_source_hash_covers_device_sources():
    # every source that defines device code (kernels, device functions or device data)
    src = os.path.join(ROOT, "paper_1806_10284_gb300", "csrc")
    device = {f for f in os.listdir(src)
              if "__global__" in open(os.path.join(src, f)).read() or "__device__" in open(os.path.join(src, f)).read()}
    assert device and device <= set(bench.KERNEL_SOURCES), device - set(bench.KERNEL_SOURCES)
    h = bench.kernel_source_hash()
    assert len(h) == 16 and h == bench.kernel_source_hash()


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parsed():
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2062, 2070, 1300.4, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    c = s.stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    s2 = bench.ClockSampler(0)
    assert s2.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] == os.cpu_count() and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
