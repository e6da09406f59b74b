"""Host logic of bench.py that needs no GPU: the clock record parsed from
nvidia-smi's CSV lines, the roofline's peak taken from the measured-peaks
file (with its fallback), and the DRAM traffic figure taken from the ncu
summary only while the summary's recorded kernel-source hash matches."""
import hashlib
import json

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _Thread:
    def join(self, timeout=None):
        pass


def test_clock_record_median_max_and_reasons():
    cs = bench.ClockSampler(0)
    cs.proc, cs.t = _Proc(), _Thread()
    cs.lines = [
        "0, 1800, 2070, 1100.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1900, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1700, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = cs.stop()
    assert rec == {"sm_mhz": 1800.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}


def test_clock_record_flags_thermal_slowdown():
    cs = bench.ClockSampler(0)
    cs.proc, cs.t = _Proc(), _Thread()
    cs.lines = ["0, 1500, 2070, 900, 0x40, Active, Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_record_absent_without_samples():
    cs = bench.ClockSampler(0)
    assert cs.stop() is None          # never started
    cs.proc, cs.t = _Proc(), _Thread()
    assert cs.stop() is None          # started, no parsable line


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak()[1].startswith("fallback")
    burst, sus, prov = bench.measured_peaks()
    assert (burst, sus, prov["file"]) == (1900.0, 1700.0, None)
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"bf16_tflops": 1872.8, "bf16_tflops_sustained": 1661.8, "hbm_gbs": 6788.3, "sm_max_mhz": 2070.0}))
    assert bench.measured_peak() == (1661.8, "measured bf16 cuBLAS, sustained")
    burst, sus, prov = bench.measured_peaks()
    assert (burst, sus, prov["file"], prov["sm_max_mhz"]) == (1872.8, 1661.8, "MEASURED_PEAKS.json", 2070.0)


def test_traffic_only_while_the_kernel_is_unchanged(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()
    summary = tmp_path / "summary.md"
    summary.write_text("kernel_source_sha256: %s\ndram_bytes_per_launch_full_size: 1.5e10\n" % h)
    monkeypatch.setattr(bench, "KERNEL_SOURCE", str(src))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(summary))
    assert bench.ncu_traffic() == 1.5e10
    src.write_text("// kernel v2\n")
    assert bench.ncu_traffic() is None
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(tmp_path / "missing.md"))
    assert bench.ncu_traffic() is None
