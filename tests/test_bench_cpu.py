"""Host-side helpers of bench.py (no GPU): the clock record taken during the
timed region, the DRAM traffic figure tied to the kernel sources it was
measured on, and the operation counts behind the tensor and FP32 figures."""
import os
import time

import pytest

import bench


class _FakeSmi:
    """Stands in for the background nvidia-smi process: terminate() and
    communicate() return canned CSV rows."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def kill(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _row(ts, sm, reasons=("Not Active",) * 4, uuid="GPU-abc"):
    stamp = time.strftime("%Y/%m/%d %H:%M:%S", time.localtime(ts)) + ".%03d" % int((ts % 1) * 1000)
    return ", ".join([stamp, uuid, str(sm), "2070", "900.00 W", "0x0"] + list(reasons))


def _sampler(rows, windows, uuid=None):
    c = bench.ClockSampler(uuid)
    c.proc = _FakeSmi("\n".join(rows) + "\n")
    for w in windows:
        c.mark(*w)
    return c.stop()


def test_clock_record_takes_the_timed_region():
    t0 = time.time() - 100
    rows = [_row(t0 + 0.2 * i, 1000 if i < 10 else 2070) for i in range(30)]   # slow before the window
    rec = _sampler(rows, [(t0 + 2.0, t0 + 5.8)])
    assert rec["window"] == "timed region" and rec["samples"] == 20
    assert rec["sm_mhz"] == 2070 and rec["sm_max_mhz"] == 2070 and rec["reasons"] == []


def test_clock_record_names_active_throttle_reasons():
    t0 = time.time() - 100
    reasons = ("Not Active", "Not Active", "Not Active", "Active")             # sw_power_cap
    rows = [_row(t0 + 0.2 * i, 2000, reasons if i == 5 else ("Not Active",) * 4) for i in range(10)]
    rows.append(_row(t0 + 0.2 * 3, 1500, ("Active", "Not Active", "Not Active", "Not Active"), uuid="GPU-other"))
    rec = _sampler(rows, [(t0, t0 + 2.0)], uuid="GPU-abc")        # another GPU's row is ignored
    assert rec["reasons"] == ["sw_power_cap"] and rec["sm_mhz"] == 2000


def test_clock_record_short_window_falls_back_to_the_run():
    t0 = time.time() - 100
    rows = [_row(t0 + 0.2 * i, 1900 + i) for i in range(9)]
    rec = _sampler(rows, [(t0 + 0.61, t0 + 0.69)])                # under three samples inside
    assert rec["window"].startswith("whole run") and rec["samples"] == 9 and rec["sm_mhz"] == 1904


def test_clock_record_without_nvidia_smi():
    c = bench.ClockSampler()
    c.proc = None
    assert c.stop()["samples"] == 0


def test_traffic_is_dropped_when_the_kernel_sources_change(tmp_path, monkeypatch):
    f = tmp_path / "summary.md"
    f.write_text("traffic_bytes_per_launch: 2222723328\nkernel_source_sha256_16: %s\n" % bench.kernel_source_hash())
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic() == 2222723328.0
    f.write_text("traffic_bytes_per_launch: 2222723328\nkernel_source_sha256_16: 0123456789abcdef\n")
    assert bench.ncu_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.md"))
    assert bench.ncu_traffic() is None


def test_committed_traffic_summary_names_a_hash():
    text = open(bench.TRAFFIC_FILE).read()
    assert "kernel_source_sha256_16:" in text and "traffic_bytes_per_launch:" in text
    for rel in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(bench.ROOT, rel)), rel


def test_operation_counts():
    # N = 4096: three radix-16 passes; per pass and row six MMAs of 2 x 32 x 16 operations
    assert bench.tc_flops(4096, 64, 4680) == 4680 * 3 * 65 * 256 * 6 * 2 * 32 * 16
    assert bench.tc_flops(4096, 64, 4680) == pytest.approx(1.435e12, rel=1e-3)
    # 5 N log2 N per complex FFT (F + 1 per segment) and 6 per complex product
    assert bench.fp32_flops(2048, 32, 1) == 33 * 5 * 2048 * 11 + 32 * 6 * 2048
