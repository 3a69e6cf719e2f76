"""Host logic of bench.py that needs no GPU: the clock record taken during
the timed region (median SM clock, throttle reasons) and the roofline
denominators."""
import json

import bench


def test_clock_summary_reads_median_max_and_active_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap (csv,noheader,nounits)
    path.write_text("\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active",
    ]) + "\n")
    s = bench.Clocks(str(path)).summary(0)
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    s1 = bench.Clocks(str(path)).summary(1)
    assert s1["reasons"] == ["hw_thermal_slowdown"] and s1["sm_mhz"] == 1200.0


def test_clock_summary_without_samples(tmp_path):
    assert bench.Clocks(str(tmp_path / "missing.csv")).summary(0) is None


def test_peaks_prefer_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.HBM_FALLBACK_GBS, "of fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.6}))
    assert bench.peaks() == (6789.6, "of measured")


def test_algorithmic_bytes_per_crossing():
    # leaf box 16 + face links 24 + node word 4, then kappa*rho, U_LL and the
    # U read-modify-write per wavelength
    assert bench.bytes_per_crossing(1) == 60
    assert bench.bytes_per_crossing(4) == 44 + 16 * 4
