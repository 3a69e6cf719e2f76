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


def test_roofline_of_a_profiled_step():
    """achieved = algorithmic bytes / the union of the marcher's spans; the
    per-launch figure over the summed spans; DRAM traffic per average launch
    and L2 bytes from the per-crossing figures."""
    prof = {"march_crossings": 1e12, "records": 3e11, "march_sum_ms": 60000.0, "march_launches": 20000,
            "march_ms": 40000.0, "step_ms": 65000.0, "flush_ms": 30000.0}
    r = bench.roofline_of(prof, 1, 6000.0, "of measured", l2_peak=7000.0)
    alg = 1e12 * 60 + 3e11 * bench.RECORD_BYTES
    assert abs(r["achieved"] - alg / 40.0 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 6000.0) < 1e-12
    assert abs(r["achieved_over_summed_launch_spans"] - alg / 60.0 / 1e9) < 1e-6 * r["achieved"]
    assert abs(r["traffic"] - bench.MARCH_DRAM_BYTES_PER_CROSSING * 1e12 / 20000) < 1.0
    assert abs(r["l2"]["achieved"] - bench.MARCH_L2_BYTES_PER_CROSSING * 1e12 / 40.0 / 1e9) < 1e-6
    assert abs(r["kernel_busy_share_of_step"] - 40000 / 65000) < 1e-12
    assert bench.roofline_of(prof, 1, 6000.0, "of measured")["l2"] is None
