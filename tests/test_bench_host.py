"""Host logic of the benchmark on the CPU: the clock record taken during
the timed region, the algorithmic byte counts the phases are measured
against (per particle: sort 304 B over 8 digit passes, 24 B per extra box
pass; build 152 B plus 194 B per cell and 168 B per group; upward 28 B plus
843 B per cell at p = 4; image field 64 B), and the reference arm's line."""
import bench


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return "0, %s, %s, 812.5, 0x0000000000000000, %s, %s, %s, %s" % (sm, mx, hw, hwt, swt, pcap)


def test_clock_summary_median_max_and_reasons():
    lines = [_line(2070, 2070), _line(1980, 2070, pcap="Active"), _line(2070, 2070), "garbage",
             _line("[N/A]", 2070), "", _line(1500, 2070, swt="Active")]
    c = bench.summarise_clocks(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == 2025.0  # median of 2070, 1980, 2070, 1500
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap", "sw_thermal_slowdown"]
    assert bench.summarise_clocks([_line(2070, 2070, hw="Active", hwt="Active")])["reasons"] == [
        "hw_slowdown", "hw_thermal_slowdown"]
    assert bench.summarise_clocks(["garbage", ""]) is None


def test_phase_bytes_per_particle():
    n, nc, ng = 1 << 20, 1000, 100
    b = bench.phase_bytes(n, nc, ng, 4)
    assert b["ms_sort"] == 304 * n  # 8 digit passes of 24 B + 112 B
    assert bench.phase_bytes(n, nc, ng, 4, nbox=96)["ms_sort"] == (304 + 24) * n
    assert bench.phase_bytes(n, nc, ng, 4, nbox=300)["ms_sort"] == (304 + 48) * n
    assert b["ms_build"] == 152 * n + 194 * nc + 168 * ng
    assert b["ms_upward"] == 28 * n + 843 * nc  # 91 + 16 * 35 + 4 * 48 per cell at p = 4
    assert b["ms_periodic"] == 64 * n
    assert abs(bench.fp32_peak_tflops(2070.0, 152) - 80.54784) < 1e-9
    assert abs(bench.fp32_peak_tflops(2070.0, 148) - 80.54784 * 148 / 152) < 1e-9


def test_accuracy_bar_flag():
    assert bench.meets_bar({"median": 6.8e-4, "p99": 8.6e-3})
    assert not bench.meets_bar({"median": 1.03e-3, "p99": 5e-3})
    assert bench.meets_bar({"median": 5e-4, "p99": 1.1e-2})  # the metric bars the median only
    assert not bench.with_bar({"median": 5e-4, "p99": 1.1e-2})["p99_le_1e-2"]
    assert not bench.meets_bar(None)


def test_line_summary_keeps_the_named_keys():
    rec = {"a": 1, "b": {"c": 2}, "bulky": list(range(100))}
    assert bench._summary(rec, ("a", "b", "missing")) == {"a": 1, "b": {"c": 2}, "missing": None}
    assert bench._summary(None, ("a",)) is None
    assert bench._summary({"error": "x"}, ("a",)) == {"error": "x"}


def test_reference_arm_line(capsys):
    """bench.py --impl reference times the oracle on a bounded sample and
    prints one JSON line with the keys the comparison needs; ranks other than
    0 print nothing."""
    import argparse
    import json
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    assert bench.run_reference(args, rank=1, world=2) == 0
    assert capsys.readouterr().out == ""
    assert bench.run_reference(args, rank=0, world=1) == 0
    line = json.loads(capsys.readouterr().out.strip().split("\n")[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    # the step time is the sample's own wall time, so the run fits its clock
    assert 0 < line["ms_per_step"] < 600e3
    assert line["extrapolated_full_evaluation_updates_per_s"] > 0
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_line_rounding_keeps_structure_and_five_digits():
    """The printed line's floats go to five significant digits; integers,
    strings, booleans, None and the nesting are kept."""
    import bench
    rec = {"a": 153861860.76649404, "b": [0.000123456789, 7], "c": {"d": True, "e": None, "f": "x"},
           "g": 0.0, "h": float("inf")}
    out = bench._sig(rec)
    assert out["a"] == 153860000.0
    assert out["b"] == [0.00012346, 7]
    assert out["c"] == {"d": True, "e": None, "f": "x"}
    assert out["g"] == 0.0 and out["h"] == float("inf")
