"""Host logic of the benchmark's clock record (no GPU): the samples inside the timed window
decide the median SM clock and the throttle reasons; with fewer than three inside, the whole
sampled span is reported beside them; malformed lines are skipped."""
import bench


def sampler(lines, window):
    s = bench.ClockSampler(0)
    s.lines = list(lines)
    if window is not None:
        s.mark(*window)
    return s.summary()


def line(sm, mx=2070, pw=900.0, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return f"{sm}, {mx}, {pw}, {hw}, {hwt}, {swt}, {cap}"


def test_samples_inside_the_timed_window_decide_the_record():
    lines = [(0.00, line(1200)), (0.10, line(2070)), (0.15, line(2070, cap="Active")), (0.20, line(2055)),
             (0.25, line(2070)), (0.40, line(1000, hwt="Active"))]
    out = sampler(lines, (0.08, 0.26))
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]  # the thermal sample lies outside the window
    assert "sampled_span" not in out and out["timed_window_ms"] == 180.0


def test_short_window_reports_the_sampled_span_beside_it():
    lines = [(0.00, line(2070)), (0.05, line(2070)), (0.11, line(1500, hw="Active")), (0.30, line(2070))]
    out = sampler(lines, (0.10, 0.12))
    assert out["samples"] == 1 and out["reasons"] == ["hw_slowdown"]
    span = out["sampled_span"]
    assert span["samples"] == 4 and span["reasons"] == ["hw_slowdown"] and span["sm_mhz"] == 2070.0
    assert "note" in out


def test_malformed_lines_and_no_window():
    lines = [(0.0, "[N/A], 2070, 900, x, x, x, x"), (0.1, "garbage"), (0.2, line(1980)), (0.3, line(2000))]
    out = sampler(lines, None)
    assert out["samples"] == 2 and out["sm_mhz"] == 1990.0 and out["reasons"] == []
    empty = sampler([], (0.0, 1.0))
    assert empty["samples"] == 0 and empty["sm_mhz"] is None
