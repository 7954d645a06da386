"""Host-side arithmetic of bench.py that needs no GPU."""
import math

import bench


def test_records_roofline_counts_the_backward_like_the_forward():
    fma, xu_s, hbm = 38.7e12, 2 / 10.0e12 + 2 / 5.0e12 + 1 / 4.9e12, 6783.5
    r = bench.records_roofline(2_000_000, 0.5, fma, xu_s, hbm)
    ops = bench.OPS_PER_EVAL + bench.OPS_PER_EMIT_BWD
    assert r["ops_per_unit"] == ops and r["units"] == 2_000_000
    # 2e6 records x ops in 0.5 ms
    assert math.isclose(r["achieved"], 2e6 * ops / 5e-4 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / 38.7)
    # the transcendental mix: XU_PER_EVAL operations take xu_s seconds at peak
    assert math.isclose(r["xu"]["peak"], bench.XU_PER_EVAL / xu_s / 1e12)
    assert math.isclose(r["xu"]["frac"], 2e6 * xu_s / 5e-4)
    assert math.isclose(r["hbm"]["achieved_gbs"], 2e6 * bench.REC_BYTES_BWD / 5e-4 / 1e9)
    assert math.isclose(r["hbm"]["frac"], r["hbm"]["achieved_gbs"] / hbm)
    assert r["replayed_tiles"] is False


def test_records_roofline_is_absent_without_records_or_time():
    assert bench.records_roofline(0, 1.0, 1e12, 1e-12, 1.0) is None
    assert bench.records_roofline(10, 0.0, 1e12, 1e-12, 1.0) is None


def test_raster_traffic_only_while_the_captured_source_matches(tmp_path, monkeypatch):
    # the committed summary's traffic applies to the raster sources it was
    # captured on; with the same sources it is reported, after any change
    # it is null
    assert bench.raster_traffic("clustered-100k-1080p") > 1e9
    changed = tmp_path / "raster.cu"
    changed.write_text("// another kernel\n")
    monkeypatch.setattr(bench, "RASTER_SOURCES", (str(changed),) + tuple(bench.RASTER_SOURCES[1:]))
    assert bench.raster_traffic("clustered-100k-1080p") is None
    assert bench.raster_traffic("no-such-workload") is None


def test_hbm_peak_says_which_denominator_it_is(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6783.5})
    assert bench.hbm_peak() == (6783.5, "hbm_gbs of MEASURED_PEAKS.json (of measured)")
    monkeypatch.setattr(bench, "measured_peaks", lambda: {})
    v, basis = bench.hbm_peak()
    assert v == 6800.0 and basis.endswith("(of fallback)")
