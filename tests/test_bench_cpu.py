"""Host-side pieces of the benchmark (CPU only): the algorithmic byte count of the QR, the
roofline denominators, and the clock sampler's summary of nvidia-smi records."""
import json
import os

import bench


def test_qr_bytes_is_the_sum_of_the_passes():
    n, m = 1000, 7
    total, upd = bench.qr_bytes(n, m)
    step1 = 8 * n * m                                        # one pass over W
    steps34 = sum(4 * n * i + 8 * n + 4 * n for i in range(m))   # read Q'_{i-1}, read w_i, write q'_i
    assert total == step1 + steps34
    assert upd == steps34 + 8 * n * (m - 1)                  # the update launches also read w_{i+1}
    tb, _ = bench.qr_bytes(n, m, esz=2)
    assert tb == step1 + sum(2 * n * i + 8 * n + 2 * n for i in range(m))


def test_bench_workload_constants_match_the_documented_configuration():
    assert (bench.N_ROWS, bench.M_COLS, bench.K_SKETCH, bench.COND) == (1 << 20, 500, 2000, 1e10)
    total, _ = bench.qr_bytes(bench.N_ROWS, bench.M_COLS)
    assert abs(total - 5.34e11) / 5.34e11 < 1e-2


def test_peaks_read_the_measured_file_or_fall_back():
    peak, kind = bench.peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_clock_summary_reports_loaded_clocks_and_throttle_reasons(tmp_path):
    rows = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 345, 2070, 90.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle sample
    ]
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3
    assert not os.path.exists(c.path)                       # the temporary record is removed


def test_job_rate_is_whole_job_units_over_the_slowest_rank():
    assert bench.job_rate(1e9, 4, 500.0) == 4 * 1e9 / 0.5
