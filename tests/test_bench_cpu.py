"""Host logic of the benchmark that decides whether a measurement stands: the summary of
the clock samples taken during the timed region, and the host-core count of the oracle's
all-cores leg."""
import bench


def test_clock_rows_summary():
    rows = [
        "0, 345, 2070, 95.1, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 901.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1210.7, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1180.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "garbage line",
    ]
    out = bench.parse_clock_rows([r + "\n" for r in rows])
    assert out["samples"] == 5                   # the malformed line is not a sample
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0               # median of the loaded samples (idle 345 out)
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_rows_report_every_slowdown_seen():
    rows = ["0, 1500, 2070, 1390.0, 0x88, Active, Not Active, Active, Not Active",
            "0, 2070, 2070, 900.0, 0x0, Not Active, Active, Not Active, Not Active"]
    out = bench.parse_clock_rows(rows)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1785.0


def test_clock_rows_empty():
    assert bench.parse_clock_rows([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                                          "samples": 0}


def test_host_workers_is_positive_and_bounded():
    import os
    n = bench._host_workers()
    assert 1 <= n <= (os.cpu_count() or 1)
