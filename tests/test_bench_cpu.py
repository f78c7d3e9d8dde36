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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the oracle alone (no GPU): one JSON line with the
    arm's metric, unit, the reference markers and a zero-copy e2e object."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    run = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-stride", "5000"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert run.returncode == 0, run.stderr[-2000:]
    lines = [ln for ln in run.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 times the oracle and prints; other ranks exit 0 at once."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    run = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--gpus", "2", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=120, cwd=root, env=env)
    assert run.returncode == 0, run.stderr[-2000:]
    assert not [ln for ln in run.stdout.splitlines() if ln.startswith("{")]


def test_alu_roofline_follows_the_queried_sms_and_the_sampled_clock():
    """The ALU peak is the device's SM count x 128 lanes x the median SM clock of the timed
    region; the fraction follows from the algorithmic operations per particle-step."""
    clk = {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0}
    r = bench.alu_roofline(active_steps=2e9, adv_ms=100.0, step_ms_total=125.0, sm_count=100,
                           clk=clk, peaks={})
    peak = 100 * 128 * 1500e6 / 1e12
    assert r["peak"] == peak
    assert abs(r["achieved"] - bench.OPS_PER_PARTICLE_STEP * 2e10 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-12
    assert abs(r["frac_at_350_ops"] - 350 * 2e10 / 1e12 / peak) < 1e-12
    assert abs(r["advance_share_of_step"] - 0.8) < 1e-12
    assert "100 SMs" in r["peak_source"] and "1500 MHz" in r["peak_source"]
    # no clock samples: the device's maximum clock
    r2 = bench.alu_roofline(2e9, 100.0, 125.0, 100, {"sm_mhz": None, "sm_max_mhz": 2070.0}, {})
    assert r2["peak"] == 100 * 128 * 2070e6 / 1e12 and "maximum" in r2["peak_source"]
