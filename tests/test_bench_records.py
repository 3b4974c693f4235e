"""Host logic of bench.py (no GPU).  The clock record: the SM clock and the
throttle reasons of the nvidia-smi samples taken inside the timed region, or,
for a region shorter than the sampling period, of the samples just before and
just after it, and the summary says which.  The pair-kernel roofline record:
each fraction recomputes from the fields printed beside it."""
import bench

IDLE = "2070, 2070, 480.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "1850, 2070, 1390.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
HOT = "1500, 2070, 1200.00, 0x0000000000000040, Not Active, Active, Not Active, Not Active"


def _sampler(samples, t_start, t_end):
    c = bench.ClockSampler(0)
    c.lines = list(samples)
    c.t_start, c.t_end = t_start, t_end
    return c


def test_samples_inside_the_region():
    c = _sampler([(0.0, IDLE), (1.0, CAPPED), (1.2, CAPPED), (1.4, IDLE), (3.0, HOT)], 0.5, 2.0)
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 1850.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["window"].startswith("samples inside")


def test_short_region_takes_the_neighbouring_samples():
    # a 5 ms region between two samples 200 ms apart
    c = _sampler([(0.0, IDLE), (0.2, HOT), (0.4, CAPPED)], 0.201, 0.206)
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == (1500.0 + 1850.0) / 2
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"] and "just before and just after" in s["window"]


def test_no_sampler_gives_no_clock():
    s = _sampler([], 0.0, 1.0).summary()
    assert s["samples"] == 0 and s["sm_mhz"] is None and s["reasons"] == []


def test_pair_roofline_fractions_follow_from_the_line():
    # every fraction of the roofline record recomputes from the fields printed
    # beside it (synthetic launch: 1 GB in 0.15 ms on the 1M-atom workload,
    # a fifth of the launches pruning)
    rates = {"fp32_tflops": 74.0, "clock_mhz": 2070, "sm_count": 152}
    clk = {"sm_mhz": 2070.0}
    r = bench.pair_roofline(1.0e9, 0.15, 0.2, (6789.6, "measured"), rates, clk, bench.COUNTER_ATOMS, 200_000,
                            50.0e6, 85.0e6, 345.7 ** 3)
    secs = r["ms_per_launch"] * 1e-3
    assert abs(r["frac"] - r["alg_bytes_per_launch"] / secs / 1e9 / r["peak"]) < 1e-12
    assert abs(r["achieved"] - r["alg_bytes_per_launch"] / secs / 1e9) < 1e-6
    fs = r["flop_side"]
    assert abs(fs["frac"] - fs["flops_per_launch"] / secs / 1e12 / fs["fp32_peak_tflops"]) < 1e-12
    # the ncu counters recorded for the current pair.cu, weighted by the pruning launches
    assert r["traffic"] is not None and "dram_frac" in r and "issue_frac" in r
    assert abs(r["dram_frac"] - r["traffic"] / secs / 1e9 / r["peak"]) < 1e-12
    assert abs(r["issue_frac"] - r["inst_executed_per_launch"] / (secs * 2070e6 * 152 * 4)) < 1e-12
    plain = bench.recorded_pair_counters(0.0, bench.COUNTER_ATOMS)
    pruning = bench.recorded_pair_counters(1.0, bench.COUNTER_ATOMS)
    assert abs(r["traffic"] - (0.8 * plain["dram_bytes"] + 0.2 * pruning["dram_bytes"])) < 1.0
    # another workload size: no counters (they were scaled to the 1M-atom one)
    assert bench.recorded_pair_counters(0.2, 300_000) == {}
