"""The clock record of bench.py (host logic, no GPU): the SM clock and the
throttle reasons of the nvidia-smi samples taken inside the timed region, or,
for a region shorter than the sampling period, of the samples just before and
just after it, and the summary says which."""
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
