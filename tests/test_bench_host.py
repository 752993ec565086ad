"""Host logic of bench.py on the CPU: the clock summary (throttle reasons, the timed
window, the nvidia-smi fallback) and the deadline-bounded oracle timer."""
import time

import numpy as np

import bench


def _sampler(nv, window, smi_lines=()):
    c = bench.ClockSampler(0)
    c.nv = list(nv)
    c.nv_max = 2032
    c.window = list(window)
    c.lines = list(smi_lines)
    return c


def test_clock_summary_uses_only_samples_inside_the_timed_window():
    nv = [(0.5, 900, 0x1), (1.0, 2032, 0), (1.5, 2000, 0), (2.0, 1980, 0), (3.0, 600, 0x1)]
    s = _sampler(nv, (1.0, 2.0)).summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2000.0
    assert s["sm_mhz_min"] == 1980.0
    assert s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == []          # idle (0x1) outside the window is not reported


def test_clock_summary_names_each_throttle_reason_bit():
    for bit, name in ((0x4, "sw_power_cap"), (0x8, "hw_slowdown"), (0x20, "sw_thermal_slowdown"),
                      (0x40, "hw_thermal_slowdown")):
        s = _sampler([(1.0, 2032, 0), (1.1, 1700, bit | 0x1)], (0.0, 2.0)).summary()
        assert s["reasons"] == [name]
    s = _sampler([(1.0, 1500, 0x4 | 0x40)], (0.0, 2.0)).summary()
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_falls_back_to_nvidia_smi_lines():
    lines = ["0, 2032, 2032, 700.1, Not Active, Not Active, Not Active, Active",
             "0, 1990, 2032, 800.0, Not Active, Not Active, Not Active, Not Active",
             "garbage", "0, [N/A], 2032, 1.0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler([], (None, None), lines).summary()
    assert s["samples"] == 2
    assert s["sm_mhz"] == (2032.0 + 1990.0) / 2
    assert s["reasons"] == ["sw_power_cap"]
    assert s["source"] == "nvidia-smi every 200 ms"
    assert _sampler([], (None, None)).summary()["samples"] == 0


def test_clock_sampler_runs_without_a_gpu():
    with bench.ClockSampler(0) as c:
        c.mark_start()
        time.sleep(0.02)
        c.mark_end()
    s = c.summary()
    assert s["samples"] >= 0 and isinstance(s["reasons"], list)


class _FakeOracle:
    """Stands in for oracle.linearize in the timer test (records what ran)."""

    def __init__(self, seconds):
        self.seconds, self.ran = seconds, []

    def linearize(self, tag, pts, *rest):
        time.sleep(self.seconds)
        self.ran.append(tag)


def test_bounded_oracle_timer_stops_at_the_deadline(monkeypatch):
    import oracle
    fake = _FakeOracle(0.01)
    monkeypatch.setattr(oracle, "linearize", fake.linearize)
    jobs = [(i, np.zeros((100 + i, 3), np.float32), None, None) for i in range(400)]
    v, wall, done = bench._time_oracle_bounded(jobs, 4, 0.1)
    assert 4 <= done < 400 and done == len(fake.ran)
    assert sorted(fake.ran) == list(range(done))          # taken in list order, none twice
    assert abs(v - sum(100 + i for i in range(done)) / wall) < 1e-6 * v
    assert wall < 0.1 + 0.1                                # at most one factor per thread past the deadline
    fake.ran.clear()
    v, wall, done = bench._time_oracle_bounded(jobs[:10], 3, 60.0)
    assert done == 10 and sorted(fake.ran) == list(range(10))
