"""bench.py's clock record: nvidia-smi rows are time-stamped, and only the rows
taken inside the timed region count; a region shorter than the sampling
interval falls back to the rows around it.  Checked on CPU with fake
nvidia-smi output (no process is started)."""
import datetime
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _stamp(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def _sampler(tmp_path, rows, t0, t1):
    import bench
    c = bench.ClockSampler(0)
    c.proc = _DoneProcess()
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        for dt, mhz, reasons in rows:
            flags = ["Active" if r in reasons else "Not Active" for r in bench.ClockSampler.NAMES]
            f.write(f"{_stamp(t0 + dt)}, 0, {mhz}, 2070, 850.0, 0x0, " + ", ".join(flags) + "\n")
    c.t0, c.t1 = t0, t1
    return c


def test_only_rows_inside_the_timed_region_count(tmp_path):
    t0 = time.time()
    rows = [(-2.0, 1200, {"hw_slowdown"}),      # before: idle and throttled, not counted
            (0.05, 2070, set()), (0.10, 2055, {"sw_power_cap"}), (0.15, 2070, set()),
            (1.2, 900, {"sw_thermal_slowdown"})]  # after the region, not counted
    got = _sampler(tmp_path, rows, t0, t0 + 0.2).stop()
    assert got["window"] == "timed region"
    assert got["samples"] == 3
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]


def test_short_region_falls_back_to_the_rows_around_it(tmp_path):
    t0 = time.time()
    rows = [(-0.3, 2070, set()), (0.08, 2070, set()), (3.0, 1100, {"hw_thermal_slowdown"})]
    got = _sampler(tmp_path, rows, t0, t0 + 0.05).stop()
    assert got["window"] == "timed region +- 0.5 s"
    assert got["samples"] == 2
    assert got["reasons"] == []


def test_no_rows_is_reported(tmp_path):
    t0 = time.time()
    got = _sampler(tmp_path, [], t0, t0 + 0.05).stop()
    assert got["reasons"] == ["no samples"] and got["sm_mhz"] is None
