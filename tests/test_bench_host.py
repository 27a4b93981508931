"""Host-side pieces of bench.py (CPU): the clock-sample summary and the memory-node diagnostic."""
import numpy as np

import bench


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines, first):
    s = bench.ClockSampler(0)
    s.proc, s.lines, s.first = _Proc(), list(lines), first
    return s


IDLE = "1500, 2070, 300, 0x0, Not Active, Not Active, Not Active, Active"
BUSY = "2070, 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active"
HOT = "1800, 2070, 950, 0x0, Not Active, Active, Not Active, Not Active"


def test_clock_summary_uses_the_timed_samples():
    c = _sampler([IDLE, IDLE, BUSY, BUSY, BUSY], first=2).stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
    c = _sampler([IDLE, BUSY, HOT], first=1).stop()
    assert c["reasons"] == ["hw_thermal_slowdown"] and c["samples"] == 2


def test_clock_summary_falls_back_to_all_samples():
    c = _sampler([IDLE, IDLE], first=2).stop()          # no sample arrived after the mark
    assert c["samples"] == 2 and c["reasons"] == ["sw_power_cap"] and c["sm_mhz"] == 1500.0
    assert _sampler(["garbage"], first=0).stop()["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    s.wait_first(0.01)                                   # never started: returns at once
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_host_numa_counts_the_buffer_pages():
    a = np.ones(1 << 24, dtype=np.uint8)                 # 16 MiB, every page touched
    out = bench._host_numa(a.ctypes.data, a.nbytes, 0)
    assert set(out) == {"buffer_pages", "gpu_node"}
    if out["buffer_pages"] is not None:                  # /proc readable (page size varies)
        assert sum(out["buffer_pages"].values()) > 0
    assert bench._host_numa(0, 16, 99) == {"buffer_pages": None, "gpu_node": None}
