"""Host-side pieces of bench.py that need no GPU: the parsing of the nvidia-smi
clock samples taken during the timed region (median SM clock, maximum clock,
and which throttle reasons were seen active)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _DoneProcess()
    s.lines = list(lines)
    return s


def test_clock_samples_median_max_and_reasons():
    lines = [
        "2070, 2070, 900.5, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1380.0, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1390.2, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = _sampler(lines).stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3


def test_thermal_and_hardware_slowdown_are_reported():
    lines = ["1500, 2070, 1400, Active, Not Active, Active, Not Active",
             "1490, 2070, 1400, Not Active, Active, Not Active, Not Active"]
    c = _sampler(lines).stop()
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1495.0


def test_missing_nvidia_smi_is_stated():
    c = bench.ClockSampler(0).stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


def test_clock_sampler_queries_the_gpu_by_uuid():
    """nvidia-smi numbers GPUs physically and ignores CUDA_VISIBLE_DEVICES, so the
    sampler names the GPU by the UUID torch reports, not by torch's index."""
    class Props:
        uuid = "8c1f3a2e-0000-1111-2222-333344445555"

    assert bench.ClockSampler.smi_id(Props(), 3) == "GPU-8c1f3a2e-0000-1111-2222-333344445555"

    class PropsPrefixed:
        uuid = "GPU-8c1f3a2e-0000-1111-2222-333344445555"

    assert bench.ClockSampler.smi_id(PropsPrefixed(), 3) == "GPU-8c1f3a2e-0000-1111-2222-333344445555"

    class NoUuid:
        pass

    assert bench.ClockSampler.smi_id(NoUuid(), 3) == "3"
