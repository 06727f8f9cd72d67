"""CPU checks of the benchmark's own accounting: the flop count per combination (2mnk R)
against the library's planner, and the parsing of the clock samples that decide
whether a measurement stands."""
import pytest

import bench
from paper_1901_06015_gb300 import synth


def test_real_products_match_the_planner_for_every_combination():
    """bench.real_products (R of the domain case, Fig. "mixeddom") equals the planner's
    M'N'K'/(mnk) for all 2048 combinations, 16-bit complex storage included."""
    import paper_1901_06015_gb300 as mx
    combos = synth.all_combos() + synth.all_combos_16()
    assert len(combos) == 2048
    for combo in combos:
        assert bench.real_products(combo) == mx.mxg_plan(combo, 8, 8, 8).real_products, combo


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_sampler_summary():
    idle = "0, 2070, 2070, 180.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1700, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    lines = [idle] * 9 + [capped] * 3 + ["garbage line", ""]
    out = _sampler(lines).stop()
    assert out["samples"] == 12
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz_p10"] == 1700.0
    assert out["power_w_max"] == pytest.approx(1390.0)
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_thermal_reasons():
    hot = "0, 1500, 2070, 900.0, 0x0000000000000060, Active, Active, Not Active, Not Active"
    out = _sampler([hot] * 4).stop()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
