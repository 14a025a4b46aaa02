"""Host arithmetic behind bench.py's JSON line (no GPU).

The roofline's `achieved` divides algorithmic bytes by time, `roofline_fp64`
divides by the FMA peak derived from the SM count and the maximum SM clock, and
`clocks` carries the median SM clock under load and every throttle reason seen.
These tests pin each of those against hand-computed values so that a change to
the formulas shows up here rather than as a silently different number.
"""
import os
import sys
import tempfile
import types

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def test_algorithmic_bytes_of_the_headline_product():
    import bench
    # FP64 values and int32 columns per stored entry, x read and y written once:
    # the 64^3 elasticity matrix (786,432 rows, 33,980,106 entries).
    n, nnz = 786_432, 33_980_106
    assert bench.min_bytes(n, nnz) == nnz * 12 + n * 16 == 420_344_184
    # FP32 values with float vectors, BF16 values with float vectors
    assert bench.min_bytes(n, nnz, val_bytes=4, vec_bytes=4) == nnz * 8 + n * 8
    assert bench.min_bytes(n, nnz, val_bytes=2, vec_bytes=4) == nnz * 6 + n * 8
    assert bench.min_bytes(0, 0) == 0


def _fake_torch(sms):
    props = types.SimpleNamespace(multi_processor_count=sms)
    cuda = types.SimpleNamespace(get_device_properties=lambda dev: props)
    return types.SimpleNamespace(cuda=cuda)


def test_fp64_fma_peak_from_sm_count_and_clock():
    import bench
    # 2 FP64 FMA lanes per SM per clock, 2 FLOP each: 152 SMs at 2,070 MHz
    assert bench.fp64_peak_tflops(_fake_torch(152), 0, {"sm_max_mhz": 2070.0}) == pytest.approx(1.258560)
    # without a measured clock the nominal maximum is used
    assert bench.fp64_peak_tflops(_fake_torch(152), 0, None) == pytest.approx(1.258560)
    assert bench.fp64_peak_tflops(_fake_torch(76), 0, {"sm_max_mhz": 1035.0}) == pytest.approx(1.258560 / 4)


def _summary_of(rows):
    import bench
    s = bench.ClockSampler(0)
    s.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    s.f.write("\n".join(rows) + "\n")
    s.proc = object()            # a sampler that ran
    return s.summary()


def test_clock_summary_keeps_samples_under_load_and_every_reason():
    # index, sm MHz, max MHz, power W, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = ["0, 345, 2070, 120.5, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle
            "0, 2070, 2070, 980.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1010.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 995.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    s = _summary_of(rows)
    assert s["sm_mhz"] == 2070.0                 # median of the three samples above 250 W
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 4 and s["samples_under_load"] == 3


def test_clock_summary_flags_thermal_slowdown_and_falls_back_to_all_samples():
    rows = ["0, 1500, 2070, 180.0, 0x40, Not Active, Active, Not Active, Not Active",
            "0, 1600, 2070, 200.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _summary_of(rows)
    assert s["sm_mhz"] == 1550.0                 # no sample under load: the median of all
    assert s["reasons"] == ["hw_thermal_slowdown"]
    assert s["samples_under_load"] == 0


def test_clock_summary_without_nvidia_smi():
    import bench
    s = bench.ClockSampler(0)
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
