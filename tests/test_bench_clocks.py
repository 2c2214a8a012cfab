"""The benchmark's clock record on CPU: one nvidia-smi sampler runs for the
whole measurement and each timed region is summarised by the samples stamped
inside it. Samples are planted directly (no nvidia-smi, no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(mhz, power, cap=False, hw=False):
    return (f"0, {mhz}, 2070, {power}, 0x0, {'Active' if hw else 'Not Active'}, Not Active, "
            f"Not Active, {'Active' if cap else 'Not Active'}")


def _sampler(samples):
    s = bench.ClockSampler(0)
    s.proc = object()                 # stands for a running nvidia-smi
    s.lines = [(t, _line(*args)) for t, args in samples]
    return s


def test_region_reads_only_the_samples_inside_it():
    s = _sampler([(1.0, (2070, 300)), (2.0, (1740, 1390, True)), (2.2, (1700, 1380, True)),
                  (3.0, (2070, 250))])
    r = s.summary(1.9, 2.5)
    assert r["samples"] == 2
    assert r["sm_mhz"] == 1720.0
    assert r["reasons"] == ["sw_power_cap"]
    assert r["power_w_max"] == 1390.0
    assert r["sm_max_mhz"] == 2070.0


def test_short_region_takes_the_next_sample_else_the_last_one():
    s = _sampler([(1.0, (2070, 300)), (2.0, (1800, 1300, True))])
    after = s.summary(1.5, 1.6)          # nothing inside: the first sample after the start
    assert after["samples"] == 1 and after["sm_mhz"] == 1800.0 and after["reasons"] == ["sw_power_cap"]
    before = s.summary(2.5, 2.6)         # nothing after either: the last sample before
    assert before["samples"] == 1 and before["sm_mhz"] == 1800.0


def test_whole_run_summary_and_throttle_reasons():
    s = _sampler([(1.0, (2070, 300)), (2.0, (1500, 900, False, True))])
    r = s.summary()
    assert r["samples"] == 2
    assert r["reasons"] == ["hw_slowdown"]
    assert r["sm_mhz"] == (2070 + 1500) / 2


def test_no_sampler_is_reported_as_such():
    s = bench.ClockSampler(0)
    assert s.summary(0.0, 1.0)["reasons"] == ["nvidia-smi unavailable"]
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]
