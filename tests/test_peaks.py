"""The pipe issue-rate probes (cfie_measure_peaks): plausible against the
unit counts of the device (FP32 FMA 128 lanes per SM per clock, FP64 a small
fraction of it) at any clock between 0.5 and 2.2 GHz."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    from paper_1408_1578_gb300 import cfie
    ctx = cfie.Context(0)
    p = ctx.measure_peaks()
    ctx.close()
    sms = p["sms"]
    assert sms > 0
    fma_per_clock = p["fp32_fma_per_s"] / sms
    assert 128 * 0.5e9 * 0.6 < fma_per_clock < 128 * 2.2e9 * 1.05
    assert 0 < p["mufu_per_s"] < p["fp32_fma_per_s"]
    assert 0 < p["fp64_fma_per_s"] < p["fp32_fma_per_s"]
