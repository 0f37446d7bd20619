"""ns_alu_peak, the measured FMA rate used as the FP64 roof of the plain form:
its rates are those of a GB300-class device (FP64 on the order of 1 TFLOP/s,
FP32 tens of TFLOP/s, FP32 well above FP64) and repeat within a few percent."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_peak_rates_are_plausible_and_repeat(ns):
    fp64 = [ns.ns_alu_peak(ns.NS_FP64, 100.0) for _ in range(2)]
    fp32 = ns.ns_alu_peak(ns.NS_FP32, 100.0)
    print(f"FP64 {fp64[0] / 1e12:.3f} / {fp64[1] / 1e12:.3f} TFLOP/s, FP32 {fp32 / 1e12:.1f} TFLOP/s")
    assert 0.2e12 < fp64[0] < 5e12
    assert 10e12 < fp32 < 300e12
    assert fp32 > 8 * fp64[0]
    assert abs(fp64[0] - fp64[1]) < 0.1 * max(fp64)
