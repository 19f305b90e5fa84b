"""The measured FMA peaks the benchmark's ALU rooflines divide by (gbxc_measure_alu_peaks):
positive, repeatable, and of the order the SM count and clock allow (152 SMs x 128 float32 lanes
x 2 flops x 2.07 GHz = 80.6 TFLOP/s nominal float32; float64 about 1.3 TFLOP/s on this part)."""
import pytest

from gpu_common import need_gpu

pytestmark = pytest.mark.gpu


def test_alu_peaks_plausible_and_repeatable():
    G = need_gpu()
    f32a, f64a = G.gbxc_measure_alu_peaks(0)
    f32b, f64b = G.gbxc_measure_alu_peaks(0)
    assert 20.0 < f32a < 200.0 and 0.2 < f64a < 20.0
    assert f32a > 10.0 * f64a
    assert abs(f32a - f32b) <= 0.15 * f32a and abs(f64a - f64b) <= 0.15 * f64a


def test_alu_peaks_reject_null_outputs():
    G = need_gpu()
    assert G.lib().gbxc_measure_alu_peaks(0, None, None) == G.GBXC_EINVAL
