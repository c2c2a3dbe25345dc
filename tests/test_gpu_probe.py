"""The FP32 FMA-rate probe behind the CUDA-core forms' roofline
(bf_measure_fp32_peak), on the GPU: every mode returns a finite rate below
the nominal FP32 peak of the device, and the outer-product operand pattern
(mode 2, two new register operands per FMA) is no faster than packed FMAs
with one register operand (mode 1)."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1810_11451_gb300 as bf  # noqa: E402


@pytest.fixture(scope="module")
def nominal_tflops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, 2 flop per FMA, at most 2.2 GHz (a bound, not a clock reading)
    return props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12


def test_probe_modes_are_plausible(nominal_tflops):
    st = torch.cuda.current_stream()
    rates = {}
    for mode, iters in ((0, 2000), (1, 1000), (2, 2000)):
        tf, ms = bf.bf_measure_fp32_peak(iters, 3, mode, st)
        assert math.isfinite(tf) and math.isfinite(ms) and ms > 0, (mode, tf, ms)
        assert 0.2 * nominal_tflops < tf <= nominal_tflops, (mode, tf, nominal_tflops)
        rates[mode] = tf
    print("FP32 FMA probe, TFLOP/s:", {k: round(v, 1) for k, v in rates.items()})
    assert rates[2] <= 1.05 * rates[1]
