"""The throughput micro-benchmark behind the roofline (mppi_measure_peaks):
its rates are what the hardware can do — FP32 FMA close to (never above)
SMs x 128 lanes x 2 flop x the maximum SM clock, and the MUFU rates far
below it — and the SM count is read from the device."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_physical():
    import torch
    assert torch.cuda.is_available()
    from paper_2407_09812_gb300 import build as B
    B.build()
    from paper_2407_09812_gb300 import mppi
    p = mppi.measure_peaks()
    props = torch.cuda.get_device_properties(0)
    assert p["sm_count"] == props.multi_processor_count
    # 128 FP32 lanes per SM, 2 flop per FMA, at most ~2.1 GHz on this part.
    nominal = p["sm_count"] * 128 * 2 * 2.2e9
    assert 0.5 * nominal < p["fp32_flops"] <= nominal, (p["fp32_flops"], nominal)
    for op in ("ex2_ops", "lg2_ops", "rsqrt_ops", "sin_ops", "cos_ops"):
        assert 0.0 < p[op] < p["fp32_flops"] / 2, (op, p[op])
    # ex2 at least as fast as the other MUFU operations.
    assert p["ex2_ops"] >= 0.9 * max(p["lg2_ops"], p["sin_ops"])
    print("peaks", {k: round(v / 1e12, 2) if isinstance(v, float) else v for k, v in p.items()})
