"""The arithmetic-pipe probes behind the roofline of the field sum.

Pure FP32 FMA and packed FFMA2 streams must land between a third of and just
above the nominal FP32 rate of the device (SMs x 128 lanes x the maximum SM
clock), and agree with each other; the MUFU stream must be far below the FMA
rate (a quarter-rate or slower unit) but nonzero.
"""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1609_08146_gb300 as sc  # noqa: E402

MAX_SM_HZ = 2.2e9  # above any GB300 boost clock


def test_probe_rates_are_physical():
    ctx = sc.Context(0)
    try:
        before = ctx.counters()["launches"]
        p = ctx.measure_alu_peaks()
        assert ctx.counters()["launches"] - before == 12
    finally:
        ctx.close()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * MAX_SM_HZ
    for k in ("fp32_lane_ops_per_s", "fp32x2_lane_ops_per_s"):
        assert ceiling / 3 < p[k] < ceiling * 1.02, (k, p[k], ceiling)
    assert 0.7 < p["fp32x2_lane_ops_per_s"] / p["fp32_lane_ops_per_s"] < 1.4
    assert 0 < p["mufu_ops_per_s"] < 0.5 * p["fp32_lane_ops_per_s"]
