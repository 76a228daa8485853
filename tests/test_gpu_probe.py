"""The FP32 FMA throughput probe (lc_probe_fp32) that checks the force
sweep's roofline denominator: its flop count follows from the launch, and
its rate lies below the unit-count bound at any clock this GPU runs."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_fp32_rate_is_bounded(lc):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    flops, sec = lc.probe_fp32(1 << 14)
    assert flops == 4.0 * 8 * (1 << 14) * sms * 8 * 256
    rate = flops / sec
    # 128 FP32 lanes per SM, 2 flop per FMA, at most 2.2 GHz
    assert 0.1 * sms * 128 * 2 * 1.0e9 < rate < sms * 128 * 2 * 2.2e9
    with pytest.raises(lc.LCError):
        lc.probe_fp32(0)
