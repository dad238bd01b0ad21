"""The arithmetic-throughput probe (lfe_alu_peak): measured FP32 FMA
throughput within a plausible band of the unit-count peak, FP64 far below
it on this part."""
import pytest
import torch

from paper_2608_12691_b300 import lfe

pytestmark = pytest.mark.gpu


def test_alu_peak_is_plausible():
    f32, f64 = lfe.alu_peak()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    unit_peak_at_3ghz = sms * 128 * 2 * 3.0e9 / 1e12
    assert 0.2 * unit_peak_at_3ghz / 3.0 < f32 < unit_peak_at_3ghz
    assert 0.0 < f64 < f32
