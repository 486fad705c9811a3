"""hsc_measure_fma_rate: the FP32 and FP64 multiply-add issue rates that the
non-tensor rooflines are held against."""

import pytest

pytestmark = pytest.mark.gpu


def test_fma_rates_plausible(hsc):
    import torch
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fp32 = hsc.hsc_measure_fma_rate(0)
    fp64 = hsc.hsc_measure_fma_rate(0, fp64=True)
    # 128 FP32 lanes per SM at no more than ~2.2 GHz; at least a quarter of that
    nominal = sms * 128 * 2.2e9
    assert 0.25 * nominal < fp32 < 1.05 * nominal
    assert 0.0 < fp64 < fp32
