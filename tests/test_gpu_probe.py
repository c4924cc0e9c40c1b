"""GPU: the issue-rate probe behind the roofline denominators (lmvd_rate_probe).

The probe's rates must be those of the device's pipes: FP64 FMA at most the 2 lanes per clock per SM
GB300 issues (times the SM count and the maximum clock), FP64 add and multiply not faster than FMA, and
FP32 FMA tens of times faster than FP64 (GB300 issues FP64 at 1/64 of its FP32 rate). Enough iterations
that launch overhead is negligible.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_rates_are_the_pipes():
    from paper_2206_09878_gb300 import lmvd as L
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fma = L.lmvd_rate_probe(0, 20000)
    add = L.lmvd_rate_probe(1, 20000)
    mul = L.lmvd_rate_probe(2, 20000)
    f32 = L.lmvd_rate_probe(3, 20000)
    clock_max = 2.2e9                       # above GB300's 2070 MHz maximum SM clock
    assert 0 < fma <= 2 * sms * clock_max
    assert add <= 1.05 * fma and mul <= 1.05 * fma
    assert f32 >= 30 * fma
    with pytest.raises(L.LmvdError):
        L.lmvd_rate_probe(7, 10)
