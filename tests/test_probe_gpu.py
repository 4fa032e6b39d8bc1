"""The FP32 FMA throughput probe: every thread's chains end at a value fixed
by integer arithmetic (exact in FP32), so a launch that skipped work or
folded the FMAs away is caught; the measured rate must stay below the
GPU's FP32 issue ceiling (148 SMs x 128 lanes x 2 flops x 2.032 GHz)."""
import pytest
import torch

from paper_1203_4938_b300 import fft as F

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("blocks,iters", [(1, 1), (3, 7), (148, 1000), (1184, 4096)])
def test_probe_values(blocks, iters):
    out, flops = F.fma_probe(blocks, iters)
    torch.cuda.synchronize()
    assert flops == 2 * 16 * 256 * blocks * iters
    want = 120.0 + 16.0 * iters
    assert out.numel() == blocks * 256
    assert bool((out == want).all()), (out.min().item(), out.max().item(), want)


def test_probe_rate_is_physical():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 8 * 256, device="cuda")
    F.fma_probe(sms * 8, 1 << 14, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, flops = F.fma_probe(sms * 8, 1 << 14, out)
    e1.record()
    torch.cuda.synchronize()
    tflops = flops / (e0.elapsed_time(e1) * 1e-3) / 1e12
    ceiling = sms * 128 * 2 * 2.1e9 / 1e12
    assert 0.2 * ceiling < tflops < 1.05 * ceiling, (tflops, ceiling)
    assert bool((out == 120.0 + 16.0 * (1 << 14)).all())
