"""The dense tcgen05 MMA rate probe (the roofline's tensor-term denominator)
runs to completion on both operand dtypes and reports a plausible rate."""
import statistics

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2406_17284_gb300 import build
    build.build()
    from paper_2406_17284_gb300 import cat as catmod
    catmod.load()
    return catmod


@pytest.mark.parametrize("dtype,K,lo,hi", [("fp8", 32, 1500.0, 6000.0), ("fp16", 16, 750.0, 3000.0)])
def test_tensor_probe_rate(cat, dtype, K, lo, hi):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dt = cat.DTYPES[dtype]
    n = 1 << 14
    for _ in range(3):
        cat.cat_tensor_probe(dt, n, status.data_ptr())
    times = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cat.cat_tensor_probe(dt, n, status.data_ptr())
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    assert int(status.item()) == 0
    tflops = sms * n * 2.0 * 128 * 256 * K / (statistics.median(times) / 1000.0) / 1e12
    assert lo < tflops < hi, tflops
