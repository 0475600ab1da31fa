"""The FP32 FMA rate probe behind the roofline of the scatter-form kernels:
its flop count follows the launch shape, its per-thread sums are finite
(the chains stay bounded), and the measured rate lies between a third of
the derived FP32 peak and, for scalar FFMA, the derived peak itself (the
probe cannot beat the unit count it is checked against)."""
import math

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_07152_gb300 import build
    build.build()
    import paper_1511_07152_gb300.sepw as S
    return torch, S


def test_fma_probe_counts_and_rate(env):
    torch, S = env
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    out = torch.zeros(sms * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    iters = 200000
    derived = sms * 128 * 2 * 2.070e9 / 1e12  # TFLOP/s at the maximum SM clock
    for paired in (False, True):
        rates = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flops = S.sepw_fma_probe(paired, iters, out, stream)
            b.record(stream)
            b.synchronize()
            rates.append(flops / (a.elapsed_time(b) * 1e-3) / 1e12)
        assert flops == sms * 4 * 256 * iters * 8 * 2 * (2 if paired else 1)
        assert bool(torch.isfinite(out).all())
        best = max(rates)
        assert best > derived / 3, (paired, best, derived)
        if not paired:
            assert best < derived * 1.05, (best, derived)


def test_fma_probe_rejects_short_buffer(env):
    torch, S = env
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(S.SepwError):
        S.sepw_fma_probe(False, 10, out)
