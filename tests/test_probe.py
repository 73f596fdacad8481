"""The FP64 FMA throughput probe (lak_probe_fma_f64): its chains really run
(the written sums match the recurrence's closed form), the flop count matches
the launch, argument errors are refused on the host, and the measured rate is
a plausible FP64 rate (not the result of chains the compiler dropped)."""
import math

import pytest
import torch

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


def test_probe_sums_follow_the_recurrence():
    iters, grid, block = 3000, 3, 64
    out, flops = lak().probe_fma_f64(iters, grid=grid, block=block)
    torch.cuda.synchronize()
    assert flops == 2 * 8 * iters * grid * block
    b, c = 0.9999999, 1e-7                       # fixed point c / (1 - b) = 1
    got = out.cpu().tolist()
    assert len(got) == grid * block // 32
    expect = 0.0
    for lane in range(32):
        for k in range(8):
            a0 = 1.0 + 0.125 * k + 1e-3 * lane
            expect += 1.0 + (a0 - 1.0) * b ** iters
    for v in got:
        assert math.isclose(v, expect, rel_tol=1e-9), (v, expect)


def test_probe_rate_is_a_plausible_fp64_rate():
    m = lak()
    out, flops = m.probe_fma_f64(4000)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    m.probe_fma_f64(4000, out=out)
    e.record()
    e.synchronize()
    tflops = flops / (s.elapsed_time(e) * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 4 * 2.2e9 / 1e12           # 2 FP64 FMA per SM per clock, above max clock
    assert 0.3 * nominal < tflops < 1.05 * nominal, tflops


def test_probe_rejects_bad_arguments():
    m = lak()
    from paper_1409_0669_gb300 import _native
    lib = _native.load()
    out = torch.zeros(64, dtype=torch.float64, device="cuda")
    for iters, grid, block in ((0, 1, 32), (1, 0, 32), (1, 1, 48), (1, 1, 2048)):
        st = lib.lak_probe_fma_f64(out.data_ptr(), iters, grid, block, None)
        assert st == _native.LAK_EINVAL
    assert lib.lak_probe_fma_f64(None, 1, 1, 32, None) == _native.LAK_EINVAL
    del m
