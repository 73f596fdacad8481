"""Reduced-precision storage and the compensated inner product against the
FP64 oracle: mixed-sign values whose magnitudes span 1e-4..1e4 (the precision
workload), plain FP32 accumulation versus compensated accumulation."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import host

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [1, 7, 1000, 1_000_003])
@pytest.mark.parametrize("cfg", [None, (128, 0, 1, 0), (256, 37, 8, 1)], ids=str)
def test_compensated_dot_mixed_magnitude(storage, n, cfg):
    lo, hi = (-4, 4) if storage != "f16" else (-2, 2)      # FP16 range: |v| <= 65504
    x = synth.mixed_magnitude(n, 1, storage, lo, hi).cuda()
    y = synth.mixed_magnitude(n, 2, storage, lo, hi).cuda()
    m = lak()
    comp = m.vec_dot_compensated(x, y, cfg=cfg).item()
    plain = m.vec_dot(x, y, cfg=cfg).item()
    torch.cuda.synchronize()
    ref = oracle.dot(x.cpu(), y.cpu())
    xs, ys = host(x), host(y)
    abs_sum = float(np.sum(np.abs(xs * ys)))
    # twice-FP32 accumulation then FP64 combines: error far below FP32's
    assert abs(comp - ref) <= 2.0 ** -40 * abs_sum + 4 * np.spacing(abs(ref))
    assert abs(comp - ref) <= abs(plain - ref) + 2.0 ** -40 * abs_sum


def test_compensated_dot_recovers_cancelled_term():
    """Terms 2^30, 1, -2^30, 0 in one thread's group of 4: FP32 loses the 1."""
    n = 4
    x = torch.tensor([2.0 ** 30, 1.0, -(2.0 ** 30), 0.0], device="cuda")
    ones = torch.ones(n, device="cuda")
    cfg = (32, 1, 4, 0)                        # one thread reads all four terms
    assert lak().vec_dot_compensated(x, ones, cfg=cfg).item() == 1.0
    assert lak().vec_dot(x, ones, cfg=cfg).item() == 0.0


def test_compensated_dot_errors():
    m = lak()
    x = torch.ones(10, dtype=torch.float64, device="cuda")
    with pytest.raises(m.LakError, match="LAK_EDTYPE"):
        m.vec_dot_compensated(x, x)
    e = torch.empty(0, device="cuda")
    out = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    m.vec_dot_compensated(e, e, out=out)
    assert out.item() == 0.0
