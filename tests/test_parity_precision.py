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


# (a0, b0, a1, b1) in FP32 with a0*b0 + a1*b1 nearly cancelling.  Summed as
# TwoProduct + TwoSum the pair is exact; with the TwoSum's addition contracted
# into t = fma(a1, b1, s) the error term no longer matches t and the result is
# off by ~1e-7 relative (found by an exact-rational search over the two forms).
_CONTRACTION_CASES = [
    (0.7667386531829834, 1.4404219388961792, 1.5902308225631714, -1.2410086393356323),
    (1.2833300828933716, 1.2185503244400024, 0.6558557748794556, -1.6678705215454102),
    (1.9207336902618408, 1.9426051378250122, 2.9387106895446777, -1.5670535564422607),
    (0.9904922842979431, 1.8967677354812622, 0.8435077667236328, -1.7870162725448608),
    (1.6495009660720825, 0.8507484793663025, 0.9280365109443665, -1.9705771207809448),
    (0.610117495059967, 1.27778160572052, 1.0796561241149902, -0.5427595973014832),
]


@pytest.mark.parametrize("case", _CONTRACTION_CASES, ids=lambda c: f"{c[0]:.4f}")
def test_compensated_dot_exact_where_contraction_would_not_be(case):
    """One thread sums both products (32 threads, one block, one element per
    access, grid-stride: elements 0 and 32 are thread 0's).  The compensated
    result equals the exact value; a TwoSum whose addition the compiler fused
    with the product would miss it by ~1e-7 relative."""
    a0, b0, a1, b1 = case
    from fractions import Fraction
    for v in case:
        assert float(np.float32(v)) == v             # the cases are FP32 values
    exact = Fraction(a0) * Fraction(b0) + Fraction(a1) * Fraction(b1)
    x = torch.zeros(33, device="cuda")
    y = torch.zeros(33, device="cuda")
    x[0], y[0], x[32], y[32] = a0, b0, a1, b1
    comp = lak().vec_dot_compensated(x, y, cfg=(32, 1, 1, 0)).item()
    assert Fraction(comp) == exact
    assert oracle.dot(x.cpu(), y.cpu()) == float(exact)


def test_compensated_dot_precision_workload_full_size():
    """The precision workload itself: n = 1e8 FP32 values with random signs and
    magnitudes log-uniform in 1e-4..1e4 (seed 0), against the oracle's Dot2,
    with the plain FP32 dot beside it."""
    n = 100_000_000
    xh = synth.mixed_magnitude(n, 0, "f32", -4, 4)
    yh = synth.mixed_magnitude(n, 1, "f32", -4, 4)
    ref = oracle.dot(xh, yh)
    abs_sum = float(np.dot(np.abs(xh.numpy().astype(np.float64)),
                           np.abs(yh.numpy().astype(np.float64))))
    x, y = xh.cuda(), yh.cuda()
    m = lak()
    comp = m.vec_dot_compensated(x, y).item()
    plain = m.vec_dot(x, y).item()
    assert abs(comp - ref) <= 2.0 ** -40 * abs_sum + 4 * np.spacing(abs(ref))
    assert abs(comp - ref) <= abs(plain - ref)
    assert abs(comp - ref) / abs(ref) <= 1e-12


def test_compensated_dot_errors():
    m = lak()
    x = torch.ones(10, dtype=torch.float64, device="cuda")
    with pytest.raises(m.LakError, match="LAK_EDTYPE"):
        m.vec_dot_compensated(x, x)
    e = torch.empty(0, device="cuda")
    out = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    m.vec_dot_compensated(e, e, out=out)
    assert out.item() == 0.0
