"""The general and fused forms: x = alpha*y + beta*z (contiguous and strided,
negative increments), x = y + alpha*z with <x, x> in the same pass,
y = alpha*A x + beta*y, and y = A^T x as its own entry point -- against the
FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_dot, assert_normwise, host, spacing

pytestmark = pytest.mark.gpu

U = {"f32": 2.0 ** -24, "f64": 2.0 ** -53, "bf16": 2.0 ** -24, "f16": 2.0 ** -24}


def lak():
    import paper_1409_0669_gb300 as m
    return m


def check_axpby(got, alpha, y, beta, z, storage):
    a = float(np.float32(alpha)) if storage != "f64" else alpha
    b = float(np.float32(beta)) if storage != "f64" else beta
    yv, zv = host(y), host(z)
    ref = oracle.axpby(a, y.cpu(), b, z.cpu())
    bound = 4 * U[storage] * (np.abs(a * yv) + np.abs(b * zv))
    if storage in ("bf16", "f16"):
        bound = bound + spacing(oracle.round_to(ref, storage), storage)
    bad = np.nonzero(np.abs(got - ref) > bound)[0]
    assert bad.size == 0, (bad[:5], got[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("n", [1, 33, 100_003, 2_000_001])
def test_axpby(storage, n):
    y = synth.uniform(n, 1, storage).cuda()
    z = synth.uniform(n, 2, storage).cuda()
    x = torch.empty_like(y)
    lak().vec_axpby(x, -0.7, y, 1.9, z)
    torch.cuda.synchronize()
    check_axpby(host(x), -0.7, y, 1.9, z, storage)


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("steps", [(2, 1, 3), (3, 3, 3), (1, 2, 1)], ids=str)
def test_axpby_strided(storage, steps):
    n = 50_001
    sx, sy, sz = steps
    xb = torch.full((n * sx,), 7.0, dtype=synth.torch_dtype(storage), device="cuda")
    yb = synth.uniform(n * sy, 3, storage).cuda()
    zb = synth.uniform(n * sz, 4, storage).cuda()
    x, y, z = xb[::sx], yb[::sy], zb[::sz]
    lak().vec_axpby(x, 0.5, y, -1.25, z)
    torch.cuda.synchronize()
    check_axpby(host(x.contiguous()), 0.5, y.contiguous(), -1.25, z.contiguous(), storage)
    if sx > 1:
        untouched = host(xb).reshape(n, sx)[:, 1:]
        assert np.all(untouched == 7.0)


def test_axpby_strided_negative_increment():
    from paper_1409_0669_gb300 import _native
    lib = _native.load()
    n = 1000
    y = synth.uniform(n, 5, "f32").cuda()
    z = synth.uniform(n, 6, "f32").cuda()
    x = torch.zeros(n, device="cuda")
    # y read backwards: element i of y is y[n-1-i]
    yp = y.data_ptr() + (n - 1) * 4
    st = lib.vec_axpby_strided(x.data_ptr(), 1, 2.0, yp, -1, 0.5, z.data_ptr(), 1, n, 0,
                               torch.cuda.current_stream().cuda_stream)
    _native.check("vec_axpby_strided", st)
    torch.cuda.synchronize()
    ref = oracle.round_f32(oracle.axpby(2.0, y.cpu().flip(0), 0.5, z.cpu()))
    assert np.array_equal(x.cpu().numpy(), ref)      # both scalings exact: one rounding
    assert lib.vec_axpby_strided(x.data_ptr(), 0, 1.0, y.data_ptr(), 1, 1.0, z.data_ptr(), 1, n,
                                 0, None) == _native.LAK_EINVAL


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("n", [1, 1023, 1_000_003])
def test_axpy_norm2(storage, n):
    y = synth.uniform(n, 7, storage).cuda()
    z = synth.uniform(n, 8, storage).cuda()
    x = torch.empty_like(y)
    ref_x = torch.empty_like(y)
    s = lak().vec_axpy_norm2(x, y, z, 0.5).item()
    lak().vec_axpy(ref_x, y, z, 0.5)
    torch.cuda.synchronize()
    assert torch.equal(x, ref_x)
    xs = host(x)
    assert_dot(s, oracle.dot(x.cpu(), x.cpu()), xs, xs, "f64" if storage == "f64" else "f32")


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("layout", ["row", "col"])
@pytest.mark.parametrize("shape", [(1000, 1537), (64, 50_000), (3, 7)], ids=str)
def test_gemv_alpha_beta(storage, layout, shape):
    m, n = shape
    vals = synth.normal((m, n), 9, storage)
    A = vals.cuda() if layout == "row" else vals.t().contiguous().cuda().t()
    x = synth.uniform(n, 10, storage).cuda()
    y0 = synth.uniform(m, 11, storage).cuda()
    y = y0.clone()
    lak().dense_gemv(A, x, y=y, alpha=-2.5, beta=0.75)
    torch.cuda.synchronize()
    ax = oracle.gemv(vals, x.cpu(), m, n, n, "row")
    ref = -2.5 * ax + 0.75 * host(y0)
    assert_normwise(host(y), ref, storage)
    ynan = torch.full((m,), float("nan"), dtype=y0.dtype, device="cuda")
    lak().dense_gemv(A, x, y=ynan, alpha=3.0, beta=0.0)     # beta = 0: y is not read
    torch.cuda.synchronize()
    assert_normwise(host(ynan), 3.0 * ax, storage)


@pytest.mark.parametrize("layout", ["row", "col"])
def test_gemv_trans_entry_point(layout):
    m, n = 777, 3001
    vals = synth.normal((m, n), 12, "f32")
    A = vals.cuda() if layout == "row" else vals.t().contiguous().cuda().t()
    x = synth.uniform(m, 13, "f32").cuda()
    y = lak().dense_gemv_trans(A, x)
    torch.cuda.synchronize()
    ref = oracle.gemv(vals, x.cpu(), n, m, n, "col")              # A^T x
    assert_normwise(host(y), ref, "f32")
