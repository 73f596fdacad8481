"""GPU parity of dense_gemv (row- and column-major) against the FP64 oracle:
ragged shapes spanning several tiles, padded leading dimensions (NaN in the
padding), split-K column-major launches, reduced-precision storage."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_canary, assert_normwise, assert_reduced_sum, canary_buffer, host

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (1, 17), (17, 1), (5, 7), (33, 65), (127, 129), (512, 512), (1000, 1537),
          (64, 4096), (4096, 64), (2048, 2048), (3, 20000), (20000, 3)]
STORAGES = ["f32", "f64", "bf16", "f16"]


def lak():
    import paper_1409_0669_gb300 as m
    return m


def make_matrix(m, n, layout, storage, pad, seed):
    """Flat device storage of an m x n N(0,1) matrix in `layout` with leading
    dimension (n or m) + pad; the padding holds NaN."""
    vals = synth.normal((m, n), seed, storage)              # CPU, row-major values
    if layout == "row":
        lda = n + pad
        buf = torch.full((m, lda), float("nan"), dtype=vals.dtype)
        buf[:, :n] = vals
    else:
        lda = m + pad
        buf = torch.full((n, lda), float("nan"), dtype=vals.dtype)
        buf[:, :m] = vals.t()
    return buf.reshape(-1).cuda(), lda, vals


def check(got_t, ref64, storage, what, A=None, x=None, m=0, n=0, lda=0, layout="row"):
    got = host(got_t)
    if storage in ("f32", "f64"):
        assert_normwise(got, ref64, storage, what)
    else:
        absA = np.abs(oracle.widen(A.cpu()))
        abs_terms = oracle.gemv(np.nan_to_num(absA), np.abs(oracle.widen(x.cpu())), m, n, lda,
                                layout)
        assert_reduced_sum(got, ref64, abs_terms, np.full(m, n), storage, what)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("layout", ["row", "col"])
@pytest.mark.parametrize("shape", SHAPES, ids=str)
@pytest.mark.parametrize("pad", [0, 3])
def test_gemv(storage, layout, shape, pad):
    m, n = shape
    A, lda, vals = make_matrix(m, n, layout, storage, pad, seed=m * 131 + n)
    x = synth.uniform(n, 7, storage).cuda()
    buf, y = canary_buffer(m, A.dtype, A.device)
    lak().dense_gemv(A, x, y=y, m=m, n=n, lda=lda, layout=layout)
    torch.cuda.synchronize()
    ref = oracle.gemv(A.cpu(), x.cpu(), m, n, lda, layout)
    check(y, ref, storage, f"gemv {layout} {shape} lda={lda}", A, x, m, n, lda, layout)
    assert_canary(buf, m)


@pytest.mark.parametrize("cfg", [(64, 0, 1, 0), (512, 0, 16, 1), (128, 5, 8, 0), (256, 0, 2, 1),
                                 (96, 1000, 4, 0)], ids=str)
@pytest.mark.parametrize("layout", ["row", "col"])
def test_gemv_configs(cfg, layout):
    m, n = 777, 3001
    A, lda, vals = make_matrix(m, n, layout, "f32", 1, seed=3)
    x = synth.uniform(n, 8, "f32").cuda()
    y = lak().dense_gemv(A, x, m=m, n=n, lda=lda, layout=layout, cfg=cfg)
    torch.cuda.synchronize()
    check(y, oracle.gemv(A.cpu(), x.cpu(), m, n, lda, layout), "f32", f"cfg {cfg}")


def test_gemv_2d_tensor_views_and_transpose():
    """A row-major tensor, its transpose view (column-major), and B^T x through
    the column-major kernel on row-major storage."""
    m_, n_ = 300, 517
    A = synth.normal((m_, n_), 9, "f32").cuda()
    x = synth.uniform(n_, 10, "f32").cuda()
    w = synth.uniform(m_, 11, "f32").cuda()
    lk = lak()
    y_row = lk.dense_gemv(A, x)
    y_ref = oracle.gemv(A.cpu(), x.cpu(), m_, n_, n_, "row")
    assert_normwise(host(y_row), y_ref, "f32")
    At = A.t()                                    # (n_, m_), column-major view
    z = lk.dense_gemv(At, w)                      # A^T w
    z_ref = oracle.gemv(A.cpu(), w.cpu(), n_, m_, n_, "col")
    assert_normwise(host(z), z_ref, "f32")
    # same matrix in both layouts gives the same product (within tolerance)
    Acol = A.t().contiguous().t()
    y_col = lk.dense_gemv(Acol, x)
    assert_normwise(host(y_col), y_ref, "f32")


def test_gemv_identity_and_empty():
    lk = lak()
    n = 1000
    eye = torch.eye(n, device="cuda")
    x = synth.uniform(n, 12, "f32").cuda()
    assert torch.equal(lk.dense_gemv(eye, x), x)
    assert torch.equal(lk.dense_gemv(eye.t(), x), x)
    e = torch.empty(5, 0, device="cuda")
    y = torch.full((5,), 3.0, device="cuda")
    lk.dense_gemv(e, torch.empty(0, device="cuda"), y=y, m=5, n=0, lda=1, layout="row")
    assert torch.all(y == 0)


def test_gemv_colmajor_split_workspace_reuse():
    lk = lak()
    m, n = 96, 50_000                        # few row tiles, many column splits
    A, lda, _ = make_matrix(m, n, "col", "f32", 0, seed=13)
    x = synth.uniform(n, 14, "f32").cuda()
    need = lk.dense_gemv_workspace(m, n, "col", "f32")
    assert need > 0
    ws = torch.zeros(need, dtype=torch.uint8, device="cuda")
    ref = oracle.gemv(A.cpu(), x.cpu(), m, n, lda, "col")
    first = None
    for _ in range(10):
        y = lk.dense_gemv(A, x, m=m, n=n, lda=lda, layout="col", workspace=ws)
        torch.cuda.synchronize()
        assert_normwise(host(y), ref, "f32")
        first = y.clone() if first is None else first
        assert torch.equal(y, first), "split-K combine must be deterministic"
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(lk.LakError, match="LAK_EWORKSPACE"):
        lk.dense_gemv(A, x, m=m, n=n, lda=lda, layout="col", workspace=small)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_gemv_reduced_storage_vs_fp32_data(storage):
    m, n = 1024, 1024
    A32 = synth.normal((m, n), 15, "f32")
    x32 = synth.uniform(n, 16, "f32")
    dt = synth.torch_dtype(storage)
    y = lak().dense_gemv(A32.to(dt).cuda(), x32.to(dt).cuda())
    ref = oracle.gemv(A32, x32, m, n, n, "row")
    err = np.linalg.norm(host(y) - ref) / np.linalg.norm(ref)
    assert err <= 1e-2
