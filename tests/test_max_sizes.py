"""Beyond 2^31 elements: vectors of n = 2^31 + 12345 FP32 elements (8.6 GB
each) and a 65536 x 32771 row- and column-major FP32 matrix (8.6 GB), so that
every element index of the kernels' 64-bit index arithmetic is exercised past
the 32-bit range.  Checked against the oracle at sampled positions -- both
ends, both sides of 2^31, random -- and by the closed forms of the inner
product.  The CSR entry points reject nnz >= 2^31 (int32 indices)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import host

pytestmark = pytest.mark.gpu

N = 2 ** 31 + 12345


def lak():
    import paper_1409_0669_gb300 as m
    return m


def sample_idx(n, seed):
    g = synth.rng(seed)
    edges = [0, 1, 2, 2 ** 31 - 2, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, n - 2, n - 1]
    return torch.tensor(sorted(set(edges + list(g.integers(0, n, 200)))), dtype=torch.int64)


def test_copy_axpy_beyond_2_31():
    m = lak()
    g = torch.Generator(device="cuda").manual_seed(7)
    y = torch.rand(N, generator=g, device="cuda") * 2 - 1
    z = torch.rand(N, generator=g, device="cuda") * 2 - 1
    x = torch.empty_like(y)
    idx = sample_idx(N, 1)
    idx_d = idx.cuda()
    m.vec_copy(x, y)
    torch.cuda.synchronize()
    assert torch.equal(x[idx_d], y[idx_d])
    m.vec_axpy(x, y, z, 0.5)
    torch.cuda.synchronize()
    ys, zs = y[idx_d].cpu(), z[idx_d].cpu()
    ref = oracle.round_to(oracle.axpy(ys, zs, 0.5), "f32")
    assert np.array_equal(host(x[idx_d]), ref)          # one rounding each: bit-exact
    del x, y, z
    torch.cuda.empty_cache()


def test_dot_closed_forms_beyond_2_31():
    m = lak()
    ones = torch.ones(N, device="cuda")
    # the FP64 combine is exact; the FP32 output holds N rounded once to FP32,
    # the FP64 output of the compensated dot holds N itself
    assert m.vec_dot(ones, ones).item() == float(np.float32(N))
    assert m.vec_dot_compensated(ones, ones).item() == float(N)
    alt = torch.ones(N, device="cuda")
    alt[1::2] = -1.0                                       # N odd: sum is 1
    assert m.vec_dot(ones, alt).item() == 1.0
    # the last element alone (index beyond 2^31) carries the whole sum
    e = torch.zeros(N, device="cuda")
    e[N - 1] = 3.0
    assert m.vec_dot(ones, e).item() == 3.0
    del ones, alt, e
    torch.cuda.empty_cache()


@pytest.mark.parametrize("layout", ["row", "col"])
def test_gemv_beyond_2_31_entries(layout):
    rows, cols = 65536, 32771                              # 2,147,680,256 entries
    assert rows * cols > 2 ** 31
    m = lak()
    g = torch.Generator(device="cuda").manual_seed(8)
    A = torch.randn(rows, cols, generator=g, device="cuda")
    x = torch.rand(cols, generator=g, device="cuda") * 2 - 1
    if layout == "row":
        y = m.dense_gemv(A, x)
    else:                                                  # y = A^T x, the same memory column-major
        x2 = torch.rand(rows, generator=g, device="cuda") * 2 - 1
        y = m.dense_gemv(A.t(), x2)
    torch.cuda.synchronize()
    gs = synth.rng(9)
    if layout == "row":
        sel = sorted(set([0, rows - 1] + list(gs.integers(0, rows, 12))))
        for i in sel:
            ref = oracle.gemv(A[i].cpu(), x.cpu(), 1, cols, cols)[0]
            abs_ref = oracle.gemv(np.abs(host(A[i])), np.abs(host(x)), 1, cols, cols)[0]
            assert abs(float(y[i]) - ref) <= 1e-5 * abs_ref + 1e-30, (i, float(y[i]), ref)
    else:
        sel = sorted(set([0, cols - 1] + list(gs.integers(0, cols, 12))))
        xc = x2.cpu()
        for j in sel:
            col = A[:, j].cpu()
            ref = oracle.dot(col, xc)
            abs_ref = float(np.abs(host(col)) @ np.abs(host(xc)))
            assert abs(float(y[j]) - ref) <= 1e-5 * abs_ref, (j, float(y[j]), ref)
    del A
    torch.cuda.empty_cache()


def test_csr_entries_near_2_31():
    """58M rows with 5..64 random columns (about 2.0e9 stored entries, the top
    of the int32 index range): the CSR product (warp-segmented kernel), the
    row-binned product and the sparse inner product, checked at sampled rows
    (the last rows hold entries just below 2^31) and by a closed form."""
    from paper_1409_0669_gb300.csr_bin import BinnedCsr
    m_rows = 58_000_000
    rp, ci, v = synth.device_csr_block_(m_rows, 10, 5, 64, torch.float32, "cuda")
    nnz = int(rp[-1].item())
    assert 1_900_000_000 < nnz < 2 ** 31 - 1
    x = synth.device_uniform_(torch.empty(m_rows, device="cuda"), 11)
    lk = lak()
    y = lk.csr_spmv(rp, ci, v, x)
    yb = BinnedCsr(rp, ci, v, m_rows).spmv(x)
    torch.cuda.synchronize()
    xh = x.cpu()
    g = synth.rng(12)
    rows = sorted(set([0, m_rows - 2, m_rows - 1] + list(g.integers(0, m_rows, 25))))
    rph = rp[torch.tensor(rows + [r + 1 for r in rows], device="cuda")].cpu().numpy()
    for t, r in enumerate(rows):
        a, b = int(rph[t]), int(rph[len(rows) + t])
        vr, cr = v[a:b].cpu(), ci[a:b].cpu()
        ref = oracle.sparse_dot(vr, cr, xh)
        bound = 1e-5 * float(np.abs(host(vr)) @ np.abs(host(xh)[cr.numpy()]))
        assert abs(float(y[r]) - ref) <= bound, (r, float(y[r]), ref)
        assert abs(float(yb[r]) - ref) <= bound, (r, float(yb[r]), ref)
    del y, yb
    # sum over all stored entries of 1 * 1 = nnz, rounded once to the FP32 output
    ones_v = torch.ones_like(v)
    s = lk.vec_dot_sparse(ones_v, ci, torch.ones_like(x)).item()
    assert s == float(np.float32(nnz))
    del rp, ci, v, x, ones_v
    torch.cuda.empty_cache()


def test_csr_rejects_nnz_at_2_31():
    from paper_1409_0669_gb300 import _native
    lib = _native.load()
    assert lib.csr_spmv(None, None, None, None, None, 3, 3, 2 ** 31, 0, None, None) == \
        _native.LAK_EINVAL
