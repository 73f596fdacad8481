"""Row-binned CSR (csr_bin_build / csr_bin_spmv): the permutation and bin
offsets bit-exact against the oracle's stable binning, and the product
against the oracle's CSR product -- on stencils, the power-law distribution,
patterns with empty rows and rows at every bin edge, rows longer than the last
bin's bound, one row, no rows, and the 2M-row power-law matrix."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_normwise, assert_reduced_sum, host

pytestmark = pytest.mark.gpu


def check(y, rp, ci, v, x, storage, what):
    """FP32/FP64: norm-wise bar; BF16/FP16 outputs: one storage ulp plus the
    FP32 accumulation bound per row (the library's rule for reduced storage)."""
    got, ref = host(y), oracle.csr_spmv(rp, ci, v, x)
    if storage in ("f32", "f64"):
        assert_normwise(got, ref, storage, what)
    else:
        abs_terms = oracle.csr_spmv(rp, ci, np.abs(oracle.widen(v)), np.abs(oracle.widen(x)))
        nterms = np.diff(rp.numpy()).astype(np.float64)
        assert_reduced_sum(got, ref, abs_terms, nterms, storage, what)


PER_LANE, BINS = 4, 7            # LAK_CSR_BIN_PER_LANE, LAK_CSR_BINS


def CB():
    from paper_1409_0669_gb300.csr_bin import BinnedCsr
    return BinnedCsr


def _edge_pattern(seed, n=500):
    g = synth.rng(seed)
    lens = [0, 1, 4, 5, 8, 9, 16, 17, 32, 33, 64, 65, 128, 129, 256, 257, 700, 3000]
    lens += list(g.integers(0, 300, 600))
    rp = np.zeros(len(lens) + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    ci = g.integers(0, n, int(rp[-1])).astype(np.int32)
    v = g.standard_normal(int(rp[-1]))
    return torch.from_numpy(rp.astype(np.int32)), torch.from_numpy(ci), v, n


def _cases(storage):
    rp, ci, v = synth.laplacian_2d(64, storage)
    yield "lap2d_64", rp, ci, v, 64 * 64
    rp, ci, v = synth.laplacian_3d(20, storage)
    yield "lap3d_20", rp, ci, v, 20 ** 3
    rp, ci, v = synth.powerlaw_csr(30_000, 25_000, 3, storage)
    yield "powerlaw_30k", rp, ci, v, 25_000
    rp, ci, v = synth.random_csr(3000, 2000, 4, storage, 0, 40, 0.3, True)
    yield "random_empty_rows", rp, ci, v, 2000
    rp, ci, v, n = _edge_pattern(5)
    yield "bin_edges", rp, ci, synth.to_storage(v, storage), n


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_layout_and_product_vs_oracle(storage):
    for name, rp, ci, v, n in _cases(storage):
        A = CB()(rp.cuda(), ci.cuda(), v.cuda(), n)
        torch.cuda.synchronize()
        operm, obins = oracle.csr_row_bins(rp, PER_LANE, BINS)
        assert np.array_equal(A.perm.cpu().numpy()[:rp.numel() - 1], operm), name
        assert np.array_equal(A.bin_ptr.cpu().numpy(), obins), name
        x = synth.uniform(n, 7, storage)
        y = A.spmv(x.cuda())
        torch.cuda.synchronize()
        check(y, rp, ci, v, x, storage, name)


def test_every_row_written_once_and_empty_rows_zero():
    rp, ci, v = synth.random_csr(5000, 300, 8, "f32", 0, 30, 0.4, True)
    A = CB()(rp.cuda(), ci.cuda(), v.cuda(), 300)
    x = synth.uniform(300, 9, "f32").cuda()
    y = torch.full((5000,), float("nan"), device="cuda")
    A.spmv(x, y=y)
    torch.cuda.synchronize()
    yc = y.cpu().numpy()
    assert not np.isnan(yc).any()
    empty = (rp[1:] - rp[:-1]).numpy() == 0
    assert (yc[empty] == 0).all()


@pytest.mark.parametrize("m", [0, 1])
def test_tiny(m):
    rp = torch.tensor([0] + [5] * m, dtype=torch.int32)
    ci = torch.tensor([0, 3, 1, 2, 4][:5 if m else 0], dtype=torch.int32)
    v = torch.arange(1.0, 6.0)[:5 if m else 0]
    A = CB()(rp.cuda(), ci.cuda(), v.cuda(), 5)
    torch.cuda.synchronize()
    # one row of 5 entries: 5 > PER_LANE, 5 <= 2 * PER_LANE -> bin 1
    assert A.bin_ptr.cpu().tolist() == ([0] * 8 if m == 0 else [0, 0, 1, 1, 1, 1, 1, 1])
    if m:
        x = torch.tensor([1.0, 10.0, 100.0, 1000.0, 10000.0])
        y = A.spmv(x.cuda())
        torch.cuda.synchronize()
        assert y.item() == 1 * 1 + 2 * 1000 + 3 * 10 + 4 * 100 + 5 * 10000


@pytest.mark.parametrize("cfg", [(64, 0, 0, 0), (256, 0, 0, 0), (128, 7, 0, 0)])
def test_launch_shapes(cfg):
    rp, ci, v = synth.powerlaw_csr(20_000, 20_000, 11, "f32")
    A = CB()(rp.cuda(), ci.cuda(), v.cuda(), 20_000)
    x = synth.uniform(20_000, 12, "f32")
    y = A.spmv(x.cuda(), cfg=cfg)
    torch.cuda.synchronize()
    assert_normwise(host(y), oracle.csr_spmv(rp, ci, v, x), "f32", str(cfg))


def test_powerlaw_2m_full_size():
    rp, ci, v = synth.powerlaw_csr(2_000_000, 2_000_000, 1, "f32")
    A = CB()(rp.cuda(), ci.cuda(), v.cuda(), 2_000_000)
    x = synth.uniform(2_000_000, 13, "f32")
    y = A.spmv(x.cuda())
    torch.cuda.synchronize()
    operm, obins = oracle.csr_row_bins(rp, PER_LANE, BINS)
    assert np.array_equal(A.bin_ptr.cpu().numpy(), obins)
    assert np.array_equal(A.perm.cpu().numpy(), operm)
    assert_normwise(host(y), oracle.csr_spmv(rp, ci, v, x), "f32", "power-law 2M")
