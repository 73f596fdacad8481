"""SELL-C-sigma: the GPU conversion equals the oracle's layout exactly (integer
work: bit-exact), and the SELL product matches the FP64 oracle on Laplacians,
power-law rows, empty rows and sizes that are not multiples of 32."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_normwise, host

pytestmark = pytest.mark.gpu


def S():
    from paper_1409_0669_gb300.sell import SellMatrix
    return SellMatrix


CASES = [
    ("lap2d_64", lambda st: synth.laplacian_2d(64, st), 64 * 64),
    ("lap3d_20", lambda st: synth.laplacian_3d(20, st), 20 ** 3),
    ("powerlaw", lambda st: synth.powerlaw_csr(10_001, 9_000, 30, st), 9_000),
    ("empty_dup", lambda st: synth.random_csr(1_003, 700, 31, st, 0, 40, 0.3, True), 700),
    ("one_row", lambda st: synth.random_csr(1, 500, 32, st, 300, 300), 500),
    ("all_empty", lambda st: synth.random_csr(45, 10, 33, st, 0, 0), 10),
]


@pytest.mark.parametrize("sigma", [1, 32, 256, 4096])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sell_layout_matches_oracle(case, sigma):
    name, make, n = case
    rp, ci, v = make("f32")
    A = S()(rp.cuda(), ci.cuda(), v.cuda(), n, sigma=sigma)
    torch.cuda.synchronize()
    perm, slen, sptr, cols, mp = oracle.csr_to_sell(rp, ci, 32, sigma)
    m = rp.numel() - 1
    mpad = (m + 31) // 32 * 32
    assert np.array_equal(A.perm.cpu().numpy()[:mpad], perm)
    assert np.array_equal(A.slice_len.cpu().numpy()[:mpad // 32], slen)
    assert np.array_equal(A.slice_ptr.cpu().numpy(), sptr)
    assert np.array_equal(A.cols.cpu().numpy()[:A.total], cols)
    assert np.array_equal(A.map.cpu().numpy()[:A.total], mp)


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("sigma", [1, 256])
@pytest.mark.parametrize("cfg", [None, (64, 0, 1, 0), (512, 7, 8, 1)], ids=str)
def test_sell_spmv_vs_oracle(storage, sigma, cfg):
    for name, make, n in CASES:
        rp, ci, v = make(storage)
        x = synth.uniform(n, 34, storage)
        A = S()(rp.cuda(), ci.cuda(), v.cuda(), n, sigma=sigma)
        y = A.spmv(x.cuda(), cfg=cfg)
        torch.cuda.synchronize()
        ref = oracle.csr_spmv(rp, ci, v, x)
        if storage == "bf16":
            got = host(y)
            scale = oracle.csr_spmv(rp, ci, np.abs(oracle.widen(v)), np.abs(oracle.widen(x)))
            assert np.all(np.abs(got - ref) <= 2 ** -8 * np.abs(ref) + 2 ** -16 * scale + 1e-30), name
        else:
            assert_normwise(host(y), ref, storage, f"{name} sigma={sigma}")


def test_sell_repack_values():
    rp, ci, v = synth.laplacian_2d(40, "f32")
    A = S()(rp.cuda(), ci.cuda(), v.cuda(), 1600, sigma=32)
    v2 = synth.normal((v.numel(),), 35, "f32")
    A.pack(v2.cuda())
    x = synth.uniform(1600, 36, "f32")
    y = A.spmv(x.cuda())
    torch.cuda.synchronize()
    assert_normwise(host(y), oracle.csr_spmv(rp, ci, v2, x), "f32")
