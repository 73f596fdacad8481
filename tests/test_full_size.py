"""Parity at the full sweep sizes, in the launch configuration the benchmark
times: whole-vector comparisons for the vector ops (n = 1e8), sampled rows
for 16384^2 GEMV (the oracle recomputes them one by one), and the whole output
for the 3D Laplacian 128^3 and the 2M-row power-law SpMV."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_dot, assert_normwise, assert_reduced_sum, assert_ulp, host

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_vectors_1e8(storage):
    n = 100_000_000
    g = torch.Generator(device="cuda").manual_seed(0)
    dt = synth.torch_dtype(storage)
    y = (torch.rand(n, generator=g, device="cuda", dtype=dt) * 2 - 1)
    z = (torch.rand(n, generator=g, device="cuda", dtype=dt) * 2 - 1)
    x = torch.empty_like(y)
    lk = lak()
    lk.vec_axpy(x, y, z, 0.5)
    d = lk.vec_dot(y, z).item()
    c = torch.empty_like(y)
    lk.vec_copy(c, y)
    torch.cuda.synchronize()
    yc, zc = y.cpu(), z.cpu()
    assert torch.equal(c.cpu(), yc)
    ref = oracle.round_to(oracle.axpy(yc, zc, 0.5), storage)
    assert np.array_equal(host(x), ref)
    assert_dot(d, oracle.dot(yc, zc), yc.double().numpy(), zc.double().numpy(), storage)


@pytest.mark.parametrize("layout", ["row", "col"])
@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_gemv_16384(layout, storage):
    m = n = 16384
    g = torch.Generator(device="cuda").manual_seed(1)
    dt = synth.torch_dtype(storage)
    A = torch.randn(m * n, generator=g, device="cuda", dtype=dt)
    x = torch.rand(n, generator=g, device="cuda", dtype=dt) * 2 - 1
    y = lak().dense_gemv(A, x, m=m, n=n, lda=m if layout == "col" else n, layout=layout)
    torch.cuda.synchronize()
    rows = np.unique(np.concatenate([np.arange(0, 8), np.arange(m - 8, m),
                                     synth.rng(2).integers(0, m, 112)]))
    Ac = A.cpu()
    ref = oracle.gemv_entries(Ac, x.cpu(), rows, n, m if layout == "col" else n, layout)
    assert_normwise(host(y)[rows], ref, storage, f"gemv {layout} 16384^2 (sampled rows)")


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_spmv_laplacian_3d_128(storage):
    rp, ci, v = synth.laplacian_3d(128, storage)
    x = synth.uniform(128 ** 3, 3, storage)
    y = lak().csr_spmv(rp.cuda(), ci.cuda(), v.cuda(), x.cuda())
    torch.cuda.synchronize()
    assert_normwise(host(y), oracle.csr_spmv(rp, ci, v, x), storage, "lap3d 128^3")


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_spmv_powerlaw_2m(storage):
    """The power-law matrix (2M rows, 4..256 entries per row, random columns)
    in the warp-segmented kernel, whole output: FP32 / FP64 norm-wise, BF16 per
    row within one storage ulp plus the FP32 summation bound."""
    rp, ci, v = synth.powerlaw_csr(2_000_000, 2_000_000, 1, storage)
    x = synth.uniform(2_000_000, 4, storage)
    y = lak().csr_spmv(rp.cuda(), ci.cuda(), v.cuda(), x.cuda())
    torch.cuda.synchronize()
    ref = oracle.csr_spmv(rp, ci, v, x)
    if storage == "bf16":
        absref = oracle.csr_spmv(rp, ci, np.abs(oracle.widen(v)), np.abs(oracle.widen(x)))
        assert_reduced_sum(host(y), ref, absref, np.diff(rp.numpy()).astype(np.float64),
                           storage, "power-law 2M")
    else:
        assert_normwise(host(y), ref, storage, "power-law 2M")


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_vectors_1e8_reduced_storage(storage):
    """Update and inner product at n = 1e8 with BF16 / FP16 storage: every
    updated element within one storage ulp of the oracle's value, the dot within
    the inner-product bar."""
    n = 100_000_000
    g = torch.Generator(device="cuda").manual_seed(5)
    dt = synth.torch_dtype(storage)
    y = (torch.rand(n, generator=g, device="cuda", dtype=torch.float32) * 2 - 1).to(dt)
    z = (torch.rand(n, generator=g, device="cuda", dtype=torch.float32) * 2 - 1).to(dt)
    x = torch.empty_like(y)
    lk = lak()
    lk.vec_axpy(x, y, z, 0.5)
    d = lk.vec_dot(y, z).item()
    torch.cuda.synchronize()
    yc, zc = y.cpu(), z.cpu()
    assert_ulp(host(x), oracle.round_to(oracle.axpy(yc, zc, 0.5), storage), storage, 1.0,
               f"axpy {storage} 1e8")
    assert_dot(d, oracle.dot(yc, zc), host(y), host(z), storage)
