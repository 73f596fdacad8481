"""GPU parity of csr_spmv against the FP64 oracle: Laplacian stencils (with
their closed forms), power-law and random rows (empty rows, repeated
columns), every storage type and several launch shapes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_canary, assert_normwise, assert_reduced_sum, canary_buffer, host

pytestmark = pytest.mark.gpu

STORAGES = ["f32", "f64", "bf16", "f16"]


def lak():
    import paper_1409_0669_gb300 as m
    return m


def run(rp, ci, v, x, cfg=None, y=None):
    return lak().csr_spmv(rp.cuda(), ci.cuda(), v.cuda(), x.cuda(), y=y, cfg=cfg)


def check(y_t, ref, storage, what, rp=None, ci=None, v=None, x=None):
    got = host(y_t)
    if storage in ("f32", "f64"):
        assert_normwise(got, ref, storage, what)
    else:
        abs_terms = oracle.csr_spmv(rp, ci, np.abs(oracle.widen(v)), np.abs(oracle.widen(x)))
        nterms = np.diff(rp.numpy()).astype(np.float64)
        assert_reduced_sum(got, ref, abs_terms, nterms, storage, what)


def matrices(storage):
    """(name, (row_ptr, col_idx, vals), number of columns)"""
    yield "lap2d_256", synth.laplacian_2d(256, storage), 256 * 256
    yield "lap3d_32", synth.laplacian_3d(32, storage), 32 ** 3
    yield "powerlaw_20k", synth.powerlaw_csr(20_000, 20_000, 1, storage), 20_000
    yield "random_empty_dup", synth.random_csr(5003, 4001, 2, storage, 0, 40, 0.3, True), 4001
    yield "single_row", synth.random_csr(1, 3000, 3, storage, 2000, 2000), 3000
    yield "long_rows", synth.random_csr(700, 5000, 7, storage, 100, 400), 5000     # vector variant
    yield "batch_like", synth.random_csr(3000, 3000, 8, storage, 5, 64), 3000
    yield "all_empty", synth.random_csr(77, 10, 4, storage, 0, 0), 10


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("cfg", [None, (64, 0, 1, 0), (512, 9, 4, 1), (128, 0, 16, 0),
                                 (96, 0, 2, 1)], ids=str)
def test_spmv(storage, cfg):
    for name, (rp, ci, v), n in matrices(storage):
        x = synth.uniform(n, 5, storage)
        buf, y = canary_buffer(rp.numel() - 1, v.dtype, "cuda")
        run(rp, ci, v, x, cfg, y=y)
        torch.cuda.synchronize()
        ref = oracle.csr_spmv(rp, ci, v, x)
        check(y, ref, storage, f"{name} cfg={cfg}", rp, ci, v, x)
        assert_canary(buf, rp.numel() - 1)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_laplacian_closed_forms(storage):
    N = 256
    rp, ci, v = synth.laplacian_2d(N, storage)
    ones = torch.ones(N * N, dtype=synth.torch_dtype(storage))
    y = host(run(rp, ci, v, ones)).reshape(N, N)
    assert np.all(y[1:-1, 1:-1] == 0) and y.sum() == 4 * N
    assert y[0, 0] == 2 and y[0, 5] == 1
    # eigenvector of the Dirichlet Laplacian: A x = lambda x
    i = np.arange(1, N + 1)
    p, q = 3, 7
    sx = np.sin(p * np.pi * i / (N + 1))
    sy = np.sin(q * np.pi * i / (N + 1))
    xv = (sy[:, None] * sx[None, :]).ravel()
    lam = 4 - 2 * np.cos(p * np.pi / (N + 1)) - 2 * np.cos(q * np.pi / (N + 1))
    xs = synth.to_storage(xv, storage)
    got = host(run(rp, ci, v, xs))
    xq = host(xs)
    tol = 1e-12 if storage == "f64" else 1e-6
    assert np.max(np.abs(got - lam * xq)) <= tol * 8


def test_spmv_transpose_via_csc_matches_dense():
    m, n = 3000, 2000
    rp, ci, v = synth.random_csr(m, n, 6, "f32", 0, 30, 0.1)
    cp, ri, perm = oracle.csr_to_csc(rp, ci, n)
    vt = v[torch.from_numpy(perm)]
    w = synth.uniform(m, 7, "f32")
    got = run(torch.from_numpy(cp), torch.from_numpy(ri), vt, w)
    D = np.zeros((m, n))
    rpn, cin, vn = rp.numpy(), ci.numpy(), v.numpy().astype(np.float64)
    for i in range(m):
        D[i, cin[rpn[i]:rpn[i + 1]]] += vn[rpn[i]:rpn[i + 1]]
    assert_normwise(host(got), D.T @ host(w), "f32")
