"""vec_dot_sparse (sum_k vals[k] * y[idx[k]]) against the FP64 oracle: every
storage type, empty / tiny / ragged / multi-wave lengths, repeated indices,
misaligned values and indices (the scalar prologue and narrower packs), every
vector width and both increments, exact integer sums, and the power-law
matrix's own column indices at full size."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_dot, host

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


def _case(nnz, n, storage, seed):
    g = synth.rng(seed)
    idx = torch.from_numpy(g.integers(0, n, nnz).astype(np.int32))
    vals = synth.uniform(nnz, seed + 1, storage)
    y = synth.uniform(n, seed + 2, storage)
    return vals, idx, y


def _check(out, vals, idx, y, storage, what):
    ref = oracle.sparse_dot(vals, idx, y)
    gathered = host(y)[idx.numpy()] if idx.numel() else np.zeros(0)
    assert_dot(float(out.item()), ref, host(vals), gathered, storage, what)


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("nnz", [0, 1, 7, 33, 1000, 65537, 1_000_003])
def test_sparse_dot_vs_oracle(storage, nnz):
    vals, idx, y = _case(nnz, 50_000, storage, 300 + nnz % 97)
    out = lak().vec_dot_sparse(vals.cuda(), idx.cuda(), y.cuda())
    torch.cuda.synchronize()
    if nnz == 0:
        assert float(out.item()) == 0.0
    else:
        _check(out, vals, idx, y, storage, f"nnz={nnz}")


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("off_v,off_i", [(0, 0), (1, 0), (0, 1), (3, 5), (2, 2)])
def test_sparse_dot_misaligned(storage, off_v, off_i):
    nnz = 100_001
    vals, idx, y = _case(nnz + 8, 9999, storage, 311)
    v = vals.cuda()[off_v:off_v + nnz]
    i = idx.cuda()[off_i:off_i + nnz]
    out = lak().vec_dot_sparse(v, i, y.cuda())
    torch.cuda.synchronize()
    _check(out, vals[off_v:off_v + nnz], idx[off_i:off_i + nnz], y, storage,
           f"offsets {off_v},{off_i}")


@pytest.mark.parametrize("vec", [1, 2, 4, 8])
@pytest.mark.parametrize("inc", [0, 1])
@pytest.mark.parametrize("block,grid", [(64, 0), (256, 37), (512, 1)])
def test_sparse_dot_configs(vec, inc, block, grid):
    vals, idx, y = _case(77_777, 3000, "f32", 320)
    out = lak().vec_dot_sparse(vals.cuda(), idx.cuda(), y.cuda(), cfg=(block, grid, vec, inc))
    torch.cuda.synchronize()
    _check(out, vals, idx, y, "f32", f"cfg {(block, grid, vec, inc)}")


def test_sparse_dot_exact_integers_and_repeats():
    """Small integers: every partial sum is exact in FP32, so the result is the
    exact integer; one index repeated 1000 times counts 1000 times."""
    g = synth.rng(321)
    nnz = 200_000
    idx = torch.from_numpy(g.integers(0, 4096, nnz).astype(np.int32))
    idx[:1000] = 17
    vals = torch.from_numpy(g.integers(-3, 4, nnz).astype(np.float32))
    y = torch.from_numpy(g.integers(-3, 4, 4096).astype(np.float32))
    out = lak().vec_dot_sparse(vals.cuda(), idx.cuda(), y.cuda())
    torch.cuda.synchronize()
    exact = int((vals.numpy().astype(np.int64) * y.numpy().astype(np.int64)[idx.numpy()]).sum())
    assert float(out.item()) == float(exact)


def test_sparse_dot_is_the_csr_gather_at_full_size():
    """On the 2M-row power-law matrix's own (vals, col_idx): the sum of all
    entries of A x, i.e. sum_i (A x)_i = sum_k v_k x[c_k] (the oracle computes
    it in FP64; FP32 kernel within the dot bound)."""
    rp, ci, v = synth.powerlaw_csr(2_000_000, 2_000_000, 1, "f32")
    x = synth.uniform(2_000_000, 322, "f32")
    out = lak().vec_dot_sparse(v.cuda(), ci.cuda(), x.cuda())
    torch.cuda.synchronize()
    _check(out, v, ci, x, "f32", "power-law 2M")


def test_sparse_dot_argument_errors():
    from paper_1409_0669_gb300._native import LakError
    m = lak()
    v = torch.ones(10, device="cuda")
    with pytest.raises(ValueError):
        m.vec_dot_sparse(v, torch.zeros(9, dtype=torch.int32, device="cuda"), v)
    with pytest.raises(TypeError):
        m.vec_dot_sparse(v, torch.zeros(10, dtype=torch.int64, device="cuda"), v)
    with pytest.raises(LakError):
        m.vec_dot_sparse(v, torch.zeros(10, dtype=torch.int32, device="cuda"), v[:0])
