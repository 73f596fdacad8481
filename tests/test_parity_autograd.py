"""Differentiation: autograd Functions whose forward and backward run in the
library's kernels, checked by torch.autograd.gradcheck (central finite
differences in FP64) and against reference gradients built from the FP64
oracle; the CSR transpose against the oracle's stable counting sort."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import assert_normwise, host

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


def AG():
    from paper_1409_0669_gb300 import autograd
    return autograd


def test_gradcheck_fp64_dense_csr_dot():
    ag = AG()
    A = synth.normal((32, 32), 1, "f64").cuda().requires_grad_()
    x = synth.uniform(32, 2, "f64").cuda().requires_grad_()
    assert torch.autograd.gradcheck(ag.gemv, (A, x), eps=1e-6, atol=1e-7, rtol=1e-6)
    rp, ci, v = synth.banded_random_csr(1000, 3, 5, 64, "f64")
    pat = ag.CsrPattern(rp.cuda(), ci.cuda(), 1000)
    vals = v.cuda().requires_grad_()
    xs = synth.uniform(1000, 4, "f64").cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda vv, xx: ag.spmv(pat, vv, xx), (vals, xs), eps=1e-6,
                                    atol=1e-7, rtol=1e-6)
    a = synth.uniform(257, 5, "f64").cuda().requires_grad_()
    b = synth.uniform(257, 6, "f64").cuda().requires_grad_()
    assert torch.autograd.gradcheck(ag.dot, (a, b), eps=1e-6, atol=1e-7, rtol=1e-6)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_gemv_gradients_vs_oracle(storage):
    ag = AG()
    m, n = 300, 517
    A = synth.normal((m, n), 7, storage).cuda().requires_grad_()
    x = synth.uniform(n, 8, storage).cuda().requires_grad_()
    dy = synth.uniform(m, 9, storage).cuda()
    y = ag.gemv(A, x)
    y.backward(dy)
    torch.cuda.synchronize()
    assert_normwise(host(y.detach()), oracle.gemv(A.detach().cpu(), x.detach().cpu(), m, n, n),
                    storage)
    ref_dA = oracle.round_to(oracle.dense_outer(dy.cpu(), x.detach().cpu()).ravel(), storage)
    assert np.array_equal(host(A.grad), ref_dA)                # one rounded product each
    ref_dx = oracle.gemv(A.detach().cpu(), dy.cpu(), n, m, n, "col")
    assert_normwise(host(x.grad), ref_dx, storage)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_spmv_gradients_and_transpose_vs_oracle(storage):
    ag = AG()
    for rp, ci, v, n in ((*synth.laplacian_3d(24, storage), 24 ** 3),
                         (*synth.powerlaw_csr(20_000, 15_000, 10, storage), 15_000),
                         (*synth.random_csr(3000, 2000, 11, storage, 0, 30, 0.2, True), 2000)):
        m = rp.numel() - 1
        pat = ag.CsrPattern(rp.cuda(), ci.cuda(), n)
        cp, ri, perm = pat.transpose()
        ocp, ori, operm = oracle.csr_to_csc(rp, ci, n)
        assert np.array_equal(cp.cpu().numpy(), ocp)
        assert np.array_equal(ri.cpu().numpy(), ori)
        assert np.array_equal(perm.cpu().numpy(), operm)
        vals = v.cuda().requires_grad_()
        x = synth.uniform(n, 12, storage).cuda().requires_grad_()
        dy = synth.uniform(m, 13, storage).cuda()
        y = ag.spmv(pat, vals, x)
        y.backward(dy)
        torch.cuda.synchronize()
        ref_dv = oracle.round_to(oracle.sampled_outer(rp, ci, dy.cpu(), x.detach().cpu()), storage)
        assert np.array_equal(host(vals.grad), ref_dv)
        ref_dx = oracle.csr_spmv(ocp, ori, oracle.widen(v)[operm], dy.cpu())
        assert_normwise(host(x.grad), ref_dx, storage)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_dot_gradients_vs_oracle(storage):
    ag = AG()
    n = 100_003
    x = synth.uniform(n, 14, storage).cuda().requires_grad_()
    y = synth.uniform(n, 15, storage).cuda().requires_grad_()
    s = ag.dot(x, y)
    ds = torch.tensor(1.75, dtype=s.dtype, device="cuda")
    s.backward(ds)
    torch.cuda.synchronize()
    assert np.array_equal(host(x.grad), oracle.round_to(oracle.scale(y.detach().cpu(), 1.75), storage))
    assert np.array_equal(host(y.grad), oracle.round_to(oracle.scale(x.detach().cpu(), 1.75), storage))


def test_differentiation_workload_sizes():
    """The differentiation workload: dense 4096^2 FP32, CSR 3D Laplacian 64^3,
    dot n = 1e7 -- forward and backward against the oracle."""
    ag = AG()
    m = n = 4096
    g = torch.Generator(device="cuda").manual_seed(20)
    A = torch.randn(m, n, generator=g, device="cuda").requires_grad_()
    x = (torch.rand(n, generator=g, device="cuda") * 2 - 1).requires_grad_()
    dy = torch.rand(m, generator=g, device="cuda") * 2 - 1
    ag.gemv(A, x).backward(dy)
    torch.cuda.synchronize()
    rows = np.arange(0, m, 61)
    ref = oracle.dense_outer(dy.cpu(), x.detach().cpu())
    assert np.array_equal(host(A.grad).reshape(m, n)[rows], oracle.round_to(ref[rows].ravel(), "f32").reshape(len(rows), n))
    assert_normwise(host(x.grad), oracle.gemv(A.detach().cpu(), dy.cpu(), n, m, n, "col"), "f32")
    rp, ci, v = synth.laplacian_3d(64, "f32")
    pat = ag.CsrPattern(rp.cuda(), ci.cuda(), 64 ** 3)
    vals = v.cuda().requires_grad_()
    xs = synth.uniform(64 ** 3, 21, "f32").cuda().requires_grad_()
    dys = synth.uniform(64 ** 3, 22, "f32").cuda()
    ag.spmv(pat, vals, xs).backward(dys)
    torch.cuda.synchronize()
    assert np.array_equal(host(vals.grad), oracle.round_to(oracle.sampled_outer(rp, ci, dys.cpu(), xs.detach().cpu()), "f32"))
    # the Laplacian is symmetric: A^T dy = A dy
    assert_normwise(host(xs.grad), oracle.csr_spmv(rp, ci, v, dys.cpu()), "f32")
    a = synth.uniform(10_000_000, 23, "f32").cuda().requires_grad_()
    b = synth.uniform(10_000_000, 24, "f32").cuda().requires_grad_()
    ag.dot(a, b).backward()
    torch.cuda.synchronize()
    assert torch.equal(a.grad, b.detach()) and torch.equal(b.grad, a.detach())


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
@pytest.mark.parametrize("mean_len", [3, 17, 20, 150])
def test_sampled_outer_lane_groups(storage, mean_len):
    """Every lane-group width of the sampled outer product (one thread per row
    for short rows; 8, 16 and 32 lanes for longer ones), ragged row lengths and
    empty rows, bit-exact against the oracle's one rounded product per entry."""
    m = 1537
    rp, ci, _ = synth.random_csr(m, 3001, 40 + mean_len, storage, 0, 2 * mean_len, 0.15, True)
    dy = synth.uniform(m, 41, storage).cuda()
    x = synth.uniform(3001, 42, storage).cuda()
    dv = lak().csr_sampled_outer(rp.cuda(), ci.cuda(), dy, x)
    torch.cuda.synchronize()
    ref = oracle.round_to(oracle.sampled_outer(rp, ci, dy.cpu(), x.cpu()), storage)
    assert np.array_equal(host(dv), ref)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("m,n", [(1, 7), (5000, 33), (700, 4099)])
def test_dense_outer_row_loop(storage, m, n):
    """dense_outer with more rows than row groups (each block walks many rows),
    a column count that is not a multiple of the vector width, and one row."""
    dy = synth.uniform(m, 43, storage).cuda()
    x = synth.uniform(n, 44, storage).cuda()
    dA = lak().dense_outer(dy, x)
    torch.cuda.synchronize()
    ref = oracle.round_to(oracle.dense_outer(dy.cpu(), x.cpu()).ravel(), storage)
    assert np.array_equal(host(dA), ref)


def test_gemv_forward_backward_replays_from_cuda_graphs():
    """The differentiable GEMV's whole forward + backward step captured once into
    a CUDA graph (gradients written into the .grad tensors allocated during
    capture) gives, on every replay with new inputs, the same output and
    gradients bit for bit as the eager calls -- the same kernels in the same
    launch shapes."""
    ag = AG()
    m, n = 300, 517
    A = synth.normal((m, n), 11, "f32").cuda().requires_grad_()
    x = synth.uniform(n, 12, "f32").cuda().requires_grad_()
    dy = synth.uniform(m, 13, "f32").cuda()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            A.grad = x.grad = None
            ag.gemv(A, x).backward(dy)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    A.grad = x.grad = None
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        y_static = ag.gemv(A, x)
        y_static.backward(dy)
    gA_static, gx_static = A.grad, x.grad
    for rep in range(3):
        with torch.no_grad():
            A.copy_(synth.normal((m, n), 20 + rep, "f32").cuda())
            x.copy_(synth.uniform(n, 30 + rep, "f32").cuda())
            dy.copy_(synth.uniform(m, 40 + rep, "f32").cuda())
        g.replay()
        torch.cuda.synchronize()
        y_g, gA, gx = y_static.detach().clone(), gA_static.clone(), gx_static.clone()
        A.grad = x.grad = None
        y_e = ag.gemv(A, x)
        y_e.backward(dy)
        torch.cuda.synchronize()
        assert torch.equal(y_g, y_e.detach())
        assert torch.equal(gA, A.grad) and torch.equal(gx, x.grad)
        assert_normwise(host(y_g), oracle.gemv(A.detach().cpu(), x.detach().cpu(), m, n, n),
                        "f32")
        A.grad, x.grad = gA_static, gx_static      # the graph writes into these
