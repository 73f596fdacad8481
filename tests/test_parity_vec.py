"""GPU parity of the vector kernels (copy, update, inner product) against the
FP64 oracle, through the C ABI, over storage types, ragged and misaligned
lengths, both loop skeletons and several launch shapes."""
import numpy as np
import pytest
import torch

import oracle
import synth
from checks import (assert_canary, assert_dot, assert_normwise, assert_ulp, canary_buffer, host)

pytestmark = pytest.mark.gpu

STORAGES = ["f32", "f64", "bf16", "f16"]
SIZES = [1, 3, 31, 32, 33, 1023, 65537, 1_000_003]
CFGS = [None, (128, 0, 1, 0), (256, 7, 16, 1), (64, 1, 4, 0), (512, 0, 8, 1), (96, 300, 2, 0)]


def lak():
    import paper_1409_0669_gb300 as m
    return m


def dev_vec(n, seed, storage, offset=0):
    """A device vector whose data starts `offset` elements into its allocation."""
    v = synth.uniform(n + offset, seed, storage).cuda()
    return v[offset:]


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("cfg", CFGS, ids=str)
def test_copy(storage, n, cfg):
    y = dev_vec(n, 1, storage)
    buf, x = canary_buffer(n, y.dtype, y.device)
    lak().vec_copy(x, y, cfg=cfg)
    torch.cuda.synchronize()
    assert torch.equal(x.cpu().view(torch.uint8), y.cpu().view(torch.uint8))
    assert_canary(buf, n)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("cfg", CFGS, ids=str)
def test_axpy_half_alpha(storage, n, cfg):
    y = dev_vec(n, 2, storage)
    z = dev_vec(n, 3, storage)
    buf, x = canary_buffer(n, y.dtype, y.device)
    lak().vec_axpy(x, y, z, 0.5, cfg=cfg)
    torch.cuda.synchronize()
    ref = oracle.round_to(oracle.axpy(y.cpu(), z.cpu(), 0.5), storage)
    got = host(x)
    if storage in ("f32", "f64"):
        assert np.array_equal(got, ref), "alpha = 0.5 must be bit-exact"
    else:
        assert_ulp(got, ref, storage, 1.0, "axpy")
    assert_canary(buf, n)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("n", [33, 65537, 1_000_003])
def test_axpy_general_alpha(storage, n):
    alpha = -1.3718
    y = dev_vec(n, 4, storage)
    z = dev_vec(n, 5, storage)
    x = torch.empty_like(y)
    lak().vec_axpy(x, y, z, alpha)
    torch.cuda.synchronize()
    a_used = float(np.float32(alpha)) if storage != "f64" else alpha
    zv = host(z)
    ref = oracle.axpy(y.cpu(), z.cpu(), a_used)
    got = host(x)
    if storage == "f64":
        bound = 2.0 ** -52 * (np.abs(ref) + np.abs(a_used * zv))
        assert np.all(np.abs(got - ref) <= bound)
        assert_normwise(got, ref, storage)
    else:
        assert_ulp(got, oracle.round_to(ref, storage), storage, 1.0, "axpy")


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("offsets", [(1, 1, 1), (1, 0, 0), (0, 3, 1), (5, 5, 5)], ids=str)
def test_axpy_misaligned(storage, offsets):
    n = 100_003
    ox, oy, oz = offsets
    y = dev_vec(n, 6, storage, oy)
    z = dev_vec(n, 7, storage, oz)
    xb = torch.zeros(n + ox, dtype=y.dtype, device="cuda")
    x = xb[ox:]
    lak().vec_axpy(x, y, z, 0.5)
    torch.cuda.synchronize()
    ref = oracle.round_to(oracle.axpy(y.cpu(), z.cpu(), 0.5), storage)
    assert np.array_equal(host(x), ref)
    if ox:
        assert torch.all(xb[:ox] == 0)


def test_axpy_in_place():
    n = 70_001
    y = dev_vec(n, 8, "f32")
    z = dev_vec(n, 9, "f32")
    ref = oracle.round_to(oracle.axpy(y.cpu(), z.cpu(), 0.5), "f32")
    lak().vec_axpy(y, y, z, 0.5)          # x == y
    torch.cuda.synchronize()
    assert np.array_equal(host(y), ref)


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("cfg", CFGS, ids=str)
def test_dot(storage, n, cfg):
    x = dev_vec(n, 10, storage)
    y = dev_vec(n, 11, storage)
    out = lak().vec_dot(x, y, cfg=cfg)
    torch.cuda.synchronize()
    ref = oracle.dot(x.cpu(), y.cpu())
    assert_dot(float(out.item()), ref, host(x), host(y), storage, f"dot n={n}")


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_dot_closed_forms(storage):
    m = lak()
    dt = synth.torch_dtype(storage)
    for n in (1, 1000, 65536, 10_000_019):
        ones = torch.ones(n, dtype=dt, device="cuda")
        assert m.vec_dot(ones, ones).item() == float(n)          # exact
    a = torch.arange(1, 100_001, dtype=dt, device="cuda")
    s = m.vec_dot(a, torch.ones_like(a)).item()
    exact = 100_000 * 100_001 / 2
    if storage == "f64":
        assert s == exact
    else:                     # 5000050000 is not a float32; FP32 partials round
        assert abs(s - exact) <= 1e-5 * float(torch.linalg.norm(a.double())) * 100_000 ** 0.5
    alt = torch.tensor([1.0, -1.0] * 5000 + [1.0], dtype=dt, device="cuda")
    assert m.vec_dot(alt, torch.ones_like(alt)).item() == 1.0
    x = dev_vec(4097, 12, storage)
    for k in (0, 2048, 4096):
        e = torch.zeros_like(x)
        e[k] = 1
        assert m.vec_dot(x, e).item() == x[k].item()


def test_dot_deterministic_symmetric_and_workspace_reuse():
    m = lak()
    n = 3_000_017
    x = dev_vec(n, 13, "f32")
    y = dev_vec(n, 14, "f32")
    ws = torch.zeros(m.vec_dot_workspace(n, "f32"), dtype=torch.uint8, device="cuda")
    outs = [m.vec_dot(x, y, workspace=ws).item() for _ in range(20)]
    assert len(set(outs)) == 1, "same configuration must give the same bits"
    assert m.vec_dot(y, x, workspace=ws).item() == outs[0]
    # the workspace counter is back at zero after each call
    assert int(ws[:4].cpu().view(torch.int32).item()) == 0
    # interleave sizes on one workspace
    for k in (5, 1_000_000, 17, n):
        r = m.vec_dot(x[:k], y[:k], workspace=ws).item()
        assert_dot(r, oracle.dot(x[:k].cpu(), y[:k].cpu()), host(x[:k]), host(y[:k]), "f32")


def test_dot_empty_and_errors():
    m = lak()
    e = torch.empty(0, device="cuda")
    out = torch.full((1,), 7.0, device="cuda")
    m.vec_dot(e, e, out=out)
    assert out.item() == 0.0
    x = dev_vec(1000, 15, "f32")
    small = torch.zeros(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.LakError, match="LAK_EWORKSPACE"):
        m.vec_dot(x, x, workspace=small)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_reduced_storage_error_vs_fp32_data(storage):
    """Error of reduced-precision storage against the oracle on the ORIGINAL
    FP32 data (quantisation included) stays within 1e-2 norm-wise."""
    n = 1_000_003
    x32 = synth.uniform(n, 16, "f32")
    y32 = synth.uniform(n, 17, "f32")
    xs, ys = x32.to(synth.torch_dtype(storage)).cuda(), y32.to(synth.torch_dtype(storage)).cuda()
    m = lak()
    d = m.vec_dot(xs, ys).item()
    ref = oracle.dot(x32, y32)
    assert abs(d - ref) <= 1e-2 * np.linalg.norm(x32.numpy()) * np.linalg.norm(y32.numpy())
    out = torch.empty_like(xs)
    m.vec_axpy(out, xs, ys, 0.5)
    ref_x = oracle.axpy(x32, y32, 0.5)
    err = np.linalg.norm(host(out) - ref_x) / np.linalg.norm(ref_x)
    assert err <= 1e-2


def test_shared_workspace_across_ops_and_shapes():
    """One workspace serves dot and split-K column-major GEMV calls of changing
    shapes: scratch data never lands on another call's counters."""
    m = lak()
    ws = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    x = dev_vec(2_000_003, 20, "f32")
    y = dev_vec(2_000_003, 21, "f32")
    for (rows, cols) in ((96, 50_000), (4096, 64), (700, 9000), (33, 20_000)):
        A = synth.normal((cols, rows), rows + cols, "f32").cuda()      # A^T stored row-major
        xv = dev_vec(cols, 22, "f32")
        for _ in range(3):
            d = m.vec_dot(x, y, workspace=ws).item()
            assert_dot(d, oracle.dot(x.cpu(), y.cpu()), host(x), host(y), "f32")
            g = m.dense_gemv(A.t(), xv, workspace=ws)                     # column-major view
            torch.cuda.synchronize()
            assert_normwise(host(g), oracle.gemv(A.cpu(), xv.cpu(), rows, cols, rows, "col"),
                            "f32", f"gemv col {rows}x{cols}")
    assert torch.all(ws[:65536] == 0), "counter area must be left zero"
