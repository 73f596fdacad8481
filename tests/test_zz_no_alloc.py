"""vec_dot_noalloc -- the inner product for callers that cannot hand the library
any device scratch memory (their memory manager owns all device buffers, or
they call from another language with no device allocator).  It must give the
same result as vec_dot, which takes a caller-provided workspace, within the
inner-product tolerance, on consecutive calls that share its built-in scratch.

This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.
"""
import ctypes

import pytest
import torch

import oracle
import synth
from checks import TOL, assert_dot, host

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1409_0669_gb300  # noqa: F401  (loads the library)
    from paper_1409_0669_gb300 import _native
    return _native


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16"])
def test_noalloc_matches_vec_dot_on_consecutive_calls(storage):
    nat = _lib()
    lib = nat.load()
    import paper_1409_0669_gb300 as lak
    code = nat.DTYPES[storage]
    stream = torch.cuda.current_stream().cuda_stream
    odt = torch.float64 if storage == "f64" else torch.float32
    # different lengths back to back: the second call reuses the scratch the
    # first one left behind
    for n, seed in ((3_000_017, 1), (1001, 2), (3_000_017, 3)):
        x = synth.uniform(n, seed, storage).cuda()
        y = synth.uniform(n, seed + 50, storage).cuda()
        ref = lak.vec_dot(x, y).item()                       # workspace-based entry point
        for _ in range(2):                                   # two calls in a row
            out = torch.full((1,), float("nan"), dtype=odt, device="cuda")
            st = lib.vec_dot_noalloc(out.data_ptr(), x.data_ptr(), y.data_ptr(), n, code, None,
                                     stream)
            nat.check("vec_dot_noalloc", st)
            torch.cuda.synchronize()
            got = out.item()
            xs, ys = host(x), host(y)
            scale = float((xs * xs).sum() ** 0.5 * (ys * ys).sum() ** 0.5)
            assert abs(got - ref) <= TOL[storage] * scale
            assert_dot(got, oracle.dot(x.cpu(), y.cpu()), xs, ys, storage)


def test_noalloc_rejects_more_blocks_than_its_scratch_holds():
    nat = _lib()
    lib = nat.load()
    n = 10_000_000
    x = torch.ones(n, device="cuda")
    out = torch.zeros(1, device="cuda")
    too_many = nat.LakCfg(128, nat.DOT_NOALLOC_MAX_BLOCKS + 1, 1, 0)
    st = lib.vec_dot_noalloc(out.data_ptr(), x.data_ptr(), x.data_ptr(), n, 0,
                             ctypes.byref(too_many), None)
    assert st == nat.LAK_EINVAL
    assert "built-in scratch" in nat.last_error()
    ok = nat.LakCfg(128, nat.DOT_NOALLOC_MAX_BLOCKS, 1, 0)
    st = lib.vec_dot_noalloc(out.data_ptr(), x.data_ptr(), x.data_ptr(), n, 0, ctypes.byref(ok),
                             None)
    nat.check("vec_dot_noalloc", st)
    torch.cuda.synchronize()
    assert out.item() == float(n)
