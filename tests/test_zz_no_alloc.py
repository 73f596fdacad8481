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
from checks import assert_dot, host

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1409_0669_gb300  # noqa: F401  (loads the library)
    from paper_1409_0669_gb300 import _native
    return _native


@pytest.mark.parametrize("offset", [0, 1], ids=["aligned", "offset1"])
@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16"])
def test_noalloc_matches_vec_dot_on_consecutive_calls(storage, offset):
    """Same bits as vec_dot (both plan the same launch, so the blocks sum in
    the same order), two calls in a row at each length, lengths changing from
    call to call so that each call meets the scratch the previous one left.
    offset = 1 starts both operands one element past an aligned address, where
    the launch narrows its vector width and adds a scalar prologue."""
    nat = _lib()
    lib = nat.load()
    import paper_1409_0669_gb300 as lak
    code = nat.DTYPES[storage]
    stream = torch.cuda.current_stream().cuda_stream
    odt = torch.float64 if storage == "f64" else torch.float32
    for n, seed in ((3_000_017, 1), (1001, 2), (0, 3), (1, 4), (33, 5), (3_000_017, 6)):
        xb = synth.uniform(n + offset, seed, storage).cuda()
        yb = synth.uniform(n + offset, seed + 50, storage).cuda()
        x, y = xb[offset:], yb[offset:]
        ref = lak.vec_dot(x, y).item()                       # workspace-based entry point
        for _ in range(2):                                   # two calls in a row
            out = torch.full((1,), float("nan"), dtype=odt, device="cuda")
            st = lib.vec_dot_noalloc(out.data_ptr(), x.data_ptr() if n else None,
                                     y.data_ptr() if n else None, n, code, None, stream)
            nat.check("vec_dot_noalloc", st)
            torch.cuda.synchronize()
            got = out.item()
            assert got == ref, (n, got, ref)                 # bit-identical to vec_dot
            if n == 0:
                assert got == 0.0
                continue
            xs, ys = host(x), host(y)
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
