"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point that include/lak.h declares; argument checks that return
before any CUDA call behave as documented (no compute without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lak.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    from paper_1409_0669_gb300 import _native
    return _native.load(path)


def declared_symbols():
    text = open(HEADER).read()
    return re.findall(r"LAK_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("vec_axpy", "vec_dot", "dense_gemv", "csr_spmv"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1409_0669_gb300 import _native
    so = _native.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_symbols():
        assert name in exported, name
        assert getattr(lib, name) is not None
    assert set(declared_symbols()) == set(_native.EXPORTS)


def test_only_the_abi_is_exported(lib):
    from paper_1409_0669_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    text_syms = {l.split()[-1] for l in out.splitlines() if l.split()[1] in ("T", "t")}
    ours = {s for s in text_syms if not s.startswith("_")}
    assert ours <= set(declared_symbols()) | {"_init", "_fini"}, ours - set(declared_symbols())


def test_abi_version(lib):
    assert lib.lak_abi_version() == 1


def _err(lib):
    return lib.lak_last_error().decode()


def test_host_side_argument_checks(lib):
    from paper_1409_0669_gb300._native import LakCfg, LAK_EINVAL, LAK_EDTYPE, LAK_ELAYOUT, LAK_OK
    # negative length
    assert lib.vec_axpy(None, None, None, 1.0, -1, 0, None, None) == LAK_EINVAL
    assert "n=-1" in _err(lib)
    # unknown dtype
    assert lib.vec_copy(None, None, 4, 7, None, None) == LAK_EDTYPE
    # empty vectors are a no-op, even with NULL pointers
    assert lib.vec_copy(None, None, 0, 0, None, None) == LAK_OK
    assert lib.vec_axpy(None, None, None, 2.0, 0, 1, None, None) == LAK_OK
    # bad configurations
    for bad in (LakCfg(48, 0, 0, 0), LakCfg(1024, 0, 0, 0), LakCfg(256, -1, 0, 0),
                LakCfg(256, 0, 3, 0), LakCfg(256, 0, 4, 2)):
        assert lib.vec_copy(None, None, 4, 0, ctypes.byref(bad), None) == LAK_EINVAL
    # NULL pointers with work to do
    assert lib.vec_copy(None, None, 4, 0, None, None) == LAK_EINVAL
    # dense_gemv: layout and leading dimension
    assert lib.dense_gemv(None, None, None, 4, 4, 4, 5, 0, None, 0, None, None) == LAK_ELAYOUT
    assert lib.dense_gemv(None, None, None, 4, 8, 4, 0, 0, None, 0, None, None) == LAK_EINVAL
    assert "lda=4" in _err(lib)
    assert lib.dense_gemv(None, None, None, 8, 4, 4, 1, 0, None, 0, None, None) == LAK_EINVAL
    assert lib.dense_gemv(None, None, None, 0, 4, 4, 0, 0, None, 0, None, None) == LAK_OK
    # csr_spmv: sizes
    assert lib.csr_spmv(None, None, None, None, None, -1, 3, 0, 0, None, None) == LAK_EINVAL
    assert lib.csr_spmv(None, None, None, None, None, 0, 3, 0, 0, None, None) == LAK_OK
    assert lib.csr_spmv(None, None, None, None, None, 3, 3, 1 << 31, 0, None, None) == LAK_EINVAL
    # misaligned element pointers are rejected (an FP32 element at an odd address)
    assert lib.vec_copy(ctypes.c_void_p(0x1001), ctypes.c_void_p(0x2000), 4, 0, None,
                        None) == LAK_EINVAL
    # default-configuration table
    assert lib.lak_set_default_cfg(9, 0, None) == LAK_EINVAL
    assert lib.lak_set_default_cfg(0, 9, None) == LAK_EDTYPE
    assert lib.lak_set_default_cfg(0, 0, ctypes.byref(LakCfg(0, 0, 0, 0))) == LAK_EINVAL
    assert lib.lak_set_default_cfg(0, 0, ctypes.byref(LakCfg(128, 0, 4, 1))) == LAK_OK
    assert lib.lak_set_default_cfg(0, 0, None) == LAK_OK


def test_size_buckets(lib):
    """Bucket = algorithmic bytes against 8 / 64 / 512 MiB (host only)."""
    from paper_1409_0669_gb300._native import LAK_EINVAL, LAK_EDTYPE, LakCfg
    MiB = 1 << 20
    # copy / dot: 2 n s bytes; axpy 3 n s
    for op, k in ((0, 2), (2, 2), (1, 3)):
        for s, dt in ((4, 0), (8, 1), (2, 2)):
            for bound, b in ((8 * MiB, 1), (64 * MiB, 2), (512 * MiB, 3)):
                n = -(-bound // (k * s))             # first n at or above the bound
                assert lib.lak_size_bucket(op, dt, n, n, 0) == b, (op, dt, n)
                if (n - 1) * k * s < bound:
                    assert lib.lak_size_bucket(op, dt, n - 1, n - 1, 0) == b - 1
    assert lib.lak_size_bucket(0, 0, 0, 0, 0) == 0
    # dense GEMV: (mn + m + n) s
    assert lib.lak_size_bucket(3, 1, 2048, 2048, 0) == 1       # 33.6 MB
    assert lib.lak_size_bucket(4, 0, 16384, 16384, 0) == 3     # 1.07 GB
    assert lib.lak_size_bucket(3, 0, 4096, 4096, 0) == 2       # 67 MB
    # CSR: nnz (s + 4) + (m + 1) 4 + (m + n) s -- the 3D Laplacian 128^3 in FP32
    assert lib.lak_size_bucket(5, 0, 128 ** 3, 128 ** 3, 14_581_760) == 2
    assert lib.lak_size_bucket(5, 0, 256 ** 2, 256 ** 2, 326_656) == 0
    assert lib.lak_size_bucket(7, 0, 1, 1, 0) == LAK_EINVAL
    assert lib.lak_size_bucket(0, 9, 1, 1, 0) == LAK_EDTYPE
    assert lib.lak_size_bucket(0, 0, -1, 1, 0) == LAK_EINVAL
    # per-bucket defaults: bucket range is -1 (all) .. 3
    cfg = ctypes.byref(LakCfg(128, 0, 4, 0))
    assert lib.lak_set_default_cfg_bucket(0, 0, 4, cfg) == LAK_EINVAL
    assert lib.lak_set_default_cfg_bucket(0, 0, -2, cfg) == LAK_EINVAL
    for b in (-1, 0, 3):
        assert lib.lak_set_default_cfg_bucket(0, 0, b, cfg) == 0
    assert lib.lak_set_default_cfg_bucket(0, 0, -1, None) == 0


def test_bucket_choice_keeps_best_worst_case():
    """autotune.choose_per_bucket: per bucket, the config with the best worst
    ratio over that bucket's sizes (host logic, made-up timings)."""
    from paper_1409_0669_gb300.autotune import choose_per_bucket
    res = {
        100: [{"cfg": [64, 0, 1, 0], "us": 5.0}, {"cfg": [128, 0, 2, 0], "us": 5.5},
              {"cfg": [256, 0, 4, 0], "us": 9.0}],
        200: [{"cfg": [64, 0, 1, 0], "us": 12.0}, {"cfg": [128, 0, 2, 0], "us": 8.5},
              {"cfg": [256, 0, 4, 0], "us": 8.0}],
        900: [{"cfg": [64, 0, 1, 0], "us": 50.0}, {"cfg": [256, 0, 4, 0], "us": 30.0}],
    }
    per = choose_per_bucket(res, {100: 1, 200: 1, 900: 2})
    # bucket 1: [128,0,2,0] has worst ratio min(5/5.5, 8/8.5) = 0.909; [64..] 0.667; [256..] 0.556
    assert per[1]["cfg"] == [128, 0, 2, 0]
    assert abs(per[1]["worst_ratio"] - 5.0 / 5.5) < 1e-12
    assert per[1]["sizes"] == [100, 200]
    assert per[2]["cfg"] == [256, 0, 4, 0] and per[2]["worst_ratio"] == 1.0


def test_python_binding_imports_and_fails_loudly_without_library(tmp_path):
    from paper_1409_0669_gb300 import _native
    with pytest.raises(ImportError, match="no CPU fallback"):
        _native.load(str(tmp_path / "missing.so"))


class _FakeCudaTensor:
    """Just enough of a CUDA tensor for the binding's operand checks."""
    is_cuda = True

    def __init__(self, index, n=4):
        import torch
        self.device = torch.device("cuda", index)
        self._n = n

    def numel(self):
        return self._n

    def dim(self):
        return 1

    def stride(self, d):
        return 1

    def data_ptr(self):
        return 0x7000_0000_0000


def test_binding_refuses_operands_on_another_device(lib, monkeypatch):
    """The library launches on the current device; the binding refuses an
    operand on any other device instead of passing its address to a kernel
    that runs elsewhere (no GPU needed: the check runs before any call)."""
    import paper_1409_0669_gb300 as m
    monkeypatch.setattr(m, "_current_device", lambda: 0)
    assert m._dev_ptr(_FakeCudaTensor(0), "x") == 0x7000_0000_0000
    with pytest.raises(ValueError, match="cuda:1 but the current device is cuda:0"):
        m._dev_ptr(_FakeCudaTensor(1), "x")
    with pytest.raises(ValueError, match="cuda:1"):
        m._vec_arg(_FakeCudaTensor(1), "y")
    with pytest.raises(ValueError):
        m._on_current_device(_FakeCudaTensor(0), _FakeCudaTensor(1))
    m._on_current_device(_FakeCudaTensor(0), _FakeCudaTensor(1, n=0), None)   # empty: no address
    from paper_1409_0669_gb300 import batch
    with pytest.raises(ValueError, match="cuda:1"):
        batch._ptr(_FakeCudaTensor(1))


def test_every_entry_point_cites_the_paper_or_says_it_has_no_counterpart():
    """Each declaration's own comment (the nearest one before it) cites the
    paper's section that defines the operation, or states that the paper has
    no counterpart."""
    text = open(HEADER).read()
    missing = []
    for m in re.finditer(r"LAK_API\s+[\w\s\*]+?\b(\w+)\s*\(", text):
        before = text[:m.start()]
        comment = before[before.rfind("/*"):]
        if not re.search(r"Sec\.|counterpart", comment):
            missing.append(m.group(1))
    assert not missing, missing
