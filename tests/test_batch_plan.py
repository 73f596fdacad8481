"""lak_batch_plan is host-only: its work table (unit counts, prefix offsets,
per-instance vector-width decisions) is checked here without a GPU."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def nat():
    import __graft_entry__
    __graft_entry__._build_module().build()
    from paper_1409_0669_gb300 import _native
    _native.load()
    return _native


def plan(nat, op, storage, descs, cfg=None):
    lib = nat.load()
    arr = (type(descs[0]) * len(descs))(*descs)
    info = nat.BatchInfo()
    cptr = ctypes.byref(cfg) if cfg is not None else None
    assert lib.lak_batch_plan(nat.OPS[op], nat.DTYPES[storage], arr, len(descs), cptr, None, 0,
                              ctypes.byref(info)) == 0
    buf = (ctypes.c_uint8 * info.table_bytes)()
    assert lib.lak_batch_plan(nat.OPS[op], nat.DTYPES[storage], arr, len(descs), cptr, buf,
                              info.table_bytes, ctypes.byref(info)) == 0
    raw = bytes(buf)
    offs = np.frombuffer(raw[64:64 + 8 * (len(descs) + 1)], dtype=np.int64)
    return info, offs, raw


def test_axpy_units_and_offsets(nat):
    cfg = nat.LakCfg(512, 0, 16, 0)          # unit = 256 KB of FP32 = 65536 elements
    sizes = [0, 1, 65536, 65537, 200000]
    descs = [nat.AxpyDesc(0x1000 * (i + 1) * 256, 0x2000 * (i + 1) * 256, 0x3000 * (i + 1) * 256,
                          n, 0.5) for i, n in enumerate(sizes)]
    info, offs, _ = plan(nat, "axpy", "f32", descs, cfg)
    assert info.unit_elems == 65536
    assert list(offs) == [0, 0, 1, 2, 4, 8]
    assert info.total_units == 8 and info.workspace_bytes == 0


def test_dot_empty_instances_still_get_a_unit(nat):
    cfg = nat.LakCfg(256, 0, 4, 0)           # unit = 65536 FP32 elements
    descs = [nat.DotDesc(8 * (i + 1), 256 * (i + 1), 512 * (i + 1), n)
             for i, n in enumerate([0, 65536, 65537, 0])]
    info, offs, _ = plan(nat, "dot", "f32", descs, cfg)
    assert list(offs) == [0, 1, 2, 4, 5]
    assert info.workspace_bytes == 65536 + 8 * 5


def test_gemv_rows_per_unit_and_spmv_units(nat):
    cfg = nat.LakCfg(128, 0, 8, 0)           # unit = 65536 entries
    g = [nat.GemvDesc(256, 512, 768, m, n, max(n, 1))
         for m, n in ((2000, 64), (40, 4096), (3, 100000), (0, 5), (7, 0))]
    info, offs, _ = plan(nat, "gemv_row", "f32", g, cfg)
    # rows per unit: 1024 -> 2 units; 16 -> 3 units; 1, rounded up to the 4 rows a lane
    # group takes at once -> 1 unit; none; n = 0: all 7 -> 1
    assert list(offs) == [0, 2, 5, 6, 6, 7]
    # CSR: one block's rows (64) per unit
    c = [nat.CsrDesc(256, 512, 768, 1024, 1280, m, m, 5 * m) for m in (1, 64, 65, 1000)]
    info, offs, _ = plan(nat, "spmv", "f32", c, nat.LakCfg(64, 0, 4, 0))
    assert list(offs) == [0, 1, 2, 4, 20]
    assert info.workspace_bytes == 65536          # the zero-filled ticket counters


def test_gemv_plan_rejects_blocks_over_128(nat):
    g = [nat.GemvDesc(256, 512, 768, 100, 100, 100)]
    with pytest.raises(AssertionError):
        plan(nat, "gemv_row", "f32", g, nat.LakCfg(256, 0, 4, 0))
    info, offs, _ = plan(nat, "gemv_row", "f32", g, nat.LakCfg(128, 0, 4, 0))
    assert info.cfg.block == 128


def test_plan_rejects_bad_input(nat):
    lib = nat.load()
    info = nat.BatchInfo()
    d = (nat.AxpyDesc * 1)(nat.AxpyDesc(0, 0, 0, -5, 1.0))
    assert lib.lak_batch_plan(nat.OPS["axpy"], 0, d, 1, None, None, 0, ctypes.byref(info)) == -1
    assert lib.lak_batch_plan(nat.OPS["copy"], 0, d, 1, None, None, 0, ctypes.byref(info)) == -1
    assert lib.lak_batch_plan(nat.OPS["axpy"], 9, d, 1, None, None, 0, ctypes.byref(info)) == -2
    many = (nat.DotDesc * 20000)()
    assert lib.lak_batch_plan(nat.OPS["dot"], 0, many, 20000, None, None, 0,
                              ctypes.byref(info)) == -1
    assert "dot instances" in nat.last_error()


def test_batch_default_cfg_comes_from_the_installed_entry(nat, tmp_path, monkeypatch):
    """A plan without a cfg takes the entry installed with
    lak_set_batch_default_cfg (as the autotuner's cache installs it), falls back
    to the built-in shape when the entry is removed, and an explicit cfg still
    wins; invalid entries are refused."""
    lib = nat.load()
    g = [nat.GemvDesc(256, 512, 768, 100, 1000, 1000)]
    builtin = plan(nat, "gemv_row", "f32", g)[0].cfg.as_tuple()
    try:
        tuned = nat.LakCfg(96, 152 * 4, 4, 1)
        assert lib.lak_set_batch_default_cfg(nat.OPS["gemv_row"], nat.DTYPES["f32"],
                                             ctypes.byref(tuned)) == 0
        assert plan(nat, "gemv_row", "f32", g)[0].cfg.as_tuple() == (96, 608, 4, 1)
        # other storage types and ops keep their own defaults
        assert plan(nat, "gemv_row", "f64", g)[0].cfg.as_tuple() != (96, 608, 4, 1)
        explicit = nat.LakCfg(64, 0, 8, 0)
        assert plan(nat, "gemv_row", "f32", g, explicit)[0].cfg.as_tuple() == (64, 0, 8, 0)
        for bad in (nat.LakCfg(256, 0, 4, 0), nat.LakCfg(48, 0, 4, 0), nat.LakCfg(64, -1, 4, 0),
                    nat.LakCfg(64, 0, 3, 0), nat.LakCfg(64, 0, 4, 2)):
            assert lib.lak_set_batch_default_cfg(nat.OPS["gemv_row"], nat.DTYPES["f32"],
                                                 ctypes.byref(bad)) == nat.LAK_EINVAL
        assert lib.lak_set_batch_default_cfg(nat.OPS["copy"], 0, None) == nat.LAK_EINVAL
        # the autotuner's cache file format, installed through apply_cache
        import json

        import paper_1409_0669_gb300 as lak
        from paper_1409_0669_gb300 import autotune
        monkeypatch.setattr(autotune, "cache_key", lambda: "TEST GPU|sms=152")
        monkeypatch.setattr(lak, "_user_batch_defaults", set())     # leave no trace
        path = tmp_path / "cache.json"
        path.write_text(json.dumps({"TEST GPU|sms=152": {"batch:gemv_row:f32": [32, 0, 8, 0]},
                                    "OTHER|sms=1": {"batch:gemv_row:f32": [128, 0, 2, 0]}}))
        assert autotune.apply_cache(str(path), only_batch=True) == 1
        assert plan(nat, "gemv_row", "f32", g)[0].cfg.as_tuple() == (32, 0, 8, 0)
    finally:
        assert lib.lak_set_batch_default_cfg(nat.OPS["gemv_row"], nat.DTYPES["f32"], None) == 0
    assert plan(nat, "gemv_row", "f32", g)[0].cfg.as_tuple() == builtin


def test_gemv_long_rows_period_and_units(nat):
    """Rows of lane groups of 8+ lanes are taken R at a time by one group, R rows
    a stride P apart that start at the same offset modulo the access width: P is
    the smallest such stride, and a unit holds a whole number of R * P rows."""
    import struct
    cases = [  # (n, lda, vec) -> (lanes per row, period, rows per group)
        (1001, 1001, 4, 32, 4, 4),      # 4004 B rows, 16-byte accesses: P = 4, R = 4
        (1002, 1002, 4, 32, 2, 4),      # 4008 B: P = 2
        (1024, 1024, 4, 32, 1, 4),      # 4096 B: P = 1
        (300, 301, 4, 16, 4, 4),        # 16 lanes per row
        (100, 101, 4, 8, 4, 4),         # 8 lanes per row
        (2049, 2049, 8, 32, 8, 4),      # 32-byte accesses: P = 8
        (2050, 2052, 8, 32, 2, 4),      # 8208 B rows: P = 2
        (300, 300, 8, 8, 2, 4),         # 8 lanes per row at 32 bytes: 1200 B rows, P = 2
    ]
    for n, lda, vec, G, P, R in cases:
        m = 333
        g = [nat.GemvDesc(256, 512, 768, m, n, lda)]
        info, offs, raw = plan(nat, "gemv_row", "f32", g, nat.LakCfg(128, 0, vec, 0))
        base = (64 + 8 * 2 + 15) // 16 * 16
        rpu, vec_ok, group, period = struct.unpack_from("<qiii", raw, base + 48)
        assert group == G and period == P, (n, lda, vec, group, period)
        assert rpu % (R * P) == 0 and rpu >= min(65536 // n, m)
        assert list(offs) == [0, -(-m // rpu)]
    # 4 lanes per row (short rows at 32-byte accesses) take 4 rows at a time too
    info, offs, raw = plan(nat, "gemv_row", "f32", [nat.GemvDesc(256, 512, 768, 50, 100, 101)],
                           nat.LakCfg(128, 0, 8, 0))
    rpu, _, group, period = struct.unpack_from("<qiii", raw, (64 + 16 + 15) // 16 * 16 + 48)
    assert group == 4 and period == 8 and rpu % 32 == 0
    # FP64 at 16 elements per access (two 32-byte loads): 1-2 lanes per short row,
    # one row at a time
    info, offs, raw = plan(nat, "gemv_row", "f64", [nat.GemvDesc(256, 512, 768, 50, 100, 101)],
                           nat.LakCfg(128, 0, 16, 0))
    rpu, _, group, period = struct.unpack_from("<qiii", raw, (64 + 16 + 15) // 16 * 16 + 48)
    assert group < 4 and period == 1


def test_shipped_defaults_leave_caller_settings_alone(nat, tmp_path, monkeypatch):
    """The batched runner installs the shipped autotuned defaults when the first
    batch is planned, but not over a default the caller set before."""
    import json

    import paper_1409_0669_gb300 as lak
    from paper_1409_0669_gb300 import autotune
    from paper_1409_0669_gb300 import batch as B
    lib = nat.load()
    monkeypatch.setattr(autotune, "cache_key", lambda: "TEST GPU|sms=152")
    monkeypatch.setattr(B.torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(B, "_installed", set())
    monkeypatch.setattr(lak, "_user_batch_defaults", set())
    path = tmp_path / "shipped.json"
    path.write_text(json.dumps({"TEST GPU|sms=152": {"batch:gemv_row:f32": [32, 0, 8, 0],
                                                     "batch:axpy:f32": [256, 0, 4, 0]}}))
    g = [nat.GemvDesc(256, 512, 768, 100, 1000, 1000)]
    a = [nat.AxpyDesc(256, 512, 768, 1000, 0.5)]
    try:
        lak.set_batch_default_cfg("gemv_row", "f32", (64, 0, 4, 0))     # the caller's
        assert B.install_tuned_defaults(str(path)) == 1                 # axpy only
        assert plan(nat, "gemv_row", "f32", g)[0].cfg.as_tuple() == (64, 0, 4, 0)
        assert plan(nat, "axpy", "f32", a)[0].cfg.as_tuple() == (256, 0, 4, 0)
        assert B.install_tuned_defaults(str(path)) == 0                 # once per device
    finally:
        for op in ("gemv_row", "axpy"):
            assert lib.lak_set_batch_default_cfg(nat.OPS[op], nat.DTYPES["f32"], None) == 0
