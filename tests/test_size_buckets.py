"""Per-size-bucket launch defaults on the device: the configuration a call
resolves to follows its size bucket, per-bucket overrides stay in their
bucket, the autotuner's bucket cache installs into the right buckets, and a
bucket tuning pass on two sizes keeps a configuration that was timed."""
import json

import pytest
import torch

pytestmark = pytest.mark.gpu


def lak():
    import paper_1409_0669_gb300 as m
    return m


def sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_resolve_follows_bucket():
    m = lak()
    # FP64 dot: 1e6 elements = 16 MB (bucket 1), 1e8 = 1.6 GB (bucket 3)
    assert m.size_bucket("dot", "f64", 10 ** 6, 10 ** 6) == 1
    assert m.size_bucket("dot", "f64", 10 ** 8, 10 ** 8) == 3
    c1 = m.resolve_cfg("dot", "f64", 10 ** 6, 10 ** 6)
    c3 = m.resolve_cfg("dot", "f64", 10 ** 8, 10 ** 8)
    assert (c1.block, c1.vec) == (512, 4) and c1.grid == min(sms(), -(-10 ** 6 // (512 * 4)))
    assert (c3.block, c3.vec) == (256, 4) and c3.grid == 4 * sms()
    # column-major FP64 GEMV 2048^2 (33.6 MB, bucket 1): explicit grid from the table
    g = m.resolve_cfg("gemv_col", "f64", 2048, 2048)
    assert g.block == 512 and g.vec == 4 and g.grid == 2 * sms()
    # 16-bit storage has its own rows: the dot of 1e6 BF16 values (4 MB, bucket
    # 0) takes the BF16-tuned entry (256 threads, 16 per access, automatic grid),
    # the copy keeps the FP32 entry at the same bytes per access (128 threads,
    # 8 x 4 B -> 16 x 2 B); FP16 takes the same rows
    for st in ("bf16", "f16"):
        d = m.resolve_cfg("dot", st, 10 ** 6, 10 ** 6)
        assert (d.block, d.vec) == (256, 16)
        b = m.resolve_cfg("copy", st, 10 ** 6, 10 ** 6)
        assert (b.block, b.vec) == (128, 16)
    g = m.resolve_cfg("gemv_row", "bf16", 1024, 1024)
    assert (g.block, g.vec) == (128, 2)


def test_bucket_override_stays_in_its_bucket():
    m = lak()
    n_small, n_large = 10 ** 5, 10 ** 8
    b_small = m.size_bucket("axpy", "f32", n_small, n_small)
    before_large = m.resolve_cfg("axpy", "f32", n_large, n_large)
    try:
        m.set_default_cfg("axpy", "f32", (96, 0, 2, 1), bucket=b_small)
        s = m.resolve_cfg("axpy", "f32", n_small, n_small)
        assert (s.block, s.vec, s.increment) == (96, 2, 1)
        l = m.resolve_cfg("axpy", "f32", n_large, n_large)
        assert (l.block, l.grid, l.vec, l.increment) == (before_large.block, before_large.grid,
                                                         before_large.vec, before_large.increment)
        # the call itself runs with the override and is exact
        y = torch.rand(n_small, device="cuda")
        z = torch.rand(n_small, device="cuda")
        x = torch.empty_like(y)
        m.vec_axpy(x, y, z, 0.5)
        assert torch.equal(x, torch.addcmul(y, z, torch.tensor(0.5, device="cuda")))
    finally:
        m.set_default_cfg("axpy", "f32", None)


def test_apply_cache_with_bucket_keys(tmp_path):
    from paper_1409_0669_gb300 import autotune
    m = lak()
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({autotune.cache_key(): {"copy:f64:2": [64, 0, 1, 0]}}))
    try:
        assert autotune.apply_cache(str(path)) == 1
        n2 = 10 ** 7                                    # 160 MB: bucket 2
        assert m.size_bucket("copy", "f64", n2, n2) == 2
        c = m.resolve_cfg("copy", "f64", n2, n2)
        assert (c.block, c.vec) == (64, 1)
        c0 = m.resolve_cfg("copy", "f64", 1000, 1000)
        assert c0.block != 64 or c0.vec != 1
    finally:
        m.set_default_cfg("copy", "f64", None)


def test_tune_buckets_small_space():
    """Two sizes in two buckets, three candidate configs: the kept config of
    each bucket is one of the candidates and its reported worst ratio is 1 for
    a single-size bucket."""
    from paper_1409_0669_gb300 import autotune
    from paper_1409_0669_gb300._native import LakCfg
    cands = [LakCfg(128, 0, 4, 0), LakCfg(256, 0, 2, 0), LakCfg(512, 0, 8, 1)]
    results, buckets = {}, {}
    for n in (100_000, 3_000_000):
        prob = autotune.Problem("axpy", "f32", n)
        results[n] = autotune.tune("axpy", "f32", n, reps=5, cfgs=cands, problem=prob)
        buckets[n] = autotune.problem_bucket(prob)
        assert all(r["us"] >= 0 for r in results[n])
    assert buckets[100_000] == 0 and buckets[3_000_000] == 1
    per = autotune.choose_per_bucket(results, buckets)
    for b in (0, 1):
        assert per[b]["cfg"] in [list(c.as_tuple()) for c in cands]
        assert per[b]["worst_ratio"] == 1.0


def test_tiny_dot_runs_as_one_block():
    """A dot whose automatic grid would be at most two blocks runs as one block
    (no grid-wide combine); three blocks' worth keeps its grid.  FP64 bucket 0
    reads 2 elements per access with 256 threads: 1024 elements are two blocks'
    worth, 1537 three."""
    m = lak()
    assert m.resolve_cfg("dot", "f32", 1000, 1000).grid == 1
    assert m.resolve_cfg("dot", "f64", 1024, 1024).grid == 1
    assert m.resolve_cfg("dot", "f64", 1537, 1537).grid == 3
    for dt, n in ((torch.float32, 1000), (torch.float64, 1024), (torch.float64, 1537)):
        x = torch.ones(n, dtype=dt, device="cuda")
        y = torch.full((n,), 0.5, dtype=dt, device="cuda")
        assert float(m.vec_dot(x, y)) == n / 2          # exact: a sum of halves
