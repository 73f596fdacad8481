"""The copy-first study (Sec. 3.2, 3.4 repeated on GB300) on a reduced space
and small sizes: the report has its structure, every copy-derived best is one
of the kept copy candidates, no copy-derived best beats the op's own best
over the same space by more than timing noise, and the markdown table renders
from the report."""
import pytest

pytestmark = pytest.mark.gpu


def test_copy_first_study_reduced_space():
    from paper_1409_0669_gb300 import autotune
    from paper_1409_0669_gb300._native import LakCfg
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cfgs = [LakCfg(b, k * sms, v, inc) for (b, k, v, inc) in
            ((64, 0, 4, 0), (128, 8, 8, 0), (256, 0, 2, 0), (256, 4, 4, 1), (512, 2, 8, 0),
             (512, 0, 16, 0), (128, 32, 1, 0), (32, 16, 4, 0), (256, 16, 8, 1), (512, 1, 1, 0),
             (128, 0, 4, 1), (64, 32, 8, 0))]
    sizes = {"copy": 1_000_000, "axpy": 1_000_000, "dot": 1_000_000, "gemv_row": 512,
             "gemv_col": 512, "spmv": "lap2d_256"}
    rep = autotune.copy_first_study("f32", sizes, reps=5, cfgs=cfgs)
    assert rep["space"] <= len(cfgs) and rep["candidates"] >= 1
    cands = {tuple(c) for c in rep["candidate_cfgs"]}
    assert len(cands) == rep["candidates"]
    for c in cands:
        assert any(tuple(c) == tuple(x.as_tuple()) for x in cfgs)
    for op in ("axpy", "dot", "gemv_row", "gemv_col", "spmv"):
        r = rep["ops"][op]
        assert tuple(r["best_from_copy"]["cfg"]) in cands
        assert r["best_from_copy"]["GBs"] <= 1.3 * r["own_best"]["GBs"], (op, r)   # timing noise
        assert abs(r["ratio"] - r["best_from_copy"]["GBs"] / r["own_best"]["GBs"]) < 1e-12
        assert r["default"]["GBs"] > 0
    assert tuple(rep["shared_cfg"]) in cands
    assert 0 < rep["shared_worst_ratio"] <= 1.3
    rep["label"] = "small"
    table = autotune.study_table([rep])
    assert table.count("\n| F32, small |") == 5
