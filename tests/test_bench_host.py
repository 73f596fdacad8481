"""Host-side logic of bench.py, on CPU: the max-over-ranks timing rule with
world-size-2 gloo process groups (replicas only: no data-path collective),
the choice of watched launches, the roofline classification, the recorded
DRAM-traffic lookup, and the reference arm's rank handling."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist = bench.init_dist(world, "gloo")
    bench.barrier(dist)
    t = bench.max_over_ranks(10.0 + rank * 5.0, dist)
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((rank, t))


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


class _It:
    def __init__(self, name, op, dtype, size, nbytes):
        self.name, self.op, self.dtype, self.size, self.nbytes = name, op, dtype, size, nbytes


def test_watched_items_and_roofline():
    sys.path.insert(0, ROOT)
    import bench
    items = [_It("copy_f32_1000", "copy", "f32", 1000, 8000),
             _It("copy_f32_2154435", "copy", "f32", 2154435, 2154435 * 8),
             _It("copy_f32_100000000", "copy", "f32", 100000000, 800000000),
             _It("gemv_col_f64_2048", "gemv_col", "f64", 2048, (2048 * 2048 + 4096) * 8),
             _It("gemv_col_f64_16384", "gemv_col", "f64", 16384, (16384 ** 2 + 32768) * 8),
             _It("spmv_lap3d_128_f32", "spmv", "f32", 2097152, 141819908),
             _It("spmv_powerlaw_2m_f32", "spmv", "f32", 2000000, 279882208)]
    w = bench.watched_items(items)
    names = {items[i].name for i in w}
    assert "copy_f32_1000" not in names
    assert {"copy_f32_2154435", "copy_f32_100000000", "gemv_col_f64_2048", "gemv_col_f64_16384",
            "spmv_lap3d_128_f32", "spmv_powerlaw_2m_f32"} <= names
    fp64 = bench.fp64_peak_tflops(152, 2070.0)
    assert abs(fp64 - 1.25856) < 1e-9
    # FP64 GEMV at 478 us: 1.12 TFLOP/s is closer to the FP64 roof than 4.5 TB/s to HBM
    bind, other = bench.roofline_of(items[4], 0.478, 6793.1, "measured", fp64)
    assert bind["bound"] == "alu" and other["bound"] == "hbm"
    assert abs(bind["achieved"] - 2 * 16384 ** 2 / 0.478e-3 / 1e12) < 1e-9
    bind32, none = bench.roofline_of(items[2], 0.117, 6793.1, "measured", fp64)
    assert bind32["bound"] == "hbm" and none is None
    # nnz recovered from the byte count of the 3D Laplacian
    assert abs(bench.flops_of(items[5]) / 2 - 14581760) < 1


def test_recorded_traffic_requires_unchanged_sources_and_cfg(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    class It:
        name, op = "gemv_row_f64_16384", "gemv_row"
    state = {"digest": "d1", "cfg": [64, 0, 4, 0]}
    monkeypatch.setattr(bench, "_sources_digest", lambda op: state["digest"])
    monkeypatch.setattr(bench, "_item_cfg", lambda it: list(state["cfg"]))
    rec = {It.name: {"dram_bytes": 123, "sources_sha256": "d1", "cfg": [64, 0, 4, 0]}}
    path = tmp_path / "t.json"
    path.write_text(json.dumps(rec))
    assert bench.recorded_traffic(str(path), It) == 123
    state["digest"] = "d2"                       # a kernel source changed
    assert bench.recorded_traffic(str(path), It) is None
    state["digest"], state["cfg"] = "d1", [128, 0, 2, 0]   # another launch shape
    assert bench.recorded_traffic(str(path), It) is None

    class Missing:
        name, op = "missing", "copy"
    assert bench.recorded_traffic(str(path), Missing) is None
    # every op the sweep launches has its kernel sources listed, and they exist
    for op in ("copy", "axpy", "dot", "gemv_row", "gemv_col", "spmv"):
        for rel in bench.TRAFFIC_SOURCES[op]:
            assert os.path.exists(os.path.join(ROOT, rel)), rel


def test_reference_arm_runs_only_on_rank0(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"]) == 0
    assert capsys.readouterr().out == ""


def test_e2e_counts_each_distinct_input_once():
    """The end-to-end step copies a shared input (the y and z read by copy,
    update and dot of one size) once, and reads back every launch's result."""
    sys.path.insert(0, ROOT)
    import torch

    import bench
    y = torch.zeros(1000, dtype=torch.float32)
    z = torch.zeros(1000, dtype=torch.float32)
    x = torch.zeros(1000, dtype=torch.float32)
    out = torch.zeros(1, dtype=torch.float32)
    items = [bench.Item("copy", "copy", "f32", 1000, 8000, None, (), h2d=(y,), d2h=(x,)),
             bench.Item("axpy", "axpy", "f32", 1000, 12000, None, (), h2d=(y, z), d2h=(x,)),
             bench.Item("dot", "dot", "f32", 1000, 8000, None, (), h2d=(y, z), d2h=(out,))]
    h2d, d2h = bench.e2e_copy_bytes(items)
    assert h2d == 2 * 4000                   # y and z once each
    assert d2h == 2 * 4000 + 4               # x after copy, x after axpy, the dot
    # a view of the same storage with another length is another input
    items.append(bench.Item("copy2", "copy", "f32", 500, 4000, None, (), h2d=(y[:500],),
                            d2h=(x[:500],)))
    h2d, _ = bench.e2e_copy_bytes(items)
    assert h2d == 2 * 4000 + 2000
