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


def _fake_run_parts(bench):
    """The pieces of a full-size run's report, filled with long-decimal values
    (the worst case for the printed length)."""
    import math
    v = math.pi * 1000.0
    per = {}
    for op in ("copy", "axpy", "dot", "gemv_row", "gemv_col"):
        for dt in ("f32", "f64"):
            per[f"{op}_{dt}"] = {"size": 100000000, "GBs": v, "frac_hbm": v / 7000.0,
                                 "us": v / 9.0, "bound": "alu" if dt == "f64" else "hbm",
                                 "frac_bound": 0.123456789, "copy_same_bytes_GBs": v,
                                 "frac_copy_same_bytes": 0.987654321}
    for mat in ("lap3d", "powerlaw"):
        for dt in ("f32", "f64"):
            per[f"spmv_{mat}_{dt}"] = {"size": 2097152, "GBs": v, "frac_hbm": 0.7777777,
                                       "us": 43.123456, "bound": "gather", "frac_bound": 0.81,
                                       "gather_floor_us": 33.3333, "frac_gather_floor": 0.8,
                                       "us_events_in_sweep": 45.555}
    for name in ("copy_f64_2154435", "axpy_f64_2154435", "dot_f64_2154435",
                 "gemv_row_f64_2048"):
        per["paper_point_" + name] = {"GBs": v, "us": 9.87654, "us_events_in_sweep": 12.3456,
                                      "copy_same_bytes_GBs": v, "frac_copy_same_bytes": 0.99}
    roof = {"bound": "alu", "achieved": 1.1601234567, "peak": 1.2586012345,
            "unit": "TFLOP/s", "frac": 0.9217654321, "traffic": 2148597760,
            "kernel": "gemv_row_f64_16384", "share": 0.0961234567,
            "bytes_per_launch": 2147745792, "flops_per_launch": 536870912.0,
            "ms_per_launch": 0.46271234567,
            "peak_source": "measured: FP64 FMA probe (independent chains) x SMs at the "
                           "median SM clock under load, and more words to be cut",
            "peak_nominal": 1.2586012345,
            "other": {"bound": "hbm", "achieved": 4641.123456, "peak": 6785.9, "unit": "GB/s",
                      "frac": 0.683987654}}
    e2e = {"value": 349.987654321, "unit": "GB/s", "h2d_bytes_per_step": 14123456789,
           "d2h_bytes_per_step": 4512345678, "ms_per_step": 72.4123456,
           "steps": 5, "rounds_ms_per_step": [72.1, 72.4, 73.0], "pipeline": "x" * 300,
           "host_binding": "cpus 0-71"}
    cpu = {"value": 6.612345678, "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": "s" * 600,
           "all_cores": {"value": 98.7654321, "cores": 72, "unit": "GB/s", "sample": "t" * 300},
           "plain_loop": {"value": 25.4321, "cores": 1, "unit": "GB/s", "sample": "u" * 300},
           "host": "Neoverse-V2 " + "h" * 200}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 512}
    return per, roof, e2e, cpu, clocks


def test_headline_is_compact_and_complete():
    """The run's last stdout line stays small enough for a log tail to hold it
    whole, and carries the headline, roofline, end-to-end, CPU-baseline and
    clock keys; the large sections stay out of it."""
    sys.path.insert(0, ROOT)
    import bench
    per, roof, e2e, cpu, clocks = _fake_run_parts(bench)
    line = bench.headline(value=5266.123456789, ms_per_step=4.8123456789, steps=20, warmup=5,
                          world=1, workload=bench.WORKLOAD, bytes_per_step=25312345678,
                          launches=124, roofline=roof, per_kernel=per, e2e=e2e, cpu=cpu,
                          clocks=clocks, detail_path="/some/where/bench_detail.json",
                          probe={"tflops": 1.2345678901, "sm_mhz": 2070.0,
                                 "fma_per_sm_per_clk": 1.9612345, "ms_per_launch": 40.1234},
                          gprobe={"gathers_per_s": 270.123456e9, "per_sm_per_clk": 0.8612345,
                                  "us": 118.7654, "sm_mhz": 2070.0})
    text = json.dumps(line, separators=(",", ":"))
    assert len(text.encode()) <= bench.HEADLINE_MAX_BYTES, len(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "per_kernel", "e2e", "cpu_baseline", "clocks", "gpu_launches"):
        assert key in line, key
    assert line["config"]["workload"] == bench.WORKLOAD
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in line["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in line["e2e"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in line["cpu_baseline"], key
    assert set(line["per_kernel"]) == {k for k in per if not k.startswith("paper_point_")}
    assert line["gpu_launches"] == 124 * 20
    assert line["detail"] == "bench_detail.json"
    for big in ("precision", "batched", "autograd", "fused", "spmv_formats", "small_config",
                "size_curves"):
        assert big not in line
    assert json.loads(text)["value"] == round(5266.123456789, 2)


def test_cpu_chunks_cover_the_sample_exactly():
    """The all-cores CPU leg runs the oracle on fixed chunks of the sample: the
    chunks' bytes add up to the sample's, and the chunked results are the
    single-call results (GEMV and CSR rows concatenate to the full product; the
    chunked dot's hi + lo parts add up to the full dot)."""
    sys.path.insert(0, ROOT)
    import math

    import numpy as np

    import bench
    import oracle
    items = bench.cpu_sample_items()
    chunks = bench.cpu_chunks(items)
    assert abs(sum(b for _, b in chunks) - sum(it[2] for it in items)) < 1e-6 * sum(
        it[2] for it in items)
    pos = 0
    for _, _, b, call in items:
        kind = call[0]
        got, acc = [], 0.0
        while acc < b * (1 - 1e-12):
            fn, cb = chunks[pos]
            got.append(fn())
            acc += cb
            pos += 1
        if kind == "dot":
            parts = [p for hi_lo in got for p in hi_lo]
            assert math.isclose(math.fsum(parts), oracle.dot(call[1], call[2]), rel_tol=1e-15,
                                abs_tol=1e-300)
        elif kind == "gemv":
            _, A, x, g, lay = call
            assert np.array_equal(np.concatenate(got), oracle.gemv(A, x, g, g, g, lay))
        elif kind == "spmv":
            assert np.array_equal(np.concatenate(got),
                                  oracle.csr_spmv(call[1], call[2], call[3], call[4]))
        elif kind == "axpy":
            assert np.array_equal(np.concatenate(got), oracle.axpy(call[1], call[2], 0.5))
    assert pos == len(chunks)


def test_clock_samples_are_taken_from_the_timed_window():
    """Only nvidia-smi samples that arrived while the timed region ran count
    (when any did); throttle reasons are read from the same samples."""
    sys.path.insert(0, ROOT)
    import bench

    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler(0)
    s.proc = _Proc()
    row = "{mhz}, 2070, 500.0, 0x0, {hw}, Not Active, Not Active, Not Active"
    s.lines = [(1.0, row.format(mhz=1000, hw="Active")),        # before: idle, throttled
               (2.0, row.format(mhz=2070, hw="Not Active")),
               (2.5, row.format(mhz=2060, hw="Not Active")),
               (9.0, row.format(mhz=900, hw="Not Active"))]     # after
    c = s.stop((1.5, 3.0))
    assert c["samples"] == 2 and c["sm_mhz"] == 2065.0 and c["reasons"] == []
    c = s.stop((5.0, 6.0))                 # nothing inside: every sample counts
    assert c["samples"] == 4 and c["reasons"] == ["hw_slowdown"]
