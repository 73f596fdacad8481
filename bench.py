#!/usr/bin/env python3
"""Benchmark of the bandwidth-bound kernels on GB300: achieved HBM GB/s per
kernel and for the whole sweep, against the measured copy roofline.

One step = one pass of every kernel over the FP32 + FP64 size sweep:
  vectors n = round(10^(3+k/3)), k = 0..15 (1e3 .. 1e8), U(-1, 1):
      copy x <- y, update x <- y + 0.5 z, inner product <y, z>
  dense GEMV y = A x, A ~ N(0, 1), 512^2 .. 16384^2, row- and column-major
  CSR SpMV: 3D 7-point Laplacian 128^3 (6/-1) and power-law random CSR with
      2,000,000 rows (row length 4..256, mean 16), values N(0, 1)
Every buffer is read once per step and gigabytes of other traffic pass between
two reads of the same buffer, so L2 (126 MB) holds nothing useful across
reuses; the whole step moves ~25 GB.

Bytes are algorithmic (minimum) bytes, the paper's convention (Sec. 3): for
GEMV the right-hand side counts once; for SpMV x counts once.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the deliberately slow baseline)
on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HBM GB/s & % of peak per kernel; bf16/batched vs plain fp32 time at stated err"
WORKLOAD = ("fp32+fp64 size sweep: vectors 1e3..1e8 (16 sizes; copy, x=y+0.5z, <y,z>), "
            "GEMV row+col 512^2..16384^2, CSR SpMV 3D Laplacian 128^3 + power-law 2M rows")


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world: int, backend: str):
    if world <= 1:
        return None
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(value: float, dist, device=None) -> float:
    """Max of a per-rank scalar (the timing rule: the slowest rank sets the time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist, device=None):
    if dist is not None:
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons in the background."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, window=None):
        """Summary of the samples; with window = (t0, t1) (time.monotonic()
        values around the timed region) only the samples taken inside it, if
        any arrived there."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        lines = [ln for _, ln in self.lines]
        if window is not None:
            inside = [ln for t, ln in self.lines if window[0] <= t <= window[1]]
            if inside:
                lines = inside
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the sweep workload
# ---------------------------------------------------------------------------

class Item:
    """One kernel launch of the step: pre-marshalled C-ABI call plus its
    algorithmic byte count."""
    __slots__ = ("name", "op", "dtype", "size", "nbytes", "fn", "args", "h2d", "d2h")

    def __init__(self, name, op, dtype, size, nbytes, fn, args, h2d=(), d2h=()):
        self.name, self.op, self.dtype, self.size = name, op, dtype, size
        self.nbytes, self.fn, self.args = nbytes, fn, args
        self.h2d, self.d2h = h2d, d2h      # device tensors the e2e leg fills / reads back


def _aligned_slices(total_elems_list, dtype, device, align_elems):
    import torch
    offs, cur = [], 0
    for n in total_elems_list:
        offs.append(cur)
        cur += (n + align_elems - 1) // align_elems * align_elems
    buf = torch.empty(max(cur, 1), dtype=dtype, device=device)
    return buf, [buf[o:o + n] for o, n in zip(offs, total_elems_list)]


def build_sweep(device, stream_handle, only=None):
    """Allocate and fill the sweep's inputs and return the ordered launch list.
    `only` (a compiled regex) keeps just the launches whose name matches, and
    allocates nothing for the others."""
    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300 import _native

    lib = _native.load()
    items = []
    sizes = synth.vector_sweep_sizes()
    gsizes = synth.gemv_sweep_sizes()
    keep = []                                   # keep tensors alive
    def want(name):
        return only is None or only.search(name) is not None

    for storage, es, seed0 in (("f32", 4, 100), ("f64", 8, 200)):
        dt = synth.torch_dtype(storage)
        code = _native.DTYPES[storage]
        vec_names = [f"{op}_{storage}_{n}" for op in ("copy", "axpy", "dot") for n in sizes]
        if not any(want(nm) for nm in vec_names):
            sizes_used = []
        else:
            sizes_used = sizes
        # vectors: one flat buffer per role, 256-byte aligned sub-vectors
        if not sizes_used:
            ybuf = zbuf = xbuf = None
            ys = zs = xs = []
        else:
            ybuf, ys = _aligned_slices(sizes, dt, device, 64)
            zbuf, zs = _aligned_slices(sizes, dt, device, 64)
            xbuf, xs = _aligned_slices(sizes, dt, device, 64)
            synth.device_uniform_(ybuf, seed0 + 1)
            synth.device_uniform_(zbuf, seed0 + 2)
            xbuf.zero_()
        outs = torch.zeros(len(sizes), dtype=dt, device=device)
        keep += [ybuf, zbuf, xbuf, outs]
        for n, y, x in zip(sizes_used, ys, xs):
            items.append(Item(f"copy_{storage}_{n}", "copy", storage, n, 2 * n * es,
                              lib.vec_copy, (x.data_ptr(), y.data_ptr(), n, code, None,
                                             stream_handle), h2d=(y,), d2h=(x,)))
        for n, y, z, x in zip(sizes_used, ys, zs, xs):
            items.append(Item(f"axpy_{storage}_{n}", "axpy", storage, n, 3 * n * es,
                              lib.vec_axpy, (x.data_ptr(), y.data_ptr(), z.data_ptr(), 0.5, n,
                                             code, None, stream_handle), h2d=(y, z), d2h=(x,)))
        for k, (n, y, z) in enumerate(zip(sizes_used, ys, zs)):
            wsb = lak.vec_dot_workspace(n, storage)
            ws = torch.zeros(wsb, dtype=torch.uint8, device=device)
            keep.append(ws)
            items.append(Item(f"dot_{storage}_{n}", "dot", storage, n, 2 * n * es,
                              lib.vec_dot, (outs[k:k + 1].data_ptr(), y.data_ptr(), z.data_ptr(),
                                            n, code, ws.data_ptr(), wsb, None, stream_handle),
                              h2d=(y, z), d2h=(outs[k:k + 1],)))
        # dense GEMV, both layouts
        for layout, lcode in (("row", 0), ("col", 1)):
            for k, n in enumerate(gsizes):
                if not want(f"gemv_{layout}_{storage}_{n}"):
                    continue
                A = torch.empty(n * n, dtype=dt, device=device)
                synth.device_normal_(A, seed0 + 10 + k + (50 if layout == "col" else 0))
                xg = torch.empty(n, dtype=dt, device=device)
                synth.device_uniform_(xg, seed0 + 30 + k)
                yg = torch.zeros(n, dtype=dt, device=device)
                wsb = lak.dense_gemv_workspace(n, n, layout, storage)
                ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=device)
                keep += [A, xg, yg, ws]
                nbytes = (n * n + 2 * n) * es
                items.append(Item(f"gemv_{layout}_{storage}_{n}", f"gemv_{layout}", storage,
                                  n, nbytes, lib.dense_gemv,
                                  (yg.data_ptr(), A.data_ptr(), xg.data_ptr(), n, n, n, lcode,
                                   code, ws.data_ptr(), ws.numel(), None, stream_handle),
                                  h2d=(A, xg), d2h=(yg,)))
        # CSR SpMV
        sparse = (("lap3d_128", lambda: synth.laplacian_3d(128, storage), 128 ** 3),
                  ("powerlaw_2m", lambda: synth.powerlaw_csr(2_000_000, 2_000_000, 1, storage),
                   2_000_000))
        for name, make, ncols in sparse:
            if not want(f"spmv_{name}_{storage}"):
                continue
            rp, ci, v = make()
            rpd, cid, vd = rp.to(device), ci.to(device), v.to(device)
            xsp = torch.empty(ncols, dtype=dt, device=device)
            synth.device_uniform_(xsp, seed0 + 40)
            m = rp.numel() - 1
            nnz = v.numel()
            ysp = torch.zeros(m, dtype=dt, device=device)
            keep += [rpd, cid, vd, xsp, ysp]
            nbytes = nnz * (es + 4) + (m + 1) * 4 + ncols * es + m * es
            items.append(Item(f"spmv_{name}_{storage}", "spmv", storage, m, nbytes, lib.csr_spmv,
                              (ysp.data_ptr(), rpd.data_ptr(), cid.data_ptr(), vd.data_ptr(),
                               xsp.data_ptr(), m, ncols, nnz, code, None, stream_handle),
                              h2d=(rpd, cid, vd, xsp), d2h=(ysp,)))
    items = [it for it in items if want(it.name)]
    if not items:
        raise ValueError("no launch matches the --only filter")
    return items, keep


def watched_items(items):
    """Indices of the launches timed individually: the largest size of every
    (op, dtype) -- where the roofline is read -- and the paper's own points
    (vectors of ~2e6 entries, the 2048^2 matrix).  Small launches run without
    per-launch events, which would otherwise dominate their duration."""
    best = {}
    for i, it in enumerate(items):
        key = (it.op, it.dtype, it.name.split("_")[1] if it.op == "spmv" else "")
        if key not in best or it.size > items[best[key]].size:
            best[key] = i
    idx = set(best.values())
    for i, it in enumerate(items):
        if it.size in (2154435, 2048):
            idx.add(i)
    return sorted(idx)


def run_step(items, lib_check, events=None):
    """One pass over every launch; `events` maps an item index to its
    (start, end) CUDA events."""
    for i, it in enumerate(items):
        ev = events.get(i) if events is not None else None
        if ev is not None:
            ev[0].record()
        st = it.fn(*it.args)
        if st != 0:
            lib_check(it.name, st)
        if ev is not None:
            ev[1].record()


# ---------------------------------------------------------------------------
# CPU oracle sample (the reference arm and the cpu_baseline)
# ---------------------------------------------------------------------------

def cpu_sample_items():
    """A bounded sample of the sweep for the FP64 CPU oracle: every op and
    dtype at a reduced size (vectors 1e6, GEMV 1024^2 both layouts, SpMV on the
    3D Laplacian 32^3 and a 50,000-row power-law matrix)."""
    import numpy as np

    import synth
    items = []
    for storage, es in (("f32", 4), ("f64", 8)):
        n = 1_000_000
        y = synth.uniform(n, 1, storage).numpy()
        z = synth.uniform(n, 2, storage).numpy()
        items += [("copy", storage, 2 * n * es, ("copy", y)),
                  ("axpy", storage, 3 * n * es, ("axpy", y, z)),
                  ("dot", storage, 2 * n * es, ("dot", y, z))]
        g = 1024
        A = synth.normal((g, g), 3, storage).numpy().ravel()
        xg = synth.uniform(g, 4, storage).numpy()
        for lay in ("row", "col"):
            items.append((f"gemv_{lay}", storage, (g * g + 2 * g) * es, ("gemv", A, xg, g, lay)))
        for name, (rp, ci, v), nc in (("lap3d", synth.laplacian_3d(32, storage), 32 ** 3),
                                      ("powerlaw", synth.powerlaw_csr(50_000, 50_000, 5, storage),
                                       50_000)):
            xs = synth.uniform(nc, 6, storage).numpy()
            m = rp.numel() - 1
            nnz = v.numel()
            nbytes = nnz * (es + 4) + (m + 1) * 4 + nc * es + m * es
            items.append((f"spmv_{name}", storage, nbytes,
                          ("spmv", rp.numpy(), ci.numpy(), v.numpy(), xs)))
    del np
    return items


def cpu_run(items):
    import oracle
    nbytes = 0
    for _, _, b, call in items:
        kind = call[0]
        if kind == "copy":
            oracle.copy(call[1])
        elif kind == "axpy":
            oracle.axpy(call[1], call[2], 0.5)
        elif kind == "dot":
            oracle.dot(call[1], call[2])
        elif kind == "gemv":
            _, A, x, g, lay = call
            oracle.gemv(A, x, g, g, g, lay)
        elif kind == "spmv":
            oracle.csr_spmv(call[1], call[2], call[3], call[4])
        nbytes += b
    return nbytes


CPU_SAMPLE_DESC = ("oracle (plain C, FP64 compensated sums, single thread) on a bounded sample: "
                   "f32+f64 vectors n=1e6 (copy, update, dot), GEMV 1024^2 row+col, SpMV 3D "
                   "Laplacian 32^3 + power-law 50k rows; GB/s from the same algorithmic bytes")


CHUNK_ELEMS = 1 << 18       # vector chunk of the all-cores oracle run
CHUNK_ROWS = 128            # GEMV rows per chunk
CHUNK_CSR_ROWS = 8192       # CSR rows per chunk


def cpu_chunks(items):
    """The sample split into fixed chunks (independent of the thread count, so
    every result is the same however many threads run them): a list of
    (callable, bytes) pairs, each calling the oracle on one chunk."""
    import numpy as np

    import oracle
    out = []
    for _, _, b, call in items:
        kind = call[0]
        if kind in ("copy", "axpy", "dot"):
            n = call[1].size
            for a in range(0, n, CHUNK_ELEMS):
                e = min(n, a + CHUNK_ELEMS)
                frac = (e - a) / n
                if kind == "copy":
                    out.append((lambda y=call[1][a:e]: oracle.copy(y), b * frac))
                elif kind == "axpy":
                    out.append((lambda y=call[1][a:e], z=call[2][a:e]: oracle.axpy(y, z, 0.5),
                                b * frac))
                else:
                    out.append((lambda y=call[1][a:e], z=call[2][a:e]: oracle.dot(y, z, True),
                                b * frac))
        elif kind == "gemv":
            _, A, x, g, lay = call
            for r in range(0, g, CHUNK_ROWS):
                rows = min(CHUNK_ROWS, g - r)
                sub = A[r * g:] if lay == "row" else A[r:]
                out.append((lambda sub=sub, rows=rows, lay=lay, x=x, g=g:
                            oracle.gemv(sub, x, rows, g, g, lay), b * rows / g))
        else:
            _, rp, ci, v, x = call
            m = rp.size - 1
            for r in range(0, m, CHUNK_CSR_ROWS):
                e = min(m, r + CHUNK_CSR_ROWS)
                lo, hi = int(rp[r]), int(rp[e])
                srp = (rp[r:e + 1] - lo).astype(np.int32)
                out.append((lambda srp=srp, c=ci[lo:hi], vv=v[lo:hi], x=x:
                            oracle.csr_spmv(srp, c, vv, x), b * (e - r) / m))
    return out


def plain_calls(items):
    """The sample as the plain loops (uncompensated, the data's own precision):
    (callable, bytes) pairs."""
    import oracle
    out = []
    for _, _, b, call in items:
        kind = call[0]
        if kind == "copy":
            y = call[1]
            dst = y.copy()
            out.append((lambda y=y, d=dst: oracle.plain_copy(y, d), b))
        elif kind == "axpy":
            y, z = call[1], call[2]
            dst = y.copy()
            out.append((lambda y=y, z=z, d=dst: oracle.plain_axpy(y, z, 0.5, d), b))
        elif kind == "dot":
            out.append((lambda y=call[1], z=call[2]: oracle.plain_dot(y, z), b))
        elif kind == "gemv":
            _, A, x, g, lay = call
            out.append((lambda A=A, x=x, g=g, lay=lay: oracle.plain_gemv(A, x, g, g, g, lay), b))
        else:
            _, rp, ci, v, x = call
            out.append((lambda rp=rp, ci=ci, v=v, x=x: oracle.plain_csr(rp, ci, v, x), b))
    return out


def _timed_passes(run_pass, min_seconds):
    run_pass()                                  # warm caches / page in
    t0 = time.perf_counter()
    total, passes = 0.0, 0
    while True:
        total += run_pass()
        passes += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            return total, passes, el


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def cpu_baseline(min_seconds: float = 10.0):
    """The oracle on a bounded sample, single-threaded (the reported value),
    then over every affinitised core on fixed chunks, and the plain
    uncompensated loops on one core."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    oracle.build()
    items = cpu_sample_items()
    total, passes, el = _timed_passes(lambda: cpu_run(items), min_seconds)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    chunks = cpu_chunks(items)

    def parallel_pass(pool):
        list(pool.map(lambda cb: cb[0](), chunks))
        return sum(b for _, b in chunks)

    with ThreadPoolExecutor(max_workers=cores) as pool:
        ptotal, ppasses, pel = _timed_passes(lambda: parallel_pass(pool), min_seconds / 4)
    plain = plain_calls(items)

    def plain_pass():
        for fn, _ in plain:
            fn()
        return sum(b for _, b in plain)

    qtotal, qpasses, qel = _timed_passes(plain_pass, min_seconds / 4)
    return {"value": total / el / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{CPU_SAMPLE_DESC}; {passes} passes in {el:.1f} s",
            "all_cores": {"value": ptotal / pel / 1e9, "unit": "GB/s", "cores": cores,
                          "sample": f"the same oracle calls on fixed chunks ({CHUNK_ELEMS} "
                                    f"elements, {CHUNK_ROWS} GEMV rows, {CHUNK_CSR_ROWS} CSR "
                                    f"rows) over {cores} threads; {ppasses} passes in "
                                    f"{pel:.1f} s"},
            "plain_loop": {"value": qtotal / qel / 1e9, "unit": "GB/s", "cores": 1,
                           "sample": f"plain uncompensated loops in the data's precision on "
                                     f"the same sample; {qpasses} passes in {qel:.1f} s"},
            "host": host_cpu_model(), "affinity_cores": cores}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    items = cpu_sample_items()
    for _ in range(args.warmup):
        cpu_run(items)
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        total += cpu_run(items)
    el = time.perf_counter() - t0
    value = total / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64 storage, f64 arithmetic", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": CPU_SAMPLE_DESC},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": CPU_SAMPLE_DESC},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fp64_peak_tflops(sms: int, sm_mhz: float) -> float:
    """FP64 FMA roof of GB300: 2 FP64 FMA (4 flop) per SM per clock -- the unit
    count that gives the nominal 1.25 TFLOP/s at 152 SMs and 2.07 GHz."""
    return sms * 4.0 * sm_mhz * 1e6 / 1e12


def fp64_probe(device, stream, iters: int = 10000, reps: int = 3):
    """The FP64 FMA roof measured live (lak_probe_fma_f64: 8 independent FMA
    chains per thread, every SM full), median of `reps` launches of ~40 ms
    timed with events on `stream`, with the SM clock sampled meanwhile."""
    import torch

    import paper_1409_0669_gb300 as lak
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.2)
    with torch.cuda.stream(stream):
        out, flops = lak.probe_fma_f64(iters)             # warm-up
        times = []
        for _ in range(reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            lak.probe_fma_f64(iters, out=out)
            e.record(stream)
            e.synchronize()
            times.append(s.elapsed_time(e))
    clocks = sampler.stop()
    ms = statistics.median(times)
    tf = flops / (ms * 1e-3) / 1e12
    mhz = clocks.get("sm_mhz")
    return {"tflops": tf, "ms_per_launch": ms, "flops_per_launch": flops, "sm_mhz": mhz,
            "fma_per_sm_per_clk": (tf * 1e12 / 2 / (torch.cuda.get_device_properties(device)
                                   .multi_processor_count * mhz * 1e6)) if mhz else None,
            "reasons": clocks.get("reasons")}


def flops_of(it) -> float:
    """Algorithmic floating-point operations of one launch (FMA = 2)."""
    if it.op == "axpy":
        return 2.0 * it.size
    if it.op == "dot":
        return 2.0 * it.size
    if it.op.startswith("gemv"):
        return 2.0 * it.size * it.size
    if it.op == "spmv":
        es = 8 if it.dtype == "f64" else 4
        m = it.size
        # nbytes = nnz*(es+4) + (m+1)*4 + n*es + m*es with n = m for these matrices
        nnz = (it.nbytes - (m + 1) * 4 - 2 * m * es) / (es + 4)
        return 2.0 * nnz
    return 0.0


def roofline_of(it, ms, hbm_peak, hbm_kind, fp64_peak):
    """The binding roof of one launch: HBM, or the FP64 FMA pipe for FP64
    kernels whose FP64 fraction is the larger one."""
    gbs = it.nbytes / (ms * 1e-3) / 1e9
    hbm = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
           "frac": gbs / hbm_peak, "peak_source": f"{hbm_kind} hbm_gbs (copy)"}
    if it.dtype != "f64":
        return hbm, None
    tf = flops_of(it) / (ms * 1e-3) / 1e12
    alu = {"bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
           "frac": tf / fp64_peak,
           "peak_source": "measured: FP64 FMA probe (lak_probe_fma_f64) in this run"}
    return (alu, hbm) if alu["frac"] > hbm["frac"] else (hbm, alu)


def run_batched(device, reps=10, count=4096, seed=4000):
    """4096 uneven instances per family, each family in ONE persistent launch
    (block, grid and vector width from the autotuned defaults), all families
    captured in one CUDA graph.  Compared with 4096 separate launches per
    family (issued from the host) and with one CUDA graph of those separate
    launches.  Instance sizes: vectors n ~ log-uniform 256..1M (axpy, dot);
    dense GEMV m, n ~ log-uniform 64..4096; CSR blocks of 1k..200k rows with
    5..64 entries per row (square, random columns)."""
    import ctypes

    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300 import _native
    from paper_1409_0669_gb300 import batch as B

    lib = _native.load()
    dev = device
    stream = torch.cuda.current_stream(dev)
    sh = stream.cuda_stream
    code = _native.DTYPES["f32"]
    fams = {}

    wl = synth.batch_workload(dev, count, seed)
    ys = [v[0] for v in wl["vec"]]
    zs = [v[1] for v in wl["vec"]]
    xs = [v[2] for v in wl["vec"]]
    ns = [y.numel() for y in ys]
    outs = torch.zeros(count, device=dev)
    wsd = torch.zeros(1 << 20, dtype=torch.uint8, device=dev)
    fams["axpy"] = (B.axpy_batch(xs, ys, zs, [0.5] * count),
                    [(lib.vec_axpy, (x.data_ptr(), y.data_ptr(), z.data_ptr(), 0.5, x.numel(),
                                     code, None, sh)) for x, y, z in zip(xs, ys, zs)],
                    int(sum(3 * 4 * int(n) for n in ns)))
    fams["dot"] = (B.dot_batch(ys, zs, [outs[i:i + 1] for i in range(count)]),
                   [(lib.vec_dot, (outs[i:i + 1].data_ptr(), y.data_ptr(), z.data_ptr(),
                                   y.numel(), code, wsd.data_ptr(), wsd.numel(), None, sh))
                    for i, (y, z) in enumerate(zip(ys, zs))],
                   int(sum(2 * 4 * int(n) for n in ns)))

    As = [g[0] for g in wl["gemv"]]
    gx = [g[1] for g in wl["gemv"]]
    gy = [g[2] for g in wl["gemv"]]
    fams["gemv"] = (B.gemv_batch(As, gx, gy),
                    [(lib.dense_gemv, (y.data_ptr(), A.data_ptr(), x.data_ptr(), A.shape[0],
                                       A.shape[1], A.shape[1], 0, code, None, 0, None, sh))
                     for A, x, y in zip(As, gx, gy)],
                    int(sum((A.shape[0] * A.shape[1] + A.shape[0] + A.shape[1]) * 4
                            for A in As)))

    csrs = [c[0] for c in wl["csr"]]
    cx = [c[1] for c in wl["csr"]]
    cy = [c[2] for c in wl["csr"]]
    cbytes = sum(v.numel() * 8 + (m + 1) * 4 + 2 * m * 4 for (_, _, v, m) in csrs)
    fams["spmv"] = (B.spmv_batch(csrs, cx, cy),
                    [(lib.csr_spmv, (y.data_ptr(), rp.data_ptr(), ci.data_ptr(), v.data_ptr(),
                                     x.data_ptr(), m, m, v.numel(), code, None, sh))
                     for (rp, ci, v, m), x, y in zip(csrs, cx, cy)],
                    int(cbytes))
    torch.cuda.synchronize()

    def separate(calls):
        for fn, a in calls:
            st = fn(*a)
            if st != 0:
                _native.check("separate launch", st)

    report = {"instances_per_family": count, "dtype": "f32",
              "sizes": "vectors log-uniform 256..1M; GEMV m,n log-uniform 64..4096; "
                       "CSR 1k..200k rows x 5..64 nnz/row"}
    for name, (bt, calls, nbytes) in fams.items():
        for _ in range(3):
            bt.run()
        separate(calls)
        torch.cuda.synchronize()
        t_b = _launch_ms(bt.run, reps)
        t_s = _launch_ms(lambda: separate(calls), max(3, reps // 3))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            separate_graph_calls = [(fn, a[:-1] + (torch.cuda.current_stream().cuda_stream,))
                                    for fn, a in calls]
            separate(separate_graph_calls)
        t_g = _launch_ms(g.replay, reps)
        del g
        report[name] = {"bytes": nbytes, "units": bt.total_units,
                        "us_batched": round(t_b * 1e3, 1),
                        "GBs_batched": round(nbytes / (t_b * 1e-3) / 1e9, 1),
                        "us_separate_launches": round(t_s * 1e3, 1),
                        "us_graph_of_separate": round(t_g * 1e3, 1),
                        "speedup_vs_separate": round(t_s / t_b, 2),
                        "speedup_vs_graph_of_separate": round(t_g / t_b, 2)}
    # every family's persistent launch in one CUDA graph
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for bt, _, _ in fams.values():
            bt.run()
    t_all = _launch_ms(g.replay, reps)
    tot = sum(nb for _, _, nb in fams.values())
    report["all_families_one_graph"] = {"bytes": tot, "us": round(t_all * 1e3, 1),
                                        "GBs": round(tot / (t_all * 1e-3) / 1e9, 1)}
    del g
    # the CSR family's gather floor: one sparse inner product over all its
    # entries, each instance's columns offset into the concatenation of the x
    # vectors (the same gathers, in the same order, without the row structure)
    offs, o = [], 0
    for (_, _, _, m) in csrs:
        offs.append(o)
        o += m
    vals = torch.cat([c[2] for c in csrs])
    idx = torch.cat([c[1] + off for c, off in zip(csrs, offs)])
    xall = torch.cat(cx)
    res = torch.zeros(1, device=dev)
    wsf = torch.zeros(lak.vec_dot_sparse_workspace(vals.numel(), "f32"), dtype=torch.uint8,
                      device=dev)

    def floor_call():
        lak.vec_dot_sparse(vals, idx, xall, out=res, workspace=wsf)

    floor_call()
    t_f = _launch_ms(floor_call, reps)
    report["spmv"]["entries"] = int(vals.numel())
    report["spmv"]["gather_floor_us"] = round(t_f * 1e3, 1)
    report["spmv"]["frac_gather_floor"] = round(t_f / (report["spmv"]["us_batched"] * 1e-3), 3)
    del vals, idx, xall
    del ctypes
    return report


def run_autograd(device, reps=20):
    """Forward and backward of the differentiable products on the
    differentiation workload: dense 4096^2 FP32 GEMV, CSR 3D Laplacian 64^3
    FP32, dot n = 1e7 FP32.  Each backward kernel is timed on its own (L2
    flushed by reading 256 MB before every launch) with its algorithmic bytes."""
    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300 import autograd as ag

    dev = device
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}

    def rec(name, fn, nbytes):
        for _ in range(3):
            fn()
        ms = _launch_ms(fn, reps, flush)
        out[name] = {"us": round(ms * 1e3, 2), "GBs": round(nbytes / (ms * 1e-3) / 1e9, 1)}

    m = n = 4096
    A = synth.device_normal_(torch.empty(m, n, device=dev), 1001)
    x = synth.device_uniform_(torch.empty(n, device=dev), 1002)
    dy = synth.device_uniform_(torch.empty(m, device=dev), 1003)
    dA = torch.empty(m, n, device=dev)
    dx = torch.empty(n, device=dev)
    rec("gemv_forward", lambda: lak.dense_gemv(A, x), (m * n + m + n) * 4)
    rec("gemv_backward_dA_outer", lambda: lak.dense_outer(dy, x, out=dA), (m * n + m + n) * 4)
    rec("gemv_backward_dx_transposed", lambda: lak.dense_gemv(A.t(), dy, y=dx), (m * n + m + n) * 4)
    Ar = A.clone().requires_grad_()
    xr = x.clone().requires_grad_()

    def full():
        Ar.grad = None
        xr.grad = None
        ag.gemv(Ar, xr).backward(dy)
    rec("gemv_forward_backward_autograd", full, 3 * (m * n + m + n) * 4)

    # the whole forward + backward step captured once into one CUDA graph (the
    # gradients land in the .grad tensors allocated during capture) and replayed:
    # the same kernels with no per-call host work
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(3):
            full()
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    Ar.grad = None
    xr.grad = None
    step_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(step_graph):
        ag.gemv(Ar, xr).backward(dy)
    rec("gemv_forward_backward_one_graph", step_graph.replay, 3 * (m * n + m + n) * 4)
    del step_graph

    rp, ci, v = synth.laplacian_3d(64, "f32")
    mm = rp.numel() - 1
    nnz = v.numel()
    pat = ag.CsrPattern(rp.to(dev), ci.to(dev), mm)
    vals = v.to(dev)
    xs = synth.device_uniform_(torch.empty(mm, device=dev), 1004)
    dys = synth.device_uniform_(torch.empty(mm, device=dev), 1005)
    spmv_bytes = nnz * 8 + (mm + 1) * 4 + 2 * mm * 4
    rec("spmv_forward", lambda: lak.csr_spmv(pat.row_ptr, pat.col_idx, vals, xs), spmv_bytes)
    torch.cuda.synchronize()
    import time
    t0 = time.perf_counter()
    cp, ri, perm = lak.csr_transpose(pat.row_ptr, pat.col_idx, mm)
    torch.cuda.synchronize()
    out["spmv_transpose_prepare_once_ms"] = round((time.perf_counter() - t0) * 1e3, 3)
    pat._t = (cp, ri, perm)
    dv = torch.empty(nnz, device=dev)
    vt = torch.empty(nnz, device=dev)
    rec("spmv_backward_dvals_sampled", lambda: lak.csr_sampled_outer(pat.row_ptr, pat.col_idx, dys,
                                                                   xs, out=dv),
        nnz * 4 + nnz * 4 + (mm + 1) * 4 + 2 * mm * 4)
    rec("spmv_backward_gather_values", lambda: lak.vec_gather(vals, perm, out=vt), nnz * 12)
    rec("spmv_backward_dx_transposed", lambda: lak.csr_spmv(cp, ri, vt, dys), spmv_bytes)

    nd = 10_000_000
    a = synth.device_uniform_(torch.empty(nd, device=dev), 1006)
    b = synth.device_uniform_(torch.empty(nd, device=dev), 1007)
    ds = torch.ones(1, device=dev)
    da = torch.empty_like(a)
    rec("dot_forward", lambda: lak.vec_dot(a, b), nd * 8)
    rec("dot_backward_scale", lambda: lak.vec_scale_dev(b, ds, out=da), nd * 8)
    return out


def run_fused(device, reps=20):
    """Fused forms against their unfused sequences (FP32 and FP64, n = 1e8 /
    16384^2): x = y + a z with <x, x> in one pass vs vec_axpy then vec_dot
    (3n vs 5n elements moved), and y = a A x + b y vs dense_gemv plus a
    separate update; L2 flushed (256 MB read) before every timed launch."""
    import torch

    import paper_1409_0669_gb300 as lak
    import synth

    dev = device
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}
    for storage in ("f32", "f64"):
        dt = synth.torch_dtype(storage)
        es = 8 if storage == "f64" else 4
        n = 100_000_000
        y = synth.device_uniform_(torch.empty(n, dtype=dt, device=dev), 1101)
        z = synth.device_uniform_(torch.empty(n, dtype=dt, device=dev), 1102)
        x = torch.empty_like(y)
        ws = torch.zeros(max(lak.vec_dot_workspace(n, storage),
                             lak.vec_axpy_norm2_workspace(n, storage)),
                         dtype=torch.uint8, device=dev)

        def fused():
            lak.vec_axpy_norm2(x, y, z, 0.5, workspace=ws)

        def separate():
            lak.vec_axpy(x, y, z, 0.5)
            lak.vec_dot(x, x, workspace=ws)
        for f in (fused, separate):
            f()
        tf = _launch_ms(fused, reps, flush)
        ts = _launch_ms(separate, reps, flush)
        out[f"axpy_norm2_{storage}"] = {"us_fused": round(tf * 1e3, 1),
                                        "GBs_fused": round(3 * n * es / (tf * 1e-3) / 1e9, 1),
                                        "us_separate": round(ts * 1e3, 1),
                                        "speedup": round(ts / tf, 3)}
        g = 16384
        A = synth.device_normal_(torch.empty(g, g, dtype=dt, device=dev), 1103)
        xg = synth.device_uniform_(torch.empty(g, dtype=dt, device=dev), 1104)
        yg = synth.device_uniform_(torch.empty(g, dtype=dt, device=dev), 1105)
        tmp = torch.empty_like(yg)

        def gfused():
            lak.dense_gemv(A, xg, y=yg, alpha=0.5, beta=-1.0)

        def gseparate():
            lak.dense_gemv(A, xg, y=tmp)
            lak.vec_axpby(yg, -1.0, yg, 0.5, tmp)
        for f in (gfused, gseparate):
            f()
        tf = _launch_ms(gfused, reps, flush)
        ts = _launch_ms(gseparate, reps, flush)
        out[f"gemv_axpby_{storage}"] = {"us_fused": round(tf * 1e3, 1), "us_separate": round(ts * 1e3, 1),
                                        "speedup": round(ts / tf, 3)}
        del y, z, x, A
    return out


def run_formats(device, reps=20):
    """CSR vs SELL-C-sigma (C = 32) vs row-binned CSR on the sweep's two
    matrices (3D Laplacian 128^3 with sigma = 1, power-law 2M rows with sigma =
    1024), FP32 and FP64, L2 flushed (256 MB read) before every timed launch;
    SELL bytes count the padded slots it actually reads, the binned product
    reads the CSR bytes plus its row permutation.  Conversion times once."""
    import time

    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300.csr_bin import BinnedCsr
    from paper_1409_0669_gb300.sell import SellMatrix

    dev = device
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}
    for storage in ("f32", "f64"):
        es = 8 if storage == "f64" else 4
        for name, make, ncols, sigma in (
                ("lap3d_128", lambda: synth.laplacian_3d(128, storage), 128 ** 3, 1),
                ("powerlaw_2m", lambda: synth.powerlaw_csr(2_000_000, 2_000_000, 1, storage),
                 2_000_000, 1024)):
            rp, ci, v = make()
            rpd, cid, vd = rp.to(dev), ci.to(dev), v.to(dev)
            m, nnz = rp.numel() - 1, v.numel()
            x = synth.device_uniform_(torch.empty(ncols, dtype=vd.dtype, device=dev), 1201)
            y = torch.empty(m, dtype=vd.dtype, device=dev)
            csr_bytes = nnz * (es + 4) + (m + 1) * 4 + ncols * es + m * es
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            A = SellMatrix(rpd, cid, vd, ncols, sigma=sigma)
            torch.cuda.synchronize()
            conv_ms = (time.perf_counter() - t0) * 1e3
            ns = (m + 31) // 32
            sell_bytes = A.total * (es + 4) + ns * 12 + (m + 31) // 32 * 32 * 4 + ncols * es + m * es
            best = None
            for cfg in ((256, 0, 4, 0), (128, 0, 8, 0), (512, 0, 2, 0), (256, 0, 8, 0)):
                f = (lambda c=cfg: A.spmv(x, y=y, cfg=c))
                f()
                t = _launch_ms(f, reps, flush)
                if best is None or t < best[0]:
                    best = (t, cfg)
            fc = (lambda: lak.csr_spmv(rpd, cid, vd, x, y=y))
            fc()
            tc = _launch_ms(fc, reps, flush)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Bm = BinnedCsr(rpd, cid, vd, ncols)
            torch.cuda.synchronize()
            bin_build_ms = (time.perf_counter() - t0) * 1e3
            fb = (lambda: Bm.spmv(x, y=y))
            fb()
            tb = _launch_ms(fb, reps, flush)
            bins = Bm.bin_ptr.cpu().tolist()
            del Bm
            out[f"{name}_{storage}"] = {
                "csr_us": round(tc * 1e3, 2), "csr_GBs": round(csr_bytes / (tc * 1e-3) / 1e9, 1),
                "sell_us": round(best[0] * 1e3, 2), "sell_cfg": list(best[1]),
                "sell_GBs_csr_bytes": round(csr_bytes / (best[0] * 1e-3) / 1e9, 1),
                "sell_padding": round(A.total / max(nnz, 1) - 1, 4), "sigma": sigma,
                "speedup_vs_csr": round(tc / best[0], 3), "conversion_ms": round(conv_ms, 2),
                "sell_bytes_read": sell_bytes,
                "binned_us": round(tb * 1e3, 2),
                "binned_GBs_csr_bytes": round(csr_bytes / (tb * 1e-3) / 1e9, 1),
                "binned_speedup_vs_csr": round(tc / tb, 3),
                "binned_build_ms": round(bin_build_ms, 2), "binned_rows_per_bin":
                    [bins[i + 1] - bins[i] for i in range(len(bins) - 1)]}
            del A
    return out


def run_profile_set(device):
    """Every kernel family once, at sizes above L2 but a small device footprint
    (under 5 GB), for an ncu capture of all of them in one command.  Prints one
    JSON line mapping each launch (in order) to its algorithmic bytes."""
    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300 import autograd as ag
    from paper_1409_0669_gb300 import batch as B
    from paper_1409_0669_gb300.csr_bin import BinnedCsr
    from paper_1409_0669_gb300.sell import SellMatrix

    dev = device
    launches = []

    def rec(name, nbytes, fn):
        fn()
        launches.append({"name": name, "bytes": int(nbytes)})

    n = 50_000_000
    y = synth.device_uniform_(torch.empty(n, device=dev), 1301)
    z = synth.device_uniform_(torch.empty(n, device=dev), 1302)
    x = torch.empty_like(y)
    ws = torch.zeros(64 << 20, dtype=torch.uint8, device=dev)
    out = torch.zeros(1, device=dev)
    rec("copy_f32", 8 * n, lambda: lak.vec_copy(x, y))
    rec("axpy_f32", 12 * n, lambda: lak.vec_axpy(x, y, z, 0.5))
    rec("dot_f32", 8 * n, lambda: lak.vec_dot(y, z, workspace=ws))
    rec("dot_compensated_f32", 8 * n, lambda: lak.vec_dot_compensated(y, z, workspace=ws))
    rec("axpby_f32", 12 * n, lambda: lak.vec_axpby(x, 0.5, y, -1.5, z))
    # the strided update on every second element (algorithmic bytes: the
    # elements used; DRAM moves whole sectors, so about twice as many)
    rec("axpby_strided2_f32", 12 * (n // 2),
        lambda: lak.vec_axpby(x[::2], 0.5, y[::2], -1.5, z[::2]))
    rec("axpy_norm2_f32", 12 * n, lambda: lak.vec_axpy_norm2(x, y, z, 0.5, workspace=ws))
    rec("scale_dev_f32", 8 * n, lambda: lak.vec_scale_dev(y, out.fill_(2.0), out=x))
    rec("dot_noalloc_f32", 8 * n, lambda: lak.vec_dot_noalloc(y, z))
    g = 8192
    A = synth.device_normal_(torch.empty(g, g, device=dev), 1303)
    xg = synth.device_uniform_(torch.empty(g, device=dev), 1304)
    yg = torch.empty(g, device=dev)
    gb = (g * g + 2 * g) * 4
    rec("gemv_row_f32", gb, lambda: lak.dense_gemv(A, xg, y=yg))
    rec("gemv_col_f32", gb, lambda: lak.dense_gemv(A.t(), xg, y=yg, workspace=ws))
    rec("gemv_axpby_row_f32", gb + 8 * g, lambda: lak.dense_gemv(A, xg, y=yg, alpha=2.0, beta=1.0))
    rec("dense_outer_f32", gb, lambda: lak.dense_outer(xg, yg, out=A))
    A64 = synth.device_normal_(torch.empty(g // 2, g, dtype=torch.float64, device=dev), 1305)
    x64 = synth.device_uniform_(torch.empty(g, dtype=torch.float64, device=dev), 1306)
    rec("gemv_row_f64", (g // 2 * g + g + g // 2) * 8, lambda: lak.dense_gemv(A64, x64))
    del A, A64
    for nm, (rp, ci, v), nc, sig in (
            ("lap3d_128", synth.laplacian_3d(128, "f32"), 128 ** 3, 1),
            ("powerlaw_2m", synth.powerlaw_csr(2_000_000, 2_000_000, 1, "f32"), 2_000_000, 1024)):
        rpd, cid, vd = rp.to(dev), ci.to(dev), v.to(dev)
        m, nnz = rp.numel() - 1, v.numel()
        xs = synth.device_uniform_(torch.empty(nc, device=dev), 1307)
        ys = torch.empty(m, device=dev)
        sb = nnz * 8 + (m + 1) * 4 + nc * 4 + m * 4
        rec(f"spmv_csr_{nm}_f32", sb, lambda: lak.csr_spmv(rpd, cid, vd, xs, y=ys))
        S = SellMatrix(rpd, cid, vd, nc, sigma=sig)
        rec(f"spmv_sell_{nm}_f32", sb, lambda: S.spmv(xs, y=ys))
        Bn = BinnedCsr(rpd, cid, vd, nc)
        rec(f"spmv_binned_{nm}_f32", sb, lambda: Bn.spmv(xs, y=ys))
        dv = torch.empty(nnz, device=dev)
        rec(f"sampled_outer_{nm}_f32", nnz * 8 + (m + 1) * 4 + nc * 4 + m * 4,
            lambda: lak.csr_sampled_outer(rpd, cid, ys, xs, out=dv))
        pat = ag.CsrPattern(rpd, cid, nc)
        cp, ri, perm = pat.transpose()
        rec(f"gather_{nm}_f32", nnz * 12, lambda: lak.vec_gather(vd, perm, out=dv))
        rec(f"dot_sparse_{nm}_f32", nnz * 8,
            lambda: lak.vec_dot_sparse(vd, cid, xs, out=out, workspace=ws))
        del S, Bn
    ns = synth.log_uniform_ints(512, 65_536, 1_048_576, 1308)
    bx = [torch.empty(int(k), device=dev) for k in ns]
    byy = [synth.device_uniform_(torch.empty(int(k), device=dev), 1309) for k in ns]
    bz = [synth.device_uniform_(torch.empty(int(k), device=dev), 1310) for k in ns]
    bt = B.axpy_batch(bx, byy, bz, [0.5] * len(ns))
    rec("batch_axpy_f32", 12 * int(sum(int(k) for k in ns)), bt.run)
    bouts = torch.zeros(len(ns), device=dev)
    bd = B.dot_batch(byy, bz, [bouts[i:i + 1] for i in range(len(ns))])
    rec("batch_dot_f32", 8 * int(sum(int(k) for k in ns)), bd.run)
    gm = synth.log_uniform_ints(256, 64, 4096, 1311)
    gn = synth.log_uniform_ints(256, 64, 4096, 1312)
    gA = [synth.device_normal_(torch.empty(int(a), int(b), device=dev), 1313) for a, b in zip(gm, gn)]
    gx = [synth.device_uniform_(torch.empty(int(b), device=dev), 1314) for b in gn]
    gy = [torch.empty(int(a), device=dev) for a in gm]
    bg = B.gemv_batch(gA, gx, gy)
    rec("batch_gemv_f32", 4 * int(sum(int(a) * int(b) + int(a) + int(b) for a, b in zip(gm, gn))),
        bg.run)
    del gA
    # the first 256 instances of the batched leg's CSR family (same seeds)
    cm = synth.log_uniform_ints(256, 1000, 200_000, 4005)
    csrs, cxs, cys, cb = [], [], [], 0
    for i, m in enumerate(cm):
        m = int(m)
        rp, ci, v = synth.device_csr_block_(m, 44000 + i, 5, 64, torch.float32, dev)
        csrs.append((rp, ci, v, m))
        cxs.append(synth.device_uniform_(torch.empty(m, device=dev), 64000 + i))
        cys.append(torch.zeros(m, device=dev))
        cb += v.numel() * 8 + (m + 1) * 4 + 2 * m * 4
    bs = B.spmv_batch(csrs, cxs, cys)
    rec("batch_spmv_f32", cb, bs.run)
    torch.cuda.synchronize()
    print(json.dumps({"profile_set": launches}))
    return 0


# kernel source files per op, hashed into a traffic record: a record stands only
# while these files and the resolved launch configuration are unchanged
TRAFFIC_SOURCES = {
    "copy": ("paper_1409_0669_gb300/csrc/k_vec.cu",),
    "axpy": ("paper_1409_0669_gb300/csrc/k_vec.cu",),
    "dot": ("paper_1409_0669_gb300/csrc/k_vec.cu",),
    "gemv_row": ("paper_1409_0669_gb300/csrc/k_gemv.cu", "paper_1409_0669_gb300/csrc/gemv_row.cuh"),
    "gemv_col": ("paper_1409_0669_gb300/csrc/k_gemv.cu",),
    "spmv": ("paper_1409_0669_gb300/csrc/k_spmv.cu", "paper_1409_0669_gb300/csrc/spmv_seg.cuh"),
}
_COMMON_SOURCES = ("paper_1409_0669_gb300/csrc/lak_internal.cuh",)


def _sources_digest(op):
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES[op] + _COMMON_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _item_cfg(it):
    """The launch configuration the library resolves for a sweep item."""
    import paper_1409_0669_gb300 as lak
    if it.op == "spmv":
        m, n, nnz = it.args[5], it.args[6], it.args[7]
    elif it.op.startswith("gemv"):
        m = n = it.size
        nnz = 0
    else:
        m = n = it.size
        nnz = 0
    c = lak.resolve_cfg(it.op, it.dtype, m, n, nnz)
    return [c.block, c.grid, c.vec, c.increment]


def recorded_traffic(path, it):
    """DRAM bytes per launch recorded by an ncu capture of this launch, or None
    when there is no record, or the kernel's sources or its resolved launch
    configuration changed since the capture."""
    if not path or not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh).get(it.name)
    if not rec:
        return None
    try:
        if rec.get("sources_sha256") != _sources_digest(it.op) or rec.get("cfg") != _item_cfg(it):
            return None
    except OSError:
        return None
    return rec["dram_bytes"]


def record_traffic(csv_path, out_path, only):
    """Write DRAM bytes per launch from an ncu CSV (metrics dram__bytes_read.sum
    and dram__bytes_write.sum, one captured launch per selected sweep item, in
    sweep order) into the traffic record, with the sources' digest and the
    resolved configuration of each launch."""
    import csv
    import re

    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    items, keep = build_sweep(device, torch.cuda.current_stream().cuda_stream,
                              re.compile(only) if only else None)
    per_launch = {}
    with open(csv_path) as fh:
        rows = [r for r in csv.reader(fh) if len(r) > 5]
    head = rows[0]
    i_id, i_name, i_val = head.index("ID"), head.index("Metric Name"), head.index("Metric Value")
    for r in rows[1:]:
        if r[i_name] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            per_launch.setdefault(int(r[i_id]), 0.0)
            per_launch[int(r[i_id])] += float(r[i_val].replace(",", ""))
    launches = [per_launch[k] for k in sorted(per_launch)]
    if len(launches) < len(items):
        raise SystemExit(f"{len(launches)} launches in {csv_path}, {len(items)} items selected")
    try:
        with open(out_path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    data["_about"] = ("dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu "
                      "capture; bench.py reports a value only while the kernel sources and the "
                      "launch's resolved configuration are unchanged")
    for it, b in zip(items, launches):
        data[it.name] = {"dram_bytes": int(b), "sources_sha256": _sources_digest(it.op),
                         "cfg": _item_cfg(it), "algorithmic_bytes": it.nbytes}
    with open(out_path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    del keep
    return 0


def _launch_ms(fn, reps, flush=None):
    """Device time of one call of `fn` in ms (CUDA events on the current
    stream).  With `flush` (a buffer larger than L2, read before every call to
    evict L2 without leaving dirty lines): the calls and flushes run back to
    back in one event interval and the flushes' own time is subtracted --
    GB300's event clock ticks in ~2 us steps, too coarse for one short launch.
    Without: the trimmed mean of per-call intervals."""
    from paper_1409_0669_gb300.timing import launch_time_us
    return launch_time_us(fn, reps, flush) * 1e-3


def run_precision(device, reps=20):
    """The same data stored in FP32, BF16 and FP16 (FP32 arithmetic): time of
    every kernel relative to FP32, and its error against the FP64 oracle on the
    ORIGINAL FP32 data (quantisation included); plus the compensated inner
    product on 1e8 mixed-sign values of magnitude 1e-4..1e4.  L2 is flushed
    (a 256 MB buffer read) before every timed launch."""
    import numpy as np
    import torch

    import oracle
    import paper_1409_0669_gb300 as lak
    import synth

    oracle.build()
    dev = device
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    n = 100_000_000
    g = 16384
    y32 = synth.device_uniform_(torch.empty(n, device=dev), 901)
    z32 = synth.device_uniform_(torch.empty(n, device=dev), 902)
    A32 = synth.device_normal_(torch.empty(g * g, device=dev), 903)
    xg32 = synth.device_uniform_(torch.empty(g, device=dev), 904)
    lap = synth.laplacian_3d(128, "f32")
    pl = synth.powerlaw_csr(2_000_000, 2_000_000, 1, "f32")
    xl32 = synth.device_uniform_(torch.empty(128 ** 3, device=dev), 905)
    xp32 = synth.device_uniform_(torch.empty(2_000_000, device=dev), 906)

    # FP64 oracle references on the original FP32 data
    rng = synth.rng(907)
    idx = np.sort(rng.choice(n, 1_000_000, replace=False))
    yh, zh = y32.cpu(), z32.cpu()
    ref = {"axpy": oracle.axpy(yh.numpy()[idx], zh.numpy()[idx], 0.5),
           "dot": oracle.dot(yh, zh)}
    dot_scale = float(np.linalg.norm(yh.double().numpy()) * np.linalg.norm(zh.double().numpy()))
    del yh, zh
    rows = np.sort(rng.choice(g, 96, replace=False))
    Ah, xgh = A32.cpu(), xg32.cpu()
    ref["gemv_row"] = oracle.gemv_entries(Ah, xgh, rows, g, g, "row")
    ref["gemv_col"] = oracle.gemv_entries(Ah, xgh, rows, g, g, "col")
    del Ah
    ref["spmv_lap3d"] = oracle.csr_spmv(lap[0], lap[1], lap[2], xl32.cpu())
    ref["spmv_powerlaw"] = oracle.csr_spmv(pl[0], pl[1], pl[2], xp32.cpu())

    def rel(got, r):
        return float(np.linalg.norm(got - r) / np.linalg.norm(r))

    out = {}
    base = {}
    for storage in ("f32", "bf16", "f16"):
        dt = synth.torch_dtype(storage)
        es = torch.tensor([], dtype=dt).element_size()
        y, z = y32.to(dt), z32.to(dt)
        x = torch.empty_like(y)
        A, xg = A32.to(dt), xg32.to(dt)
        Am = A.view(g, g)
        rp_l, ci_l, v_l = lap[0].to(dev), lap[1].to(dev), lap[2].to(dev).to(dt)
        rp_p, ci_p, v_p = pl[0].to(dev), pl[1].to(dev), pl[2].to(dev).to(dt)
        xl, xp = xl32.to(dt), xp32.to(dt)
        ws = torch.zeros(max(lak.vec_dot_workspace(n, storage),
                             lak.dense_gemv_workspace(g, g, "col", storage), 256),
                         dtype=torch.uint8, device=dev)
        yo = torch.empty(g, dtype=dt, device=dev)
        sl = torch.empty(rp_l.numel() - 1, dtype=dt, device=dev)
        sp = torch.empty(rp_p.numel() - 1, dtype=dt, device=dev)
        cases = {
            "axpy": (lambda: lak.vec_axpy(x, y, z, 0.5), 3 * n * es),
            "dot": (lambda: lak.vec_dot(y, z, workspace=ws), 2 * n * es),
            "gemv_row": (lambda: lak.dense_gemv(Am, xg, y=yo), (g * g + 2 * g) * es),
            "gemv_col": (lambda: lak.dense_gemv(Am.t(), xg, y=yo, workspace=ws), (g * g + 2 * g) * es),
            "spmv_lap3d": (lambda: lak.csr_spmv(rp_l, ci_l, v_l, xl, y=sl),
                           v_l.numel() * (es + 4) + rp_l.numel() * 4 + 2 * sl.numel() * es),
            "spmv_powerlaw": (lambda: lak.csr_spmv(rp_p, ci_p, v_p, xp, y=sp),
                              v_p.numel() * (es + 4) + rp_p.numel() * 4 + 2 * sp.numel() * es),
        }
        def arithmetic_error(name, storage):
            """Against the oracle on the STORED (quantised) inputs, the oracle's
            result rounded to the storage type like the kernel's: the error of
            the arithmetic alone (FP32 accumulation), without quantisation."""
            if name == "axpy":
                r = oracle.round_to(oracle.axpy(y.cpu()[idx], z.cpu()[idx], 0.5), storage)
                return rel(oracle.widen(x.cpu())[idx], r)
            if name == "dot":
                yq, zq = y.cpu(), z.cpu()
                r = oracle.dot(yq, zq)
                sc = float(np.linalg.norm(oracle.widen(yq)) * np.linalg.norm(oracle.widen(zq)))
                return abs(dot_out[0] - r) / sc
            if name in ("gemv_row", "gemv_col"):
                lay = "row" if name == "gemv_row" else "col"
                r = oracle.round_to(oracle.gemv_entries(A.cpu(), xg.cpu(), rows, g, g, lay), storage)
                return rel(oracle.widen(yo.cpu())[rows], r)
            if name == "spmv_lap3d":
                r = oracle.round_to(oracle.csr_spmv(lap[0], lap[1], v_l.cpu(), xl.cpu()), storage)
                return rel(oracle.widen(sl.cpu()), r)
            r = oracle.round_to(oracle.csr_spmv(pl[0], pl[1], v_p.cpu(), xp.cpu()), storage)
            return rel(oracle.widen(sp.cpu()), r)

        dot_out = [0.0]
        for name, (fn, nbytes) in cases.items():
            for _ in range(3):
                fn()
            ms = _launch_ms(fn, reps, flush)
            # error of this launch's result
            if name == "axpy":
                fn()
                got = oracle.widen(x.cpu())[idx]
                err = rel(got, ref["axpy"])
            elif name == "dot":
                d = fn().item()
                dot_out[0] = d
                err = abs(d - ref["dot"]) / dot_scale
            elif name in ("gemv_row", "gemv_col"):
                got = oracle.widen(fn().cpu())[rows]
                err = rel(got, ref[name])
            else:
                err = rel(oracle.widen(fn().cpu()), ref[name])
            rec = {"us": round(ms * 1e3, 2), "GBs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                   "err": err}
            if storage != "f32":
                rec["err_arith"] = arithmetic_error(name, storage)
            if storage == "f32":
                base[name] = ms
            else:
                rec["time_vs_f32"] = round(ms / base[name], 4)
            out.setdefault(name, {})[storage] = rec
        del y, z, x, A, Am, xg, v_l, v_p, xl, xp
    out["error_definition"] = ("err: norm-wise relative error vs the FP64 oracle on the original "
                               "FP32 data (dot: |s-s*| / (||x|| ||y||)), quantisation included; "
                               "stated bound 1e-2 for BF16.  err_arith: vs the oracle on the stored "
                               "(quantised) inputs with its result rounded to the storage type "
                               "like the kernel's -- the FP32 arithmetic alone")

    # compensated vs plain inner product on mixed magnitudes
    a = synth.device_mixed_magnitude_(torch.empty(n, device=dev), 908)
    b = synth.device_mixed_magnitude_(torch.empty(n, device=dev), 909)
    ws = torch.zeros(lak.vec_dot_workspace(n, "f32"), dtype=torch.uint8, device=dev)
    ah, bh = a.cpu(), b.cpu()
    r = oracle.dot(ah, bh)
    abs_sum = float(np.abs(ah.double().numpy() * bh.double().numpy()).sum())
    del ah, bh
    comp = {}
    for label, fn in (("plain_f32", lambda: lak.vec_dot(a, b, workspace=ws)),
                      ("compensated_f32", lambda: lak.vec_dot_compensated(a, b, workspace=ws))):
        for _ in range(3):
            fn()
        ms = _launch_ms(fn, reps, flush)
        v = fn().item()
        comp[label] = {"us": round(ms * 1e3, 2), "GBs": round(2 * n * 4 / (ms * 1e-3) / 1e9, 1),
                       "rel_err": abs(v - r) / abs(r), "err_over_abs_sum": abs(v - r) / abs_sum}
    comp["time_compensated_vs_plain"] = round(comp["compensated_f32"]["us"] /
                                              comp["plain_f32"]["us"], 4)
    out["dot_mixed_magnitude_1e8"] = comp
    return out


def bind_to_gpu_numa(device):
    """Pin this process to the host cores of the GPU's own NUMA node (as read
    from sysfs for its PCI address), so that pinned host buffers are
    first-touched in memory next to the GPU's host link.  Best effort: returns
    a description, or None when the platform does not say."""
    import torch
    try:
        p = torch.cuda.get_device_properties(device)
        addr = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{addr}"
        with open(base + "/local_cpulist") as fh:
            spec = fh.read().strip()
        with open(base + "/numa_node") as fh:
            node = fh.read().strip()
    except (AttributeError, OSError):
        return None
    cpus = set()
    for part in spec.split(","):
        if not part:
            continue
        lo, _, hi = part.partition("-")
        cpus.update(range(int(lo), int(hi or lo) + 1))
    allowed = os.sched_getaffinity(0)
    use = cpus & allowed
    if not use or use == allowed:
        return {"pci": addr, "numa_node": node, "cpus": spec, "bound": False}
    os.sched_setaffinity(0, use)
    return {"pci": addr, "numa_node": node, "cpus": spec, "bound": True}


HEADLINE_MAX_BYTES = 3072


def _r(v, nd):
    return None if v is None else round(float(v), nd)


def headline(*, value, ms_per_step, steps, warmup, world, workload, bytes_per_step, launches,
             roofline, per_kernel, e2e, cpu, clocks, detail_path, probe=None, gprobe=None):
    """The one JSON line the run ends with: the headline metric and the keys a
    reader needs to check it (roofline of the dominant kernel, per-kernel
    GB/s at the largest sizes, end to end, CPU baseline, clocks), kept within
    HEADLINE_MAX_BYTES.  Everything else goes to the detail file it names."""
    rl = None
    if roofline is not None:
        rl = {k: roofline.get(k) for k in ("bound", "unit", "kernel")}
        for k, nd in (("achieved", 4), ("peak", 4), ("frac", 4), ("share", 4),
                      ("ms_per_launch", 5)):
            rl[k] = _r(roofline.get(k), nd)
        rl["traffic"] = roofline.get("traffic")
        rl["bytes_per_launch"] = roofline.get("bytes_per_launch")
        rl["flops_per_launch"] = roofline.get("flops_per_launch")
        rl["peak_source"] = str(roofline.get("peak_source", ""))[:80]
        if roofline.get("peak_nominal") is not None:
            rl["peak_nominal"] = _r(roofline["peak_nominal"], 4)
        other = roofline.get("other")
        if other:
            rl["other"] = {"bound": other.get("bound"), "unit": other.get("unit"),
                           "achieved": _r(other.get("achieved"), 4),
                           "peak": _r(other.get("peak"), 4), "frac": _r(other.get("frac"), 4)}
    pk, pp = {}, {}
    for key, v in (per_kernel or {}).items():
        if key.startswith("paper_point_"):
            pp[key[len("paper_point_"):]] = _r(v.get("GBs"), 1)
            continue
        ent = {"GBs": _r(v.get("GBs"), 1), "frac_hbm": _r(v.get("frac_hbm"), 3)}
        if v.get("bound") not in (None, "hbm"):
            ent["bound"] = v["bound"]
            ent["frac_bound"] = _r(v.get("frac_bound"), 3)
        pk[key] = ent
    e2 = None
    if e2e is not None:
        e2 = {"value": _r(e2e.get("value"), 2), "unit": e2e.get("unit", "GB/s"),
              "h2d_bytes_per_step": e2e.get("h2d_bytes_per_step"),
              "d2h_bytes_per_step": e2e.get("d2h_bytes_per_step"),
              "ms_per_step": _r(e2e.get("ms_per_step"), 3)}
    cb = None
    if cpu is not None:
        cb = {"value": _r(cpu.get("value"), 3), "unit": cpu.get("unit", "GB/s"),
              "cores": cpu.get("cores"), "kind": cpu.get("kind", "oracle"),
              "sample": str(cpu.get("sample", ""))[:200]}
        for k in ("all_cores", "plain_loop"):
            if cpu.get(k):
                cb[k] = {kk: (_r(vv, 3) if isinstance(vv, float) else vv)
                         for kk, vv in cpu[k].items() if kk in ("value", "cores", "unit")}
        if cpu.get("host"):
            cb["host"] = str(cpu["host"])[:80]
    ck = None
    if clocks is not None:
        ck = {"sm_mhz": clocks.get("sm_mhz"), "sm_max_mhz": clocks.get("sm_max_mhz"),
              "reasons": clocks.get("reasons"), "samples": clocks.get("samples")}
    line = {
        "metric": METRIC, "value": _r(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": _r(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": workload, "bytes_per_step": bytes_per_step,
                   "launches_per_step": launches,
                   "l2": "no flush: inputs larger than L2, >1 GB of other traffic between "
                         "two uses of a buffer",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": rl, "per_kernel": pk, "paper_points_GBs": pp, "e2e": e2,
        "gpu_launches": launches * steps, "clocks": ck,
    }
    if cb is not None:
        line["cpu_baseline"] = cb
    if probe is not None:
        line["fp64_probe"] = {"tflops": _r(probe.get("tflops"), 4), "sm_mhz": probe.get("sm_mhz"),
                              "fma_per_sm_per_clk": _r(probe.get("fma_per_sm_per_clk"), 3)}
    if gprobe is not None:
        line["gather_probe"] = {"G_per_s": _r(gprobe.get("gathers_per_s", 0) / 1e9, 1),
                                "per_sm_per_clk": _r(gprobe.get("per_sm_per_clk"), 3)}
    if detail_path:
        line["detail"] = os.path.basename(detail_path)
    return line


def run_gb300(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    host_binding = bind_to_gpu_numa(device)
    dist = init_dist(world, "nccl")

    import paper_1409_0669_gb300 as lak  # noqa: F401
    from paper_1409_0669_gb300 import _native

    stream = torch.cuda.Stream(device=device)
    sh = stream.cuda_stream
    import re
    only = re.compile(args.only) if args.only else None
    with torch.cuda.stream(stream):
        items, keep = build_sweep(device, sh, only)
    torch.cuda.synchronize()

    def lib_check(name, st):
        raise _native.LakError(name, st, _native.last_error())

    bytes_per_step = sum(it.nbytes for it in items)
    K, W = args.steps, args.warmup
    with torch.cuda.stream(stream):
        for _ in range(W):
            run_step(items, lib_check)
    torch.cuda.synchronize()

    # per-launch events on the launching stream for the watched launches, all K steps
    watch = watched_items(items)
    ev = [{i: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for i in watch} for _ in range(K)]
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(dist, device)
    torch.cuda.synchronize()
    t_window = time.monotonic()
    with torch.cuda.stream(stream):
        start.record()
        for k in range(K):
            run_step(items, lib_check, ev[k])
        stop.record()
    torch.cuda.synchronize()
    t_window = (t_window, time.monotonic())
    barrier(dist, device)
    time.sleep(0.2)
    clocks = sampler.stop(t_window)
    elapsed_ms = start.elapsed_time(stop)
    elapsed_ms = max_over_ranks(elapsed_ms, dist, device)

    per = {}
    for i in watch:
        it = items[i]
        t = sum(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(K)) / K
        per[it.name] = (it, t)
    step_ms = elapsed_ms / K

    ms_per_step = elapsed_ms / K
    value = world * bytes_per_step / (ms_per_step * 1e-3) / 1e9
    peak, peak_kind = load_peaks()

    # dominant kernel: largest share of the step time.  The FP64 roof is the
    # FMA rate measured now (the probe); the unit-count figure is kept beside it
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    fp64_nominal = fp64_peak_tflops(sms, sm_mhz)
    probe = fp64_probe(device, stream)
    fp64_peak = probe["tflops"]
    dom_name, (dom_it, dom_ms) = max(per.items(), key=lambda kv: kv[1][1])
    bind, other = roofline_of(dom_it, dom_ms, peak, peak_kind, fp64_peak)
    roofline = dict(bind)
    roofline.update({"traffic": None, "kernel": dom_name, "share": dom_ms / step_ms,
                     "bytes_per_launch": dom_it.nbytes, "flops_per_launch": flops_of(dom_it),
                     "ms_per_launch": dom_ms})
    if other is not None:
        roofline["other"] = {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    roofline["traffic"] = recorded_traffic(args.traffic_json, dom_it)
    if roofline["bound"] == "alu":
        roofline["peak_nominal"] = fp64_nominal

    # per (op, dtype) summary at the largest size, and the paper's points.
    # Launches under 100 us are re-timed like the copy and the gather floor
    # beside them (differential, L2 flushed): the sweep's per-launch events add
    # the launch's start-up and the ~2 us event tick to them.
    short = [name for name, (it, t) in per.items()
             if t < 0.1 and it.size not in (2154435, 2048)]
    with torch.cuda.stream(stream):
        short_us = differential_us(per, short, device, lib_check)
    summary = {}
    for name, (it, t_ev) in per.items():
        if it.size in (2154435, 2048):
            continue
        key = f"{it.op}_{name.split('_')[1]}_{it.dtype}" if it.op == "spmv" else \
            f"{it.op}_{it.dtype}"
        t = short_us[name] * 1e-3 if name in short_us else t_ev
        gbs = it.nbytes / (t * 1e-3) / 1e9
        b, _ = roofline_of(it, t, peak, peak_kind, fp64_peak)
        summary[key] = {"size": it.size, "GBs": round(gbs, 1), "frac_hbm": round(gbs / peak, 4),
                        "us": round(t * 1e3, 2), "bound": b["bound"],
                        "frac_bound": round(b["frac"], 4)}
        if name in short_us:
            summary[key]["us_events_in_sweep"] = round(t_ev * 1e3, 2)
    # the copy kernel moving the same number of bytes (cold): the streaming
    # ceiling at that size, launch and DRAM-latency ramp included
    with torch.cuda.stream(stream):
        copy_same = copy_at_bytes([it.nbytes for it, _ in per.values()], device, lak)
    for key, v in summary.items():
        it = next((it for name, (it, _) in per.items()
                   if (f"{it.op}_{name.split('_')[1]}_{it.dtype}" if it.op == "spmv"
                       else f"{it.op}_{it.dtype}") == key and it.size == v["size"]), None)
        if it is not None and it.nbytes in copy_same:
            c = copy_same[it.nbytes]
            v["copy_same_bytes_GBs"] = round(c, 1)
            v["frac_copy_same_bytes"] = round(v["GBs"] / c, 4)
    # CSR SpMV: the floor set by its x gather -- the sparse inner product over
    # the matrix's own entries (vec_dot_sparse) timed alone
    with torch.cuda.stream(stream):
        floors = gather_floors(per, lak)
        gprobe = gather_probe(device)
    # The sparse inner product is a floor only where the columns are random (the
    # power-law matrix): a stencil's x reuse lets a row-parallel kernel beat an
    # entry-parallel gather, so there it is reported but the roof stays HBM.
    for key, (g_us, name) in floors.items():
        if key in summary:
            t_us = summary[key]["us"]
            hbm_us = per[name][0].nbytes / (peak * 1e9) * 1e6
            summary[key]["gather_floor_us"] = round(g_us, 2)
            summary[key]["frac_gather_floor"] = round(g_us / t_us, 4)
            if "powerlaw" in name and g_us > hbm_us:
                summary[key]["bound"] = "gather"
                summary[key]["frac_bound"] = round(g_us / t_us, 4)
    # the paper's own points (FP64, 2.15e6-entry vectors, 2048^2): timed like the
    # copy beside them (differential, L2 flushed before every launch); the
    # per-launch events of the sweep add the launch's start-up and the ~2 us
    # event tick, a fifth of a 10-us call
    pp_names = ("copy_f64_2154435", "axpy_f64_2154435", "dot_f64_2154435", "gemv_row_f64_2048")
    with torch.cuda.stream(stream):
        pp_us = differential_us(per, pp_names, device, lib_check)
    for name in pp_names:
        if name in per:
            it, t_ev = per[name]
            t = pp_us[name] * 1e-3
            gbs = it.nbytes / (t * 1e-3) / 1e9
            summary["paper_point_" + name] = {"GBs": round(gbs, 1), "us": round(t * 1e3, 2),
                                              "us_events_in_sweep": round(t_ev * 1e3, 2)}
            if it.nbytes in copy_same:
                summary["paper_point_" + name]["copy_same_bytes_GBs"] = round(
                    copy_same[it.nbytes], 1)
                summary["paper_point_" + name]["frac_copy_same_bytes"] = round(
                    gbs / copy_same[it.nbytes], 4)

    if args.sweep_json:
        rows = [{"name": n, "op": it.op, "dtype": it.dtype, "size": it.size, "bytes": it.nbytes,
                 "us": t * 1e3, "GBs": it.nbytes / (t * 1e-3) / 1e9}
                for n, (it, t) in per.items()]
        with open(args.sweep_json, "w") as fh:
            json.dump({"peak_gbs": peak, "rows": rows}, fh, indent=1)

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(items, keep, stream, device, max(1, min(K, args.e2e_steps)), lib_check,
                      dist)
        e2e["host_binding"] = host_binding

    precision = None
    if not args.no_precision and not args.only and rank == 0:
        precision = run_precision(device)
    batched = None
    if not args.no_batched and not args.only and rank == 0:
        batched = run_batched(device)
    autograd = None
    if not args.no_autograd and not args.only and rank == 0:
        autograd = run_autograd(device)
    fused = None
    if not args.no_fused and not args.only and rank == 0:
        fused = run_fused(device)
    formats = None
    if not args.no_formats and not args.only and rank == 0:
        formats = run_formats(device)
    small = None
    if not args.no_small and not args.only and rank == 0:
        small = run_small(device)
    curves = None
    if not args.no_curves and not args.only and rank == 0:
        curves = run_size_curves(device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_seconds)

    workload = WORKLOAD if not args.only else f"subset /{args.only}/ of: " + WORKLOAD
    detail = {"per_kernel": summary, "roofline": roofline, "e2e": e2e, "clocks": clocks,
              "fp64_probe": probe, "gather_probe": gprobe,
              "config": {"workload": workload, "bytes_per_step": bytes_per_step,
                         "launches_per_step": len(items)}}
    for key, val in (("cpu_baseline", cpu), ("precision", precision), ("batched", batched),
                     ("autograd", autograd), ("fused", fused), ("spmv_formats", formats),
                     ("small_config", small), ("size_curves", curves)):
        if val is not None:
            detail[key] = val
    detail_path = None
    if rank == 0 and args.detail_json:
        detail_path = args.detail_json
        with open(detail_path, "w") as fh:
            json.dump(detail, fh, indent=1)
    line = headline(value=value, ms_per_step=ms_per_step, steps=K, warmup=W, world=world,
                    workload=workload, bytes_per_step=bytes_per_step,
                    launches=len(items), roofline=roofline, per_kernel=summary, e2e=e2e,
                    cpu=cpu, clocks=clocks, detail_path=detail_path, probe=probe,
                    gprobe=gprobe)
    if rank == 0:
        print(json.dumps(line, separators=(",", ":")))
    if dist is not None:
        dist.destroy_process_group()
    del keep
    return 0


def copy_at_bytes(sizes, device, lak, reps=10):
    """GB/s of vec_copy (FP32) moving each of the given byte counts (read +
    write), L2 cold: {bytes: GB/s}."""
    import torch
    from paper_1409_0669_gb300.timing import launch_time_us
    l2 = torch.cuda.get_device_properties(device).L2_cache_size
    top = max(sizes)
    src = torch.empty(top // 8 + 1, dtype=torch.float32, device=device)
    dst = torch.empty_like(src)
    src.zero_()
    flush = torch.empty(64 << 20, dtype=torch.float32, device=device)
    out = {}
    for b in sorted(set(sizes)):
        n = b // 8
        ys, xs = src[:n], dst[:n]
        lak.vec_copy(xs, ys)
        us = launch_time_us(lambda: lak.vec_copy(xs, ys), reps, flush if b < 2 * l2 else None)
        out[b] = 8 * n / (us * 1e-6) / 1e9
    del src, dst, flush
    return out


def differential_us(per, names, device, lib_check, reps=20):
    """Device time in us of each named sweep launch on its own, L2 cold
    (differential timing, like copy_at_bytes): for launches short enough that
    per-launch CUDA events would add their start-up and the event tick."""
    import torch
    from paper_1409_0669_gb300.timing import launch_time_us
    flush = torch.empty(64 << 20, dtype=torch.float32, device=device)
    out = {}
    for name in names:
        if name not in per:
            continue
        it = per[name][0]

        def call(it=it):
            st = it.fn(*it.args)
            if st != 0:
                lib_check(it.name, st)

        call()
        out[name] = launch_time_us(call, reps, flush)
    del flush
    return out


def gather_floors(per, lak, reps=20):
    """For every timed CSR SpMV launch: the device time of the sparse inner
    product sum_k vals[k] x[col_idx[k]] over the matrix's own values and
    column indices (vec_dot_sparse) -- every stored entry streamed and its x
    gathered exactly as a CSR product must, without the rows.  No CSR kernel
    on that matrix can be faster where the gather, not HBM, is the limit.
    Returns {summary key: (us, launch name)}."""
    import torch
    from paper_1409_0669_gb300.timing import launch_time_us
    out = {}
    for name, (it, _) in per.items():
        if it.op != "spmv":
            continue
        cid, vd, xsp = it.h2d[1], it.h2d[2], it.h2d[3]
        o = torch.empty(1, dtype=torch.float64 if it.dtype == "f64" else torch.float32,
                        device=xsp.device)
        ws = torch.zeros(lak.vec_dot_sparse_workspace(cid.numel(), it.dtype), dtype=torch.uint8,
                         device=xsp.device)
        lak.vec_dot_sparse(vd, cid, xsp, out=o, workspace=ws)
        us = launch_time_us(lambda: lak.vec_dot_sparse(vd, cid, xsp, out=o, workspace=ws), reps)
        out[f"spmv_{name.split('_')[1]}_{it.dtype}"] = (us, name)
        del ws
    return out


def gather_probe(device, n_gather=32_000_000, n_y=2_000_000, reps=20):
    """The rate of fully random 4-byte gathers: vec_dot_sparse over n_gather
    uniformly random indices into an FP32 vector of n_y entries (8 MB, held in
    L2), values all one -- the hardware rate that bounds any CSR product on
    random columns.  Returns gathers per second and per SM per clock (at the
    clock sampled meanwhile)."""
    import torch

    import paper_1409_0669_gb300 as lak
    from paper_1409_0669_gb300.timing import launch_time_us
    g = torch.Generator(device=device).manual_seed(77)
    idx = torch.randint(0, n_y, (n_gather,), generator=g, device=device, dtype=torch.int32)
    vals = torch.ones(n_gather, device=device)
    y = torch.rand(n_y, generator=g, device=device)
    out = torch.empty(1, device=device)
    ws = torch.zeros(lak.vec_dot_sparse_workspace(n_gather, "f32"), dtype=torch.uint8,
                     device=device)
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.1)
    lak.vec_dot_sparse(vals, idx, y, out=out, workspace=ws)
    us = launch_time_us(lambda: lak.vec_dot_sparse(vals, idx, y, out=out, workspace=ws), reps)
    clocks = sampler.stop()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    rate = n_gather / (us * 1e-6)
    mhz = clocks.get("sm_mhz")
    del idx, vals, y, ws
    return {"gathers_per_s": rate, "us": us, "gathers": n_gather, "y_entries": n_y,
            "per_sm_per_clk": rate / (sms * mhz * 1e6) if mhz else None, "sm_mhz": mhz}


def run_small(device, reps=200):
    """The small FP32 configuration: 2D 5-point Laplacian 256^2 (65,536 rows,
    values 4/-1), x = y + 0.5 z and <x, y> on n = 65,536 (U(-1,1), seed 0),
    y = A x in CSR, and a 1024^2 row-major GEMV (N(0,1)).  Latency bound, so
    reported in microseconds: each call issued from the host back to back,
    the four calls in sequence issued from the host, and the same sequence
    captured once in a CUDA graph and replayed (operands L2-resident)."""
    import torch

    import paper_1409_0669_gb300 as lak
    import synth
    from paper_1409_0669_gb300.timing import warm_time_us
    dev = device
    n = 65536
    y = synth.uniform(n, 0, "f32").to(dev)
    z = synth.uniform(n, 1, "f32").to(dev)
    x = torch.empty_like(y)
    out = torch.zeros(1, device=dev)
    ws = torch.zeros(max(lak.vec_dot_workspace(n, "f32"), 256), dtype=torch.uint8, device=dev)
    rp, ci, v = synth.laplacian_2d(256, "f32")
    rp, ci, v = rp.to(dev), ci.to(dev), v.to(dev)
    xs = synth.uniform(n, 2, "f32").to(dev)
    ys = torch.empty(n, device=dev)
    g = 1024
    A = synth.device_normal_(torch.empty(g, g, device=dev), 3)
    xg = synth.uniform(g, 4, "f32").to(dev)
    yg = torch.empty(g, device=dev)
    calls = {
        "axpy": (lambda: lak.vec_axpy(x, y, z, 0.5), 3 * n * 4),
        "dot": (lambda: lak.vec_dot(x, y, out=out, workspace=ws), 2 * n * 4),
        "spmv_lap2d_256": (lambda: lak.csr_spmv(rp, ci, v, xs, y=ys),
                           v.numel() * 8 + rp.numel() * 4 + 2 * n * 4),
        "gemv_row_1024": (lambda: lak.dense_gemv(A, xg, y=yg), (g * g + 2 * g) * 4),
    }
    rep = {}
    for name, (fn, nbytes) in calls.items():
        us = warm_time_us(fn, reps)
        rep[name] = {"us_launches": round(us, 2), "bytes": nbytes,
                     "GBs": round(nbytes / (us * 1e-6) / 1e9, 1)}

    def sequence():
        for fn, _ in calls.values():
            fn()
    seq_us = warm_time_us(sequence, reps)
    sequence()
    torch.cuda.synchronize()
    gr = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(cap):
        with torch.cuda.graph(gr, stream=cap):
            sequence()
    torch.cuda.synchronize()
    graph_us = warm_time_us(gr.replay, reps)
    rep["sequence_4_calls"] = {"us_launches": round(seq_us, 2), "us_graph_replay": round(graph_us, 2)}
    rep["timing"] = ("device time per call, calls back to back in one CUDA-event interval "
                     "(operands L2-resident); the graph holds the same four calls")
    return rep


def run_size_curves(device, reps=10):
    """GB/s against size for copy, x = y + 0.5 z and <y, z> (n = 1e3..1e8, 3 per
    decade) and both GEMV layouts (512^2..16384^2), FP32 and FP64, with the
    default launch configuration: cold = L2 evicted before every launch (a
    256 MB read; differential event timing) where the operands fit twice in L2,
    else launch by launch; warm = operands left in L2 by the previous launch
    (back-to-back launches), for working sets that fit in L2 only."""
    import torch

    import synth
    from paper_1409_0669_gb300 import autotune
    l2 = torch.cuda.get_device_properties(device).L2_cache_size
    rows = []
    for storage in ("f32", "f64"):
        for op in ("copy", "axpy", "dot"):
            for n in synth.vector_sweep_sizes():
                rows.append((op, storage, n))
        for op in ("gemv_row", "gemv_col"):
            for n in synth.gemv_sweep_sizes():
                rows.append((op, storage, n))
    out = {}
    for op, storage, n in rows:
        prob = autotune.Problem(op, storage, n, device)
        cold = prob.time_cfg(None, reps)
        rec = {"bytes": prob.nbytes, "cold_us": round(cold, 3),
               "cold_GBs": round(prob.nbytes / (max(cold, 1e-3) * 1e-6) / 1e9, 1)}
        if prob.footprint < l2:
            warm = prob.time_warm(None, 4 * reps)
            rec.update({"warm_us": round(warm, 3),
                        "warm_GBs": round(prob.nbytes / (max(warm, 1e-3) * 1e-6) / 1e9, 1)})
        out.setdefault(f"{op}_{storage}", {})[str(n)] = rec
        del prob
    torch.cuda.empty_cache()
    return out


def e2e_copy_bytes(items):
    """(host->device, device->host) bytes of one end-to-end step: every distinct
    input tensor (same data pointer, length and dtype) once, every launch's
    results each time."""
    distinct = {(t.data_ptr(), t.numel(), t.dtype): t for it in items for t in it.h2d}
    h2d = sum(t.numel() * t.element_size() for t in distinct.values())
    d2h = sum(t.numel() * t.element_size() for it in items for t in it.d2h)
    return h2d, d2h


def run_e2e(items, keep, stream, device, steps, lib_check, dist):
    """The same step through the C ABI with inputs in pinned host memory: every
    step copies each distinct input host->device once (before its first
    launch in the step), runs the launches, and copies every result
    device->host after its launch; the copies are inside the timed region.
    Three streams form a pipeline (host->device copies, the kernels,
    device->host copies), ordered per buffer with events: a copy into a
    buffer waits for the last kernel or read-back that used it, a kernel
    waits for its input copies and for the read-back of its previous output,
    a read-back waits for its kernel.  The copies of one launch thus overlap
    the kernel and the read-back of the previous ones, in both directions at
    once."""
    import torch
    # one pinned host copy per distinct device input / output tensor
    hmap = {}
    for it in items:
        for t in tuple(it.h2d) + tuple(it.d2h):
            key = (t.data_ptr(), t.numel(), t.dtype)
            if key not in hmap:
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t)
                hmap[key] = h
    def key_of(t):
        return (t.data_ptr(), t.numel(), t.dtype)

    # every distinct input is copied once per step (copy, update and dot of one
    # size read the same y and z); every result is read back after its launch
    h2d_bytes, d2h_bytes = e2e_copy_bytes(items)
    up = torch.cuda.Stream(device=device)
    down = torch.cuda.Stream(device=device)

    def one_step(last_use, last_read):
        arrived = {}
        for it in items:
            ready = []
            for t in it.h2d:
                k = key_of(t)
                if k not in arrived:
                    if k in last_use:
                        up.wait_event(last_use[k])
                    with torch.cuda.stream(up):
                        t.copy_(hmap[k], non_blocking=True)
                    e = torch.cuda.Event()
                    e.record(up)
                    arrived[k] = e
                ready.append(arrived[k])
            for e in ready:
                stream.wait_event(e)
            for t in it.d2h:
                k = key_of(t)
                if k in last_read:
                    stream.wait_event(last_read[k])
            st = it.fn(*it.args)
            if st != 0:
                lib_check(it.name, st)
            ke = torch.cuda.Event()
            ke.record(stream)
            for t in tuple(it.h2d) + tuple(it.d2h):
                last_use[key_of(t)] = ke
            for t in it.d2h:
                k = key_of(t)
                down.wait_event(ke)
                with torch.cuda.stream(down):
                    hmap[k].copy_(t, non_blocking=True)
                de = torch.cuda.Event()
                de.record(down)
                last_read[k] = de
                last_use[k] = de

    one_step({}, {})                      # warm-up (allocator, copy engines)
    torch.cuda.synchronize()
    # three timed rounds of `steps` steps; the median round is reported (the
    # host link's rate varies by some 20 % from run to run on this machine)
    rounds = []
    for _ in range(3):
        start = torch.cuda.Event(enable_timing=True)
        stop = torch.cuda.Event(enable_timing=True)
        barrier(dist, device)
        start.record(stream)
        up.wait_event(start)
        down.wait_event(start)
        last_use, last_read = {}, {}
        for _ in range(steps):
            one_step(last_use, last_read)
        stream.wait_stream(up)
        stream.wait_stream(down)
        stop.record(stream)
        torch.cuda.synchronize()
        rounds.append(start.elapsed_time(stop) / steps)
    ms = statistics.median(rounds)
    ms = max_over_ranks(ms, dist, device)
    world = dist.get_world_size() if dist is not None else 1
    nbytes = sum(it.nbytes for it in items)
    hmap.clear()
    return {"value": world * nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
            "ms_per_step": ms, "steps": steps, "rounds_ms_per_step": [round(r, 3) for r in rounds],
            "pipeline": "3 streams: host->device copies (each distinct input once per step), "
                        "kernels, device->host copies (every result)"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the BF16/FP16-storage and compensated-dot report")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched (4096 uneven instances per family) report")
    ap.add_argument("--no-autograd", action="store_true",
                    help="skip the forward/backward (differentiation) report")
    ap.add_argument("--no-fused", action="store_true",
                    help="skip the fused-vs-separate report")
    ap.add_argument("--no-formats", action="store_true",
                    help="skip the CSR-vs-SELL report")
    ap.add_argument("--no-small", action="store_true",
                    help="skip the small-configuration (latency, CUDA graph) report")
    ap.add_argument("--no-curves", action="store_true",
                    help="skip the cold/warm GB/s-against-size report")
    ap.add_argument("--record-traffic", default=None, metavar="NCU_CSV",
                    help="write DRAM bytes per launch from an ncu CSV (launches of the --only "
                         "selection, in sweep order) into --traffic-json, then exit")
    ap.add_argument("--profile-set", action="store_true",
                    help="launch every kernel family once at a small footprint (for ncu)")
    ap.add_argument("--only", default=None,
                    help="regex: run (and allocate) only the launches whose name matches "
                         "(profiling captures); the result is then not the full workload")
    ap.add_argument("--sweep-json", default=None, help="write the per-size table here")
    ap.add_argument("--detail-json", default=os.path.join(os.getcwd(), "bench_detail.json"),
                    help="write the full report (every per-kernel entry, the precision, "
                         "batched, autograd, fused, format, small-configuration and size-curve "
                         "sections) here; the printed line names this file ('' = none)")
    ap.add_argument("--traffic-json", default=os.path.join(ROOT, "profiles", "dram_traffic.json"),
                    help="per-kernel DRAM bytes per launch recorded from an ncu capture")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.record_traffic:
        return record_traffic(args.record_traffic, args.traffic_json, args.only)
    if args.profile_set:
        import torch
        torch.cuda.set_device(0)
        return run_profile_set(torch.device("cuda", 0))
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
