"""Autotuner for the shared launch configuration (block, grid, vec, increment).

The paper's tuning space (Sec. 2) is increment type x vector length x local
size x number of work-groups (2 x 5 x 10 x 19 = 1900 configurations).  On
GB300 the same four axes become:
  increment  global (grid-stride) / local (contiguous range per block)
  vec        1, 2, 4, 8, 16 elements per thread per access group
  block      64, 128, 256, 512 threads
  grid       automatic (enough blocks to cover the data once) or a multiple of
             the SM count (1, 2, 4, 8, 16, 32 blocks per SM: persistent grids)
Each configuration is timed with CUDA events on the launching stream
(timing.launch_time_us: operands larger than L2 launch by launch; operands
that fit in L2 as `reps` (256 MB flush read, launch) pairs in one event
interval minus the flushes alone -- GB300's event clock ticks in steps of
about 2 us, too coarse for one launch of a few microseconds).

Defaults are kept per size bucket (lak_size_bucket: the call's algorithmic
bytes, below 8 MiB / 64 MiB / 512 MiB / above).  `tune_buckets` times every
configuration at several sizes, groups the sizes by bucket and keeps, per
bucket, the configuration whose worst ratio to each size's own optimum is
best.

`copy_first_study` repeats the paper's central experiment (Sec. 3.2, 3.4):
tune the copy kernel exhaustively, keep the configurations within 15 % of the
best copy, and measure how close the best of those comes to each other
operation's own optimum.

The batched persistent launches (lak_batch_plan / lak_batch_run) have their
own space -- block 32..512 (batched GEMV: up to 128), grid automatic or 1..16
blocks per SM, 2..16 elements per access (CSR: 4 or 8 entries per lane), both
increments (the CSR batch schedules dynamically, so only one) -- searched by
`tune_batch` on the batching workload itself (4096 uneven instances of one
family, synth.batch_workload), one run of the whole batch per timing.

The winners can be saved as a JSON cache keyed by GPU name and SM count and
installed as the library's per-op defaults (lak_set_default_cfg;
"batch:<op>:<storage>" entries: lak_set_batch_default_cfg).  The cache this
package ships (tuned_defaults.json) holds the batched defaults measured on
GB300; the batched runner installs it for a matching GPU on first use.

  python -m paper_1409_0669_gb300.autotune --op copy --storage f32 --size 100000000
  python -m paper_1409_0669_gb300.autotune --study [--paper-sizes] --storage f32 \
      --out profiles/copy_first_study_f32_large.json
  python -m paper_1409_0669_gb300.autotune --study-table profiles/copy_first_study_*.json
  python -m paper_1409_0669_gb300.autotune --buckets --op dot --storage f64 \
      --size 46416,215443,2154435,10000000 --out tune.json
  python -m paper_1409_0669_gb300.autotune --batch --op gemv_row --storage f32 \
      --out tune.json --save-cache paper_1409_0669_gb300/tuned_defaults.json
"""
from __future__ import annotations

import argparse
import json
import statistics
from typing import Callable, Dict, List, Optional

import torch

from . import _native
from ._native import DTYPES, LakCfg, LakError
from ._native import OPS as _OP_CODES
from .timing import launch_time_us, warm_time_us

OPS = ("copy", "axpy", "dot", "gemv_row", "gemv_col", "spmv")
BLOCKS = (32, 64, 128, 256, 512)
VECS = (1, 2, 4, 8, 16)
GRID_PER_SM = (0, 1, 2, 4, 8, 16, 32)       # 0 = automatic
_L2_FLUSH_BYTES = 256 << 20


def space(sms: int) -> List[LakCfg]:
    out = []
    for inc in (0, 1):
        for vec in VECS:
            for block in BLOCKS:
                for k in GRID_PER_SM:
                    out.append(LakCfg(block, k * sms, vec, inc))
    return out


class Problem:
    """Inputs of one op at one size on the current device, and a launcher
    that takes a configuration (pre-marshalled C-ABI call)."""

    def __init__(self, op: str, storage: str, size, device=None, seed: int = 0):
        import synth
        self.op, self.storage = op, storage
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        sh = self.stream.cuda_stream
        lib = _native.load()
        dt = synth.torch_dtype(storage)
        es = torch.tensor([], dtype=dt).element_size()
        code = DTYPES[storage]
        self.keep = []
        if op in ("copy", "axpy", "dot"):
            n = int(size)
            y = synth.device_uniform_(torch.empty(n, dtype=dt, device=self.device), seed + 1)
            z = synth.device_uniform_(torch.empty(n, dtype=dt, device=self.device), seed + 2)
            x = torch.zeros(n, dtype=dt, device=self.device)
            out = torch.zeros(1, dtype=torch.float64 if storage == "f64" else torch.float32,
                              device=self.device)
            self.keep += [y, z, x, out]
            if op == "copy":
                self.nbytes = 2 * n * es
                self.fn = lambda c: lib.vec_copy(x.data_ptr(), y.data_ptr(), n, code, c, sh)
            elif op == "axpy":
                self.nbytes = 3 * n * es
                self.fn = lambda c: lib.vec_axpy(x.data_ptr(), y.data_ptr(), z.data_ptr(), 0.5,
                                                 n, code, c, sh)
            else:
                self.nbytes = 2 * n * es
                ws = torch.zeros(1 << 20, dtype=torch.uint8, device=self.device)
                self.keep.append(ws)
                self.fn = lambda c: lib.vec_dot(out.data_ptr(), y.data_ptr(), z.data_ptr(), n,
                                                code, ws.data_ptr(), ws.numel(), c, sh)
            self.footprint = self.nbytes
            self.dims = (n, n, 0)
        elif op in ("gemv_row", "gemv_col"):
            m = n = int(size)
            A = synth.device_normal_(torch.empty(m * n, dtype=dt, device=self.device), seed + 3)
            xg = synth.device_uniform_(torch.empty(n, dtype=dt, device=self.device), seed + 4)
            yg = torch.zeros(m, dtype=dt, device=self.device)
            ws = torch.zeros(512 << 20, dtype=torch.uint8, device=self.device)
            self.keep += [A, xg, yg, ws]
            lay = 0 if op == "gemv_row" else 1
            self.nbytes = (m * n + m + n) * es
            self.fn = lambda c: lib.dense_gemv(yg.data_ptr(), A.data_ptr(), xg.data_ptr(), m, n,
                                               n if lay == 0 else m, lay, code, ws.data_ptr(),
                                               ws.numel(), c, sh)
            self.footprint = self.nbytes
            self.dims = (m, n, 0)
        elif op == "spmv":
            if size == "lap3d_128":
                rp, ci, v = synth.laplacian_3d(128, storage)
                ncols = 128 ** 3
            elif size == "lap3d_64":
                rp, ci, v = synth.laplacian_3d(64, storage)
                ncols = 64 ** 3
            elif size == "lap2d_256":
                rp, ci, v = synth.laplacian_2d(256, storage)
                ncols = 256 ** 2
            elif size == "powerlaw_2m":
                rp, ci, v = synth.powerlaw_csr(2_000_000, 2_000_000, 1, storage)
                ncols = 2_000_000
            else:
                raise ValueError(f"unknown sparse matrix {size!r}")
            rpd, cid, vd = rp.to(self.device), ci.to(self.device), v.to(self.device)
            xs = synth.device_uniform_(torch.empty(ncols, dtype=dt, device=self.device), seed + 5)
            m = rp.numel() - 1
            nnz = v.numel()
            ys = torch.zeros(m, dtype=dt, device=self.device)
            self.keep += [rpd, cid, vd, xs, ys]
            self.nbytes = nnz * (es + 4) + (m + 1) * 4 + ncols * es + m * es
            self.fn = lambda c: lib.csr_spmv(ys.data_ptr(), rpd.data_ptr(), cid.data_ptr(),
                                             vd.data_ptr(), xs.data_ptr(), m, ncols, nnz, code,
                                             c, sh)
            self.footprint = self.nbytes
            self.dims = (m, ncols, nnz)
        else:
            raise ValueError(op)
        l2 = torch.cuda.get_device_properties(self.device).L2_cache_size
        self.flush = torch.empty(_L2_FLUSH_BYTES // 4, dtype=torch.float32, device=self.device) \
            if self.footprint < 2 * l2 else None

    def time_cfg(self, cfg: Optional[LakCfg], reps: int = 10, warm: int = 2) -> float:
        """Device time of one launch in microseconds, L2 cold (raises LakError
        on a bad cfg)."""
        import ctypes
        cptr = ctypes.byref(cfg) if cfg is not None else None
        for _ in range(warm):
            st = self.fn(cptr)
            _native.check(self.op, st)
        torch.cuda.synchronize(self.device)

        def call():
            st = self.fn(cptr)
            if st != 0:
                _native.check(self.op, st)

        return launch_time_us(call, reps, self.flush, self.stream)

    def time_warm(self, cfg: Optional[LakCfg], reps: int = 10) -> float:
        """Device time of one launch with the operands left in L2 by the
        previous one (back-to-back launches), in microseconds."""
        import ctypes
        cptr = ctypes.byref(cfg) if cfg is not None else None

        def call():
            st = self.fn(cptr)
            if st != 0:
                _native.check(self.op, st)

        return warm_time_us(call, reps, self.stream)


REFINE_TOP = 8          # candidates re-timed after the sweep
REFINE_ROUNDS = 3       # extra timings of each, round-robin


def refine_top(results: List[Dict], time_cfg, nbytes: int, top: int = REFINE_TOP,
               rounds: int = REFINE_ROUNDS) -> List[Dict]:
    """Re-time the `top` fastest entries of a sorted sweep `rounds` more times,
    round-robin (a slow drift of the clock or the memory system then hits every
    candidate alike), and re-rank them by the median of all their timings.  With
    one timing per configuration over hundreds of configurations, the fastest
    looking ones are partly the luckiest draws (the minimum of many noisy
    timings); the median of four is not.  Each refined entry keeps its first
    timing as `us_sweep`."""
    head = results[:max(int(top), 0)]
    if not head or rounds < 1:
        return results
    samples = [[r["us"]] for r in head]
    for _ in range(int(rounds)):
        for r, ts in zip(head, samples):
            try:
                ts.append(time_cfg(LakCfg(*r["cfg"])))
            except LakError:
                pass
    for r, ts in zip(head, samples):
        r["us_sweep"] = r["us"]
        r["us"] = statistics.median(ts)
        r["GBs"] = nbytes / (max(r["us"], 1e-3) * 1e-6) / 1e9
    head.sort(key=lambda r: r["us"])
    return head + results[len(head):]


def tune(op: str, storage: str, size, reps: int = 10, cfgs: Optional[List[LakCfg]] = None,
         problem: Optional[Problem] = None, refine: int = REFINE_TOP) -> List[Dict]:
    """Time every configuration; results sorted fastest first, the `refine`
    fastest re-timed and re-ranked (refine_top)."""
    if cfgs is None or problem is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    prob = problem or Problem(op, storage, size, dev)
    if cfgs is None:
        cfgs = space(torch.cuda.get_device_properties(dev).multi_processor_count)
    results = []
    for c in cfgs:
        try:
            us = prob.time_cfg(c, reps)
        except LakError:
            continue
        results.append({"cfg": list(c.as_tuple()), "us": us,
                        "GBs": prob.nbytes / (max(us, 1e-3) * 1e-6) / 1e9})
    results.sort(key=lambda r: r["us"])
    return refine_top(results, lambda c: prob.time_cfg(c, reps), prob.nbytes, refine)


def copy_first_study(storage: str, sizes: Dict[str, object], keep_frac: float = 0.85,
                     reps: int = 10, cfgs: Optional[List[LakCfg]] = None) -> Dict:
    """Sec. 3.2 / 3.4 on GB300: configurations within (1 - keep_frac) of the
    best copy, evaluated on the other ops, against each op's own best over the
    same space (the whole space unless `cfgs` restricts it)."""
    copy = tune("copy", storage, sizes["copy"], reps, cfgs)
    best = copy[0]["GBs"]
    cands = [r for r in copy if r["GBs"] >= keep_frac * best]
    report = {"storage": storage, "sizes": dict(sizes), "keep_frac": keep_frac,
              "copy_best_GBs": best, "candidates": len(cands), "space": len(copy),
              "candidate_cfgs": [r["cfg"] for r in cands], "ops": {}}
    cand_cfgs = [LakCfg(*r["cfg"]) for r in cands]
    per_op = {}
    for op in ("axpy", "dot", "gemv_row", "gemv_col", "spmv"):
        prob = Problem(op, storage, sizes[op])
        own = tune(op, storage, sizes[op], reps, cfgs, prob)
        from_copy = tune(op, storage, sizes[op], reps, cand_cfgs, prob)
        per_op[op] = {tuple(r["cfg"]): r for r in from_copy}
        report["ops"][op] = {
            "own_best": own[0], "best_from_copy": from_copy[0] if from_copy else None,
            "ratio": (from_copy[0]["GBs"] / own[0]["GBs"]) if from_copy and own else None,
            "default": _default_point(prob, reps)}
        del prob
        torch.cuda.empty_cache()
    # one shared configuration: the copy candidate with the best worst-case ratio
    shared, shared_score = None, -1.0
    for c in cands:
        key = tuple(c["cfg"])
        ratios = []
        for op, table in per_op.items():
            r = table.get(key)
            if r is None:
                break
            ratios.append(r["GBs"] / report["ops"][op]["own_best"]["GBs"])
        else:
            if min(ratios) > shared_score:
                shared, shared_score = key, min(ratios)
    report["shared_cfg"] = list(shared) if shared else None
    report["shared_worst_ratio"] = shared_score if shared else None
    report["copy_top"] = copy[:10]
    return report


STUDY_SIZES = {
    # the paper's own problem sizes (vectors of 2e6 entries, a 2048^2 matrix);
    # the CSR product, which the paper leaves out, on the 64^3 Laplacian
    "paper": {"copy": 2_000_000, "axpy": 2_000_000, "dot": 2_000_000,
              "gemv_row": 2048, "gemv_col": 2048, "spmv": "lap3d_64"},
    "large": {"copy": 100_000_000, "axpy": 100_000_000, "dot": 100_000_000,
              "gemv_row": 16384, "gemv_col": 16384, "spmv": "lap3d_128"},
}

_STUDY_OP_NAMES = {"axpy": "axpy", "dot": "dot", "gemv_row": "GEMV row", "gemv_col": "GEMV col",
                   "spmv": "SpMV"}


def study_table(reports: List[Dict]) -> str:
    """Markdown table of copy-first study reports (one row per report and op):
    each op's own best, the best copy-derived configuration, their ratio; then
    one line per report with the shared configuration's worst-case ratio."""
    lines = ["| storage, sizes | op | own best GB/s | best copy-derived GB/s | ratio |",
             "|---|---|---|---|---|"]
    notes = []
    for rep in reports:
        tag = f"{rep['storage'].upper()}, {rep.get('label', '?')}"
        for op, name in _STUDY_OP_NAMES.items():
            r = rep["ops"][op]
            lines.append(f"| {tag} | {name} | {r['own_best']['GBs']:.0f} | "
                         f"{r['best_from_copy']['GBs']:.0f} | {r['ratio']:.3f} |")
        sc = rep["shared_cfg"]
        notes.append(f"- {tag}: {rep['candidates']} of {rep['space']} configurations kept; "
                     f"shared ({sc[0]}, {sc[1]}, {sc[2]}, {'local' if sc[3] else 'global'}) "
                     f"reaches {100 * rep['shared_worst_ratio']:.1f} % of every op's own best")
    return "\n".join(lines + [""] + notes) + "\n"


# ---- batched launches -------------------------------------------------------------

BATCH_OPS = ("axpy", "dot", "gemv_row", "spmv")
BATCH_GRID_PER_SM = (0, 1, 2, 4, 8, 16)          # 0 = SMs x (2048 / block threads)


def batch_space(op: str, sms: int) -> List[LakCfg]:
    """Launch configurations of one batched family."""
    blocks = (32, 64, 128) if op == "gemv_row" else (32, 64, 128, 256, 512)
    vecs = (4, 8) if op == "spmv" else (2, 4, 8, 16)
    incs = (0,) if op == "spmv" else (0, 1)
    return [LakCfg(b, k * sms, v, inc) for inc in incs for v in vecs for b in blocks
            for k in BATCH_GRID_PER_SM]


class BatchProblem:
    """One family of the batching workload (4096 uneven instances) on the
    current device; time_cfg plans the batch with a configuration and times
    one persistent launch over all instances."""

    def __init__(self, op: str, storage: str, count: int = 4096, seed: int = 4000, device=None):
        import synth
        if op not in BATCH_OPS:
            raise ValueError(op)
        self.op, self.storage, self.count = op, storage, count
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.stream = torch.cuda.current_stream(self.device)
        fam = {"axpy": "vec", "dot": "vec", "gemv_row": "gemv", "spmv": "csr"}[op]
        wl = synth.batch_workload(self.device, count, seed, synth.torch_dtype(storage),
                                  families=(fam,))
        es = torch.tensor([], dtype=synth.torch_dtype(storage)).element_size()
        self.keep = wl
        if op in ("axpy", "dot"):
            n = sum(v[0].numel() for v in wl["vec"])
            self.nbytes = (3 if op == "axpy" else 2) * n * es
            self.outs = torch.zeros(count, dtype=torch.float64 if storage == "f64"
                                    else torch.float32, device=self.device)
        elif op == "gemv_row":
            self.nbytes = sum((A.numel() + A.shape[0] + A.shape[1]) * es
                              for A, _, _ in wl["gemv"])
        else:
            self.nbytes = sum(v.numel() * (es + 4) + (m + 1) * 4 + 2 * m * es
                              for (_, _, v, m), _, _ in wl["csr"])

    def batch(self, cfg: Optional[LakCfg]):
        from . import batch as B
        wl = self.keep
        c = None if cfg is None else tuple(cfg.as_tuple())
        if self.op == "axpy":
            return B.axpy_batch([v[2] for v in wl["vec"]], [v[0] for v in wl["vec"]],
                                [v[1] for v in wl["vec"]], [0.5] * self.count, cfg=c)
        if self.op == "dot":
            return B.dot_batch([v[0] for v in wl["vec"]], [v[1] for v in wl["vec"]],
                               [self.outs[i:i + 1] for i in range(self.count)], cfg=c)
        if self.op == "gemv_row":
            return B.gemv_batch([g[0] for g in wl["gemv"]], [g[1] for g in wl["gemv"]],
                                [g[2] for g in wl["gemv"]], cfg=c)
        return B.spmv_batch([g[0] for g in wl["csr"]], [g[1] for g in wl["csr"]],
                            [g[2] for g in wl["csr"]], cfg=c)

    def time_cfg(self, cfg: Optional[LakCfg], reps: int = 5) -> float:
        """Device time of one run of the whole batch in microseconds (median
        of `reps` launches, each bracketed by events on the stream).  The
        batch reads ~1-70 GB, far more than L2 holds."""
        b = self.batch(cfg)
        b.run(self.stream)
        torch.cuda.synchronize(self.device)
        times = []
        for _ in range(reps):
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(self.stream)
            b.run(self.stream)
            e.record(self.stream)
            e.synchronize()
            times.append(s.elapsed_time(e) * 1e3)
        times.sort()
        return times[len(times) // 2]


def tune_batch(op: str, storage: str, count: int = 4096, reps: int = 5,
               cfgs: Optional[List[LakCfg]] = None,
               problem: Optional[BatchProblem] = None, refine: int = REFINE_TOP) -> List[Dict]:
    """Time every batched configuration of one family; fastest first (each
    entry: cfg, us, GB/s), the `refine` fastest re-timed and re-ranked."""
    if cfgs is None or problem is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    prob = problem or BatchProblem(op, storage, count, device=dev)
    if cfgs is None:
        cfgs = batch_space(op, torch.cuda.get_device_properties(dev).multi_processor_count)
    results = []
    for c in cfgs:
        try:
            us = prob.time_cfg(c, reps)
        except LakError:
            continue
        results.append({"cfg": list(c.as_tuple()), "us": us,
                        "GBs": prob.nbytes / (max(us, 1e-3) * 1e-6) / 1e9})
    results.sort(key=lambda r: r["us"])
    return refine_top(results, lambda c: prob.time_cfg(c, reps), prob.nbytes, refine)


def problem_bucket(prob: Problem) -> int:
    """Size bucket of a Problem's call (lak_size_bucket)."""
    lib = _native.load()
    return lib.lak_size_bucket(_OP_CODES[prob.op], DTYPES[prob.storage], *prob.dims)


def choose_per_bucket(results: Dict[object, List[Dict]], buckets: Dict[object, int]) -> Dict[int, Dict]:
    """results: size -> tune() output; buckets: size -> bucket.  Per bucket,
    the configuration (timed at every size of the bucket) whose worst ratio
    of the size's best time to its own time is largest."""
    out = {}
    for b in sorted(set(buckets.values())):
        sizes = [sz for sz, bb in buckets.items() if bb == b]
        tables = {sz: {tuple(r["cfg"]): r["us"] for r in results[sz]} for sz in sizes}
        common = set.intersection(*(set(t) for t in tables.values()))
        best_cfg, best_score = None, -1.0
        for c in sorted(common):
            score = min(min(tables[sz].values()) / tables[sz][c] for sz in sizes)
            if score > best_score:
                best_cfg, best_score = c, score
        if best_cfg is not None:
            out[b] = {"cfg": list(best_cfg), "worst_ratio": best_score, "sizes": sizes}
    return out


def tune_buckets(op: str, storage: str, sizes, reps: int = 15) -> Dict[int, Dict]:
    """Tune `op` at every size and keep one configuration per size bucket."""
    results, buckets = {}, {}
    for sz in sizes:
        prob = Problem(op, storage, sz)
        results[sz] = tune(op, storage, sz, reps, problem=prob)
        buckets[sz] = problem_bucket(prob)
        del prob
        torch.cuda.empty_cache()
    return choose_per_bucket(results, buckets)


def _default_point(prob: Problem, reps: int) -> Dict:
    us = prob.time_cfg(None, reps)
    return {"us": us, "GBs": prob.nbytes / (max(us, 1e-3) * 1e-6) / 1e9}


def cache_key() -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sms={p.multi_processor_count}"


def save_cache(path: str, entries: Dict[str, List[int]]):
    """entries: {"<op>:<storage>": [block, grid, vec, increment]} for every
    size bucket, or {"<op>:<storage>:<bucket>": [...]} for one."""
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    data.setdefault(cache_key(), {}).update(entries)
    with open(path, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)


def apply_cache(path: str, only_batch: bool = False) -> int:
    """Install the cached configurations for this GPU as library defaults
    ("batch:<op>:<storage>" entries as batched defaults); returns how many."""
    from . import set_batch_default_cfg, set_default_cfg
    with open(path) as fh:
        data = json.load(fh)
    entries = data.get(cache_key(), {})
    done = 0
    for key, cfg in entries.items():
        parts = key.split(":")
        if parts[0] == "batch":
            set_batch_default_cfg(parts[1], parts[2], tuple(cfg))
        elif only_batch:
            continue
        else:
            bucket = int(parts[2]) if len(parts) == 3 else None
            set_default_cfg(parts[0], parts[1], tuple(cfg), bucket)
        done += 1
    return done


def _main(argv=None):
    ap = argparse.ArgumentParser(description="launch-configuration autotuner")
    ap.add_argument("--op", choices=OPS)
    ap.add_argument("--storage", default="f32", choices=list(DTYPES))
    ap.add_argument("--size", default="100000000")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--top", type=int, default=15)
    ap.add_argument("--study", action="store_true", help="copy-first transfer study")
    ap.add_argument("--paper-sizes", action="store_true",
                    help="run the study at the paper's sizes (2e6-entry vectors, 2048^2)")
    ap.add_argument("--study-table", nargs="+", default=None, metavar="REPORT_JSON",
                    help="print the markdown table of saved --study reports (no GPU needed)")
    ap.add_argument("--buckets", action="store_true",
                    help="one configuration per size bucket from the comma-separated --size list")
    ap.add_argument("--batch", action="store_true",
                    help="tune the batched launch of --op on the batching workload")
    ap.add_argument("--count", type=int, default=4096, help="instances of a --batch family")
    ap.add_argument("--save-cache", default=None,
                    help="merge the winner(s) into this JSON cache under this GPU's key")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    size = args.size
    if size.isdigit():
        size = int(size)
    cache_entries = {}
    if args.batch:
        res = tune_batch(args.op, args.storage, args.count, reps=min(args.reps, 5))
        # the built-in shape: time a plan without a cfg with any installed entry
        # removed (the batched runner installs the shipped cache on first use)
        from . import _apply_batch_default
        from . import batch as _B
        prob_default = BatchProblem(args.op, args.storage, args.count)
        _B.install_tuned_defaults()
        _apply_batch_default(args.op, args.storage, None)
        default_us = prob_default.time_cfg(None)
        del prob_default
        _B._installed.discard(torch.cuda.current_device())
        _B.install_tuned_defaults()
        cache_entries[f"batch:{args.op}:{args.storage}"] = res[0]["cfg"]
        text = json.dumps({"op": args.op, "storage": args.storage, "count": args.count,
                           "top": res[:args.top], "worst": res[-3:], "count_cfgs": len(res),
                           "builtin_default_us": default_us}, indent=1)
    elif args.buckets:
        sizes = [int(v) if v.isdigit() else v for v in args.size.split(",")]
        per = tune_buckets(args.op, args.storage, sizes, args.reps)
        text = json.dumps({"op": args.op, "storage": args.storage,
                           "buckets": {str(b): v for b, v in per.items()},
                           "cache": {f"{args.op}:{args.storage}:{b}": v["cfg"]
                                     for b, v in per.items()}}, indent=1)
    elif args.study:
        label = "paper" if args.paper_sizes else "large"
        rep = copy_first_study(args.storage, STUDY_SIZES[label], reps=args.reps)
        rep["label"] = label
        text = json.dumps(rep, indent=1)
    elif args.study_table:
        reps_ = []
        for path in args.study_table:
            with open(path) as fh:
                reps_.append(json.load(fh))
        text = study_table(reps_)
    else:
        res = tune(args.op, args.storage, size, args.reps)
        text = json.dumps({"op": args.op, "storage": args.storage, "size": size,
                           "top": res[:args.top], "worst": res[-3:], "count": len(res)}, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text)
    if args.save_cache and cache_entries:
        save_cache(args.save_cache, cache_entries)


if __name__ == "__main__":
    _main()
