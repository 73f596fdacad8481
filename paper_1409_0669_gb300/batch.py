"""Batched operations: many independent instances of uneven sizes in one
persistent launch (lak_batch_plan / lak_batch_run of include/lak.h).

A Batch is planned once on the host (the C library writes the work table),
the table is copied to the device once, and `run()` launches the persistent
kernel; `run()` reads nothing from the host, so it can be captured in a CUDA
graph and replayed.  The tensors given to a Batch must stay alive and in place
while it is used.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

from . import _native
from ._native import DTYPES, OPS, AxpyDesc, BatchInfo, CsrDesc, DotDesc, GemvDesc


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None or t.numel() == 0:
        return None
    if not t.is_cuda:
        raise ValueError("batched operands must be CUDA tensors")
    from . import _dev_ptr
    return _dev_ptr(t, "batched operand")


TUNED_DEFAULTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_defaults.json")
_installed = set()


def install_tuned_defaults(path: str = TUNED_DEFAULTS) -> int:
    """Install the batched launch defaults the autotuner measured for this GPU
    model (its "batch:<op>:<storage>" entries; other GPUs keep the built-in
    shapes), except where the caller has set a default itself
    (set_batch_default_cfg).  Runs once per device per process, on the first
    batch planned there; returns the number of entries installed.  The
    defaults are process-wide."""
    dev = torch.cuda.current_device()
    if dev in _installed:
        return 0
    _installed.add(dev)
    if not os.path.exists(path):
        return 0
    import json

    from . import _apply_batch_default, _user_batch_defaults
    from .autotune import cache_key
    with open(path) as fh:
        entries = json.load(fh).get(cache_key(), {})
    done = 0
    for key, cfg in entries.items():
        parts = key.split(":")
        if parts[0] != "batch" or (parts[1], parts[2]) in _user_batch_defaults:
            continue
        _apply_batch_default(parts[1], parts[2], tuple(cfg))
        done += 1
    return done


def _cfg(cfg):
    if cfg is None:
        return None
    from . import _cfg_ptr
    return _cfg_ptr(cfg)


class Batch:
    def __init__(self, op: str, storage: str, descs, cfg=None, device=None, keep=()):
        lib = _native.load()
        install_tuned_defaults()
        self.op, self.storage = op, storage
        count = len(descs)
        arr_t = type(descs[0]) * count if count else AxpyDesc * 0
        arr = arr_t(*descs) if count else arr_t()
        info = BatchInfo()
        cptr = _cfg(cfg)
        _native.check("lak_batch_plan", lib.lak_batch_plan(OPS[op], DTYPES[storage], arr, count,
                                                           cptr, None, 0, ctypes.byref(info)))
        host = torch.empty(max(info.table_bytes, 16), dtype=torch.uint8)
        _native.check("lak_batch_plan",
                      lib.lak_batch_plan(OPS[op], DTYPES[storage], arr, count, cptr,
                                         host.data_ptr(), host.numel(), ctypes.byref(info)))
        dev = device or torch.device("cuda", torch.cuda.current_device())
        self.table = host.to(dev)
        self.workspace = torch.zeros(max(info.workspace_bytes, 256), dtype=torch.uint8, device=dev)
        self.info = info
        self.keep = tuple(keep)
        self._lib = lib

    @property
    def total_units(self) -> int:
        return int(self.info.total_units)

    def run(self, stream=None):
        from . import _on_current_device
        _on_current_device(self.table, self.workspace)
        sh = (torch.cuda.current_stream().cuda_stream if stream is None else
              (stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)))
        st = self._lib.lak_batch_run(ctypes.byref(self.info), self.table.data_ptr(),
                                     self.workspace.data_ptr(), self.workspace.numel(), sh)
        _native.check("lak_batch_run", st)


def _storage(ts):
    from . import storage_of
    s = storage_of(ts[0])
    for t in ts:
        if t.dtype != ts[0].dtype:
            raise TypeError("all operands of a batch must share one dtype")
    return s


def axpy_batch(xs: Sequence[torch.Tensor], ys, zs, alphas, cfg=None) -> Batch:
    """x_i = y_i + alpha_i z_i for every instance i."""
    s = _storage(list(xs) + list(ys) + list(zs))
    descs = [AxpyDesc(_ptr(x), _ptr(y), _ptr(z), x.numel(), float(a))
             for x, y, z, a in zip(xs, ys, zs, alphas)]
    return Batch("axpy", s, descs, cfg, keep=(xs, ys, zs))


def dot_batch(xs, ys, outs, cfg=None) -> Batch:
    """outs[i] = <x_i, y_i> (outs: one-element float32 tensors, float64 for FP64)."""
    s = _storage(list(xs) + list(ys))
    descs = [DotDesc(o.data_ptr(), _ptr(x), _ptr(y), x.numel()) for x, y, o in zip(xs, ys, outs)]
    return Batch("dot", s, descs, cfg, keep=(xs, ys, outs))


def gemv_batch(As, xs, ys, cfg=None) -> Batch:
    """y_i = A_i x_i for row-major 2-D tensors A_i (unit stride along rows)."""
    s = _storage(list(As) + list(xs) + list(ys))
    descs = []
    for A, x, y in zip(As, xs, ys):
        m, n = A.shape
        if n > 1 and A.stride(1) != 1:
            raise ValueError("batched GEMV instances must be row-major")
        lda = A.stride(0) if m > 1 else max(n, 1)
        descs.append(GemvDesc(_ptr(y), _ptr(A), _ptr(x), m, n, lda))
    return Batch("gemv_row", s, descs, cfg, keep=(As, xs, ys))


def spmv_batch(csrs, xs, ys, cfg=None) -> Batch:
    """y_i = A_i x_i for CSR matrices given as (row_ptr, col_idx, vals, n_cols)."""
    s = _storage([c[2] for c in csrs] + list(xs) + list(ys))
    descs = [CsrDesc(_ptr(y), _ptr(rp), _ptr(ci), _ptr(v), _ptr(x), rp.numel() - 1, int(ncols),
                     v.numel()) for (rp, ci, v, ncols), x, y in zip(csrs, xs, ys)]
    return Batch("spmv", s, descs, cfg, keep=(csrs, xs, ys))
