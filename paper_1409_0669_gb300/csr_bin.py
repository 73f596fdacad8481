"""Row-binned CSR matrices (csr_bin_build / csr_bin_spmv of include/lak.h):
the CSR arrays as they are plus a device row permutation that groups rows by
length, so that every warp of the product serves rows of similar length.
Building needs no host synchronisation.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _cfg_ptr, _native, _on_current_device, _stream, storage_of
from ._native import DTYPES

BINS = 7            # LAK_CSR_BINS
PER_LANE = 4        # LAK_CSR_BIN_PER_LANE


class BinnedCsr:
    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
                 n_cols: int, stream=None):
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
            raise TypeError("row_ptr and col_idx must be int32")
        _on_current_device(row_ptr, col_idx, vals)
        lib = _native.load()
        self._lib = lib
        dev = row_ptr.device
        self.row_ptr, self.col_idx, self.vals = row_ptr, col_idx, vals
        self.m, self.n, self.nnz = row_ptr.numel() - 1, int(n_cols), vals.numel()
        sh = _stream(stream)
        self.perm = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)
        self.bin_ptr = torch.empty(BINS + 1, dtype=torch.int64, device=dev)
        ws = torch.empty(max(int(lib.csr_bin_workspace(self.m)), 256), dtype=torch.uint8,
                         device=dev)
        _native.check("csr_bin_build",
                      lib.csr_bin_build(self.perm.data_ptr(), self.bin_ptr.data_ptr(),
                                        row_ptr.data_ptr(), self.m, ws.data_ptr(), ws.numel(),
                                        sh))
        self._ws = ws                                   # kept until the build has run

    def spmv(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, cfg=None,
             stream=None) -> torch.Tensor:
        s = storage_of(self.vals)
        if x.dtype != self.vals.dtype:
            raise TypeError("x must have the matrix's dtype")
        if y is None:
            y = torch.empty(self.m, dtype=self.vals.dtype, device=self.vals.device)
        _on_current_device(x, y, self.row_ptr)
        _native.check("csr_bin_spmv",
                      self._lib.csr_bin_spmv(y.data_ptr() if self.m else None,
                                             self.row_ptr.data_ptr(),
                                             self.col_idx.data_ptr() if self.nnz else None,
                                             self.vals.data_ptr() if self.nnz else None,
                                             x.data_ptr() if x.numel() else None,
                                             self.perm.data_ptr(), self.bin_ptr.data_ptr(),
                                             self.m, self.n, self.nnz, DTYPES[s], _cfg_ptr(cfg),
                                             _stream(stream)))
        return y
