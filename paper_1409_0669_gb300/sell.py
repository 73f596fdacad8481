"""SELL-C-sigma (C = 32) matrices built from CSR on the GPU (csr_to_sell_count /
csr_to_sell_fill / sell_pack_values of include/lak.h) and their product.

The conversion needs the total padded size on the host to allocate the slot
arrays, so building a SellMatrix synchronises once; products do not.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _cfg_ptr, _native, _on_current_device, _stream, storage_of
from ._native import DTYPES


class SellMatrix:
    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor,
                 n_cols: int, sigma: int = 1, stream=None):
        _on_current_device(row_ptr, col_idx, vals)
        lib = _native.load()
        self._lib = lib
        dev = row_ptr.device
        m = row_ptr.numel() - 1
        self.m, self.n, self.sigma = m, int(n_cols), int(sigma)
        mp = (m + 31) // 32 * 32
        ns = mp // 32
        sh = _stream(stream)
        self.perm = torch.empty(max(mp, 1), dtype=torch.int32, device=dev)
        self.slice_len = torch.empty(max(ns, 1), dtype=torch.int32, device=dev)
        self.slice_ptr = torch.zeros(ns + 1, dtype=torch.int64, device=dev)
        _native.check("csr_to_sell_count",
                      lib.csr_to_sell_count(row_ptr.data_ptr(), m, self.sigma, self.perm.data_ptr(),
                                            self.slice_len.data_ptr(), self.slice_ptr.data_ptr(),
                                            sh))
        total = int(self.slice_ptr[ns].item())          # the one synchronisation
        self.total = total
        self.cols = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        self.map = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        if m > 0:
            _native.check("csr_to_sell_fill",
                          lib.csr_to_sell_fill(row_ptr.data_ptr(),
                                               col_idx.data_ptr() if col_idx.numel() else None,
                                               m, self.perm.data_ptr(), self.slice_len.data_ptr(),
                                               self.slice_ptr.data_ptr(), self.cols.data_ptr(),
                                               self.map.data_ptr(), sh))
        self.vals = torch.zeros(max(total, 1), dtype=vals.dtype, device=dev)
        self.pack(vals, stream)

    def pack(self, vals: torch.Tensor, stream=None):
        """(Re)load the CSR values into the SELL slots."""
        s = storage_of(vals)
        _on_current_device(vals, self.vals)
        _native.check("sell_pack_values",
                      self._lib.sell_pack_values(self.vals.data_ptr(),
                                                 vals.data_ptr() if vals.numel() else None,
                                                 self.map.data_ptr(), self.total, DTYPES[s],
                                                 _stream(stream)))

    def spmv(self, x: torch.Tensor, y: Optional[torch.Tensor] = None, cfg=None,
             stream=None) -> torch.Tensor:
        s = storage_of(self.vals)
        if x.dtype != self.vals.dtype:
            raise TypeError("x must have the matrix's dtype")
        if y is None:
            y = torch.empty(self.m, dtype=self.vals.dtype, device=self.vals.device)
        _on_current_device(x, y, self.vals)
        _native.check("sell_spmv",
                      self._lib.sell_spmv(y.data_ptr() if self.m else None,
                                          self.slice_ptr.data_ptr(), self.slice_len.data_ptr(),
                                          self.perm.data_ptr(), self.cols.data_ptr(),
                                          self.vals.data_ptr(), x.data_ptr() if x.numel() else None,
                                          self.m, DTYPES[s], _cfg_ptr(cfg), _stream(stream)))
        return y
