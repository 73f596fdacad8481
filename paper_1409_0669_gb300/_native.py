"""ctypes binding of the C ABI declared in include/lak.h.

Loads the in-tree ``liblak_gb300.so``; importing fails loudly if it has not
been built (there is no fallback implementation of any operation).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblak_gb300.so")

# enums of lak.h
LAK_OK, LAK_EINVAL, LAK_EDTYPE, LAK_ELAYOUT, LAK_ECUDA, LAK_EWORKSPACE = 0, -1, -2, -3, -4, -5
DOT_NOALLOC_MAX_BLOCKS = 8192          # LAK_DOT_NOALLOC_MAX_BLOCKS
STATUS_NAMES = {0: "LAK_OK", -1: "LAK_EINVAL", -2: "LAK_EDTYPE", -3: "LAK_ELAYOUT",
                -4: "LAK_ECUDA", -5: "LAK_EWORKSPACE"}
DTYPES = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}
LAYOUTS = {"row": 0, "col": 1}
INCREMENTS = {"global": 0, "local": 1}
OPS = {"copy": 0, "axpy": 1, "dot": 2, "gemv_row": 3, "gemv_col": 4, "spmv": 5}

# exported symbols, in header order (checked by the ABI test)
EXPORTS = ("lak_last_error", "lak_abi_version", "lak_set_default_cfg", "lak_resolve_cfg",
           "lak_size_bucket", "lak_set_default_cfg_bucket", "vec_dot_sparse_workspace",
           "vec_dot_sparse", "csr_bin_workspace", "csr_bin_build", "csr_bin_spmv",
           "vec_copy", "vec_axpy", "vec_axpby", "vec_axpby_strided", "vec_axpy_norm2_workspace",
           "vec_axpy_norm2", "vec_dot_workspace", "vec_dot", "vec_dot_compensated",
           "vec_dot_noalloc",
           "dense_gemv_workspace", "dense_gemv", "dense_gemv_axpby", "dense_gemv_trans",
           "csr_spmv", "dense_outer", "csr_sampled_outer",
           "csr_transpose_workspace", "csr_transpose", "vec_gather", "vec_scale_dev",
           "csr_to_sell_count", "csr_to_sell_fill", "sell_pack_values", "sell_spmv",
           "lak_batch_plan", "lak_batch_run", "lak_set_batch_default_cfg", "lak_probe_fma_f64",
           "lak_probe_fma_f64_flops")


class LakCfg(ctypes.Structure):
    """lak_cfg: (block, grid, vec, increment); zero fields mean automatic."""
    _fields_ = [("block", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("vec", ctypes.c_int32), ("increment", ctypes.c_int32)]

    def as_tuple(self):
        return (self.block, self.grid, self.vec, self.increment)

    def __repr__(self):
        return "LakCfg(block=%d, grid=%d, vec=%d, increment=%d)" % self.as_tuple()


class AxpyDesc(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("alpha", ctypes.c_double)]


class DotDesc(ctypes.Structure):
    _fields_ = [("out", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class GemvDesc(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("A", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("lda", ctypes.c_int64)]


class CsrDesc(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int64), ("total_units", ctypes.c_int64),
                ("unit_elems", ctypes.c_int64), ("table_bytes", ctypes.c_size_t),
                ("workspace_bytes", ctypes.c_size_t), ("cfg", LakCfg),
                ("op", ctypes.c_int32), ("dtype", ctypes.c_int32)]


class LakError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        self.status = status
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {message}")


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t
_CFGP = ctypes.POINTER(LakCfg)

_SIGNATURES = {
    "lak_last_error": (ctypes.c_char_p, []),
    "lak_abi_version": (_I32, []),
    "lak_set_default_cfg": (_I32, [_I32, _I32, _CFGP]),
    "lak_set_default_cfg_bucket": (_I32, [_I32, _I32, _I32, _CFGP]),
    "lak_size_bucket": (_I32, [_I32, _I32, _I64, _I64, _I64]),
    "lak_resolve_cfg": (_I32, [_I32, _I32, _I64, _I64, _I64, _CFGP, _CFGP]),
    "vec_copy": (_I32, [_P, _P, _I64, _I32, _CFGP, _P]),
    "vec_axpy": (_I32, [_P, _P, _P, ctypes.c_double, _I64, _I32, _CFGP, _P]),
    "vec_axpby": (_I32, [_P, ctypes.c_double, _P, ctypes.c_double, _P, _I64, _I32, _CFGP, _P]),
    "vec_axpby_strided": (_I32, [_P, _I64, ctypes.c_double, _P, _I64, ctypes.c_double, _P, _I64,
                                 _I64, _I32, _P]),
    "vec_axpy_norm2_workspace": (_SZ, [_I64, _I32, _CFGP]),
    "vec_axpy_norm2": (_I32, [_P, _P, _P, ctypes.c_double, _P, _I64, _I32, _P, _SZ, _CFGP, _P]),
    "vec_dot_workspace": (_SZ, [_I64, _I32, _CFGP]),
    "vec_dot": (_I32, [_P, _P, _P, _I64, _I32, _P, _SZ, _CFGP, _P]),
    "vec_dot_sparse_workspace": (_SZ, [_I64, _I32, _CFGP]),
    "csr_bin_workspace": (_SZ, [_I64]),
    "csr_bin_build": (_I32, [_P, _P, _P, _I64, _P, _SZ, _P]),
    "csr_bin_spmv": (_I32, [_P, _P, _P, _P, _P, _P, _P, _I64, _I64, _I64, _I32, _CFGP, _P]),
    "vec_dot_sparse": (_I32, [_P, _P, _P, _P, _I64, _I64, _I32, _P, _SZ, _CFGP, _P]),
    "vec_dot_noalloc": (_I32, [_P, _P, _P, _I64, _I32, _CFGP, _P]),
    "vec_dot_compensated": (_I32, [_P, _P, _P, _I64, _I32, _P, _SZ, _CFGP, _P]),
    "dense_gemv_workspace": (_SZ, [_I64, _I64, _I32, _I32, _CFGP]),
    "dense_gemv": (_I32, [_P, _P, _P, _I64, _I64, _I64, _I32, _I32, _P, _SZ, _CFGP, _P]),
    "dense_gemv_axpby": (_I32, [_P, ctypes.c_double, _P, _P, ctypes.c_double, _I64, _I64, _I64,
                                _I32, _I32, _P, _SZ, _CFGP, _P]),
    "dense_gemv_trans": (_I32, [_P, _P, _P, _I64, _I64, _I64, _I32, _I32, _P, _SZ, _CFGP, _P]),
    "csr_spmv": (_I32, [_P, _P, _P, _P, _P, _I64, _I64, _I64, _I32, _CFGP, _P]),
    "dense_outer": (_I32, [_P, _P, _P, _I64, _I64, _I64, _I32, _P]),
    "csr_sampled_outer": (_I32, [_P, _P, _P, _P, _P, _I64, _I64, _I32, _P]),
    "csr_transpose_workspace": (_SZ, [_I64]),
    "csr_transpose": (_I32, [_P, _P, _P, _P, _P, _I64, _I64, _I64, _P, _SZ, _P]),
    "vec_gather": (_I32, [_P, _P, _P, _I64, _I32, _P]),
    "vec_scale_dev": (_I32, [_P, _P, _P, _I64, _I32, _P]),
    "csr_to_sell_count": (_I32, [_P, _I64, _I32, _P, _P, _P, _P]),
    "csr_to_sell_fill": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P, _P]),
    "sell_pack_values": (_I32, [_P, _P, _P, _I64, _I32, _P]),
    "sell_spmv": (_I32, [_P, _P, _P, _P, _P, _P, _P, _I64, _I32, _CFGP, _P]),
    "lak_batch_plan": (_I32, [_I32, _I32, _P, _I64, _CFGP, _P, _SZ, ctypes.POINTER(BatchInfo)]),
    "lak_batch_run": (_I32, [ctypes.POINTER(BatchInfo), _P, _P, _SZ, _P]),
    "lak_set_batch_default_cfg": (_I32, [_I32, _I32, _CFGP]),
    "lak_probe_fma_f64": (_I32, [_P, _I64, _I32, _I32, _P]),
    "lak_probe_fma_f64_flops": (_I64, [_I64, _I32, _I32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library and declare the C signatures (idempotent)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def last_error() -> str:
    return load().lak_last_error().decode(errors="replace")


def check(fn: str, status: int):
    if status != LAK_OK:
        raise LakError(fn, status, last_error())
