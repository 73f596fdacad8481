"""Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product library never loads
it, and it imports nothing from the product package: the two implementations
share no code.  The only thing they share is the input generator module
``synth``, which holds none of the operations' arithmetic.

The arithmetic lives in ``lak_oracle.c`` (plain loops, compensated Dot2 sums);
this module only widens stored values to double, calls the C routines and
rounds results back to a storage type where a caller asks for it.

Functions and the passages they follow (Rupp et al., IWOCL'14):
  copy, axpy, axpby ........ Sec. 2 (vector copy; x <- alpha*y + beta*z)
  dot ...................... Sec. 2 (inner product <x, y>)
  gemv, gemv_entries ....... Sec. 2 (row i of A times the right-hand side);
                             Sec. 3 for the byte-count convention only
  csr_spmv, csr_rows ....... textbook CSR product (the paper leaves sparse
                             formats out, Sec. 1)
  csr_to_csc, dense_outer,
  sampled_outer, scale ..... reverse-mode derivatives of the products above
  round_bf16 / round_f16 ... reduced-precision storage of the same data
  plain_* .................. NOT reference values: uncompensated FP32/FP64
                             loops that the benchmark times as the "plain CPU"
                             baseline beside the oracle
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lak_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblak_oracle.so")
_lib = None

_F64P = ctypes.POINTER(ctypes.c_double)
_F32P = ctypes.POINTER(ctypes.c_float)
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U16P = ctypes.POINTER(ctypes.c_uint16)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile ``lak_oracle.c`` into ``liblak_oracle.so`` beside it (gcc, -O2,
    -ffp-contract=off so that TwoSum / TwoProduct stay error-free)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
        os.replace(tmp, _LIB_PATH)
    except subprocess.CalledProcessError as e:
        os.unlink(tmp)
        raise RuntimeError(f"oracle build failed:\n{e.stderr}") from e
    return _LIB_PATH


def _bind(path: str):
    """Load a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    sig = {
        "orc_copy": (None, [_F64P, _F64P, _I64]),
        "orc_axpy": (None, [_F64P, _F64P, _F64P, ctypes.c_double, _I64]),
        "orc_axpby": (None, [_F64P, ctypes.c_double, _F64P, ctypes.c_double, _F64P, _I64]),
        "orc_dot": (ctypes.c_double, [_F64P, _F64P, _I64, _F64P]),
        "orc_sparse_dot": (ctypes.c_double, [_F64P, _I32P, _F64P, _I64]),
        "orc_csr_row_bins": (None, [_I32P, _I64, _I64, _I64, _I32P, _I64P]),
        "orc_scale": (None, [_F64P, _F64P, ctypes.c_double, _I64]),
        "orc_gemv": (None, [_F64P, _F64P, _F64P, _I64, _I64, _I64, ctypes.c_int]),
        "orc_gemv_entry": (ctypes.c_double, [_F64P, _F64P, _I64, _I64, _I64, ctypes.c_int]),
        "orc_csr_spmv": (None, [_F64P, _I32P, _I32P, _F64P, _F64P, _I64]),
        "orc_csr_row": (ctypes.c_double, [_I32P, _I32P, _F64P, _F64P, _I64]),
        "orc_csr_to_csc": (ctypes.c_int, [_I32P, _I32P, _I64P, _I32P, _I32P, _I64, _I64]),
        "orc_dense_outer": (None, [_F64P, _F64P, _F64P, _I64, _I64, _I64]),
        "orc_sampled_outer": (None, [_F64P, _I32P, _I32P, _F64P, _F64P, _I64]),
        "orc_round_bf16": (None, [_U16P, _F32P, _I64]),
        "orc_round_bf16_f64": (None, [_U16P, _F64P, _I64]),
        "orc_widen_bf16": (None, [_F64P, _U16P, _I64]),
        "orc_round_f16": (None, [_U16P, _F64P, _I64]),
        "orc_widen_f16": (None, [_F64P, _U16P, _I64]),
        "orc_round_f32": (None, [_F32P, _F64P, _I64]),
        "orc_csr_to_sell": (_I64, [_I32P, _I32P, _I64, _I64, _I64, _I32P, _I32P, _I64P, _I32P,
                                   _I32P]),
        "orc_sell_spmv": (None, [_F64P, _I64, _I64, _I32P, _I32P, _I64P, _I32P, _F64P, _F64P]),
        "orc_plain_copy": (None, [ctypes.c_void_p, ctypes.c_void_p, _I64]),
    }
    for suf, fp, ct in (("f32", _F32P, ctypes.c_float), ("f64", _F64P, ctypes.c_double)):
        sig[f"orc_plain_axpy_{suf}"] = (None, [fp, fp, fp, ct, _I64])
        sig[f"orc_plain_dot_{suf}"] = (ctypes.c_double, [fp, fp, _I64])
        sig[f"orc_plain_gemv_{suf}"] = (None, [fp, fp, fp, _I64, _I64, _I64, ctypes.c_int])
        sig[f"orc_plain_csr_{suf}"] = (None, [fp, _I32P, _I32P, fp, fp, _I64])
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


# ---- marshalling ------------------------------------------------------------

def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctype)


def _as_numpy(a):
    """torch CPU tensor or array-like -> numpy array (bf16 as uint16 bits)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().contiguous()
            if a.dtype == torch.bfloat16:
                return a.view(torch.int16).numpy().view(np.uint16), "bf16"
            if a.dtype == torch.float16:
                return a.view(torch.int16).numpy().view(np.uint16), "f16"
            return a.numpy(), None
    except ImportError:  # pragma: no cover
        pass
    return np.asarray(a), None


def widen(a) -> np.ndarray:
    """Stored values -> float64, exactly (FP32, FP64, BF16 bits, FP16)."""
    arr, tag = _as_numpy(a)
    arr = np.ascontiguousarray(arr).reshape(-1)
    if tag == "bf16":
        out = np.empty(arr.size, np.float64)
        _load().orc_widen_bf16(_ptr(out, _F64P), _ptr(arr, _U16P), arr.size)
        return out
    if tag == "f16":
        out = np.empty(arr.size, np.float64)
        _load().orc_widen_f16(_ptr(out, _F64P), _ptr(arr, _U16P), arr.size)
        return out
    if arr.dtype == np.float16:
        bits = arr.view(np.uint16)
        out = np.empty(arr.size, np.float64)
        _load().orc_widen_f16(_ptr(out, _F64P), _ptr(bits, _U16P), arr.size)
        return out
    return np.ascontiguousarray(arr, dtype=np.float64)


def _i32(a) -> np.ndarray:
    arr, _ = _as_numpy(a)
    return np.ascontiguousarray(arr, dtype=np.int32).reshape(-1)


# ---- operations --------------------------------------------------------------

def copy(y) -> np.ndarray:
    yv = widen(y)
    x = np.empty_like(yv)
    _load().orc_copy(_ptr(x, _F64P), _ptr(yv, _F64P), yv.size)
    return x


def axpy(y, z, alpha: float) -> np.ndarray:
    """x = y + alpha*z in double (the beta = 1 form of Sec. 2's update)."""
    yv, zv = widen(y), widen(z)
    assert yv.size == zv.size
    x = np.empty_like(yv)
    _load().orc_axpy(_ptr(x, _F64P), _ptr(yv, _F64P), _ptr(zv, _F64P), float(alpha), yv.size)
    return x


def axpby(alpha: float, y, beta: float, z) -> np.ndarray:
    """x = alpha*y + beta*z in double (Sec. 2's scaled vector addition)."""
    yv, zv = widen(y), widen(z)
    x = np.empty_like(yv)
    _load().orc_axpby(_ptr(x, _F64P), float(alpha), _ptr(yv, _F64P), float(beta),
                      _ptr(zv, _F64P), yv.size)
    return x


def dot(x, y, with_lo: bool = False):
    """<x, y> as a compensated (Dot2) sum; with_lo also returns the remainder."""
    xv, yv = widen(x), widen(y)
    assert xv.size == yv.size
    lo = ctypes.c_double(0.0)
    hi = _load().orc_dot(_ptr(xv, _F64P), _ptr(yv, _F64P), xv.size, ctypes.byref(lo))
    return (hi, lo.value) if with_lo else hi


def sparse_dot(vals, idx, y) -> float:
    """sum_k vals[k] * y[idx[k]] (compensated, increasing k)."""
    vv, yv, iv = widen(vals), widen(y), _i32(idx)
    assert vv.size == iv.size
    if iv.size:
        assert 0 <= int(iv.min()) and int(iv.max()) < yv.size
    return _load().orc_sparse_dot(_ptr(vv, _F64P), _ptr(iv, _I32P), _ptr(yv, _F64P), vv.size)


def scale(v, s: float) -> np.ndarray:
    vv = widen(v)
    out = np.empty_like(vv)
    _load().orc_scale(_ptr(out, _F64P), _ptr(vv, _F64P), float(s), vv.size)
    return out


def gemv(A, x, m: int, n: int, lda: int, layout: str = "row") -> np.ndarray:
    """y = A x; A given as its flat storage (row: A[i*lda+j], col: A[i+j*lda])."""
    Av, xv = widen(A), widen(x)
    lay = {"row": 0, "col": 1}[layout]
    need = (m - 1) * lda + n if lay == 0 else (n - 1) * lda + m
    assert m == 0 or n == 0 or Av.size >= need, "matrix storage too small for m, n, lda"
    assert xv.size >= n
    y = np.empty(m, np.float64)
    _load().orc_gemv(_ptr(y, _F64P), _ptr(Av, _F64P), _ptr(xv, _F64P), m, n, lda, lay)
    return y


def gemv_entries(A, x, rows, n: int, lda: int, layout: str = "row") -> np.ndarray:
    """Selected entries y[rows] of y = A x (sampled checks at full size)."""
    Av, xv = widen(A), widen(x)
    lay = {"row": 0, "col": 1}[layout]
    lib = _load()
    return np.array([lib.orc_gemv_entry(_ptr(Av, _F64P), _ptr(xv, _F64P), int(i), n, lda, lay)
                     for i in rows], dtype=np.float64)


def csr_spmv(row_ptr, col_idx, vals, x) -> np.ndarray:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    vv, xv = widen(vals), widen(x)
    m = rp.size - 1
    y = np.empty(m, np.float64)
    _load().orc_csr_spmv(_ptr(y, _F64P), _ptr(rp, _I32P), _ptr(ci, _I32P),
                         _ptr(vv, _F64P), _ptr(xv, _F64P), m)
    return y


def csr_rows(row_ptr, col_idx, vals, x, rows) -> np.ndarray:
    rp, ci = _i32(row_ptr), _i32(col_idx)
    vv, xv = widen(vals), widen(x)
    lib = _load()
    return np.array([lib.orc_csr_row(_ptr(rp, _I32P), _ptr(ci, _I32P), _ptr(vv, _F64P),
                                     _ptr(xv, _F64P), int(i)) for i in rows], dtype=np.float64)


def csr_to_csc(row_ptr, col_idx, n: int):
    """(col_ptr, row_idx, perm): the CSC form of an m-by-n CSR matrix."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    m = rp.size - 1
    nnz = int(rp[-1]) if m >= 0 and rp.size else 0
    col_ptr = np.empty(n + 1, np.int32)
    row_idx = np.empty(max(nnz, 1), np.int32)
    perm = np.empty(max(nnz, 1), np.int64)
    rc = _load().orc_csr_to_csc(_ptr(col_ptr, _I32P), _ptr(row_idx, _I32P), _ptr(perm, _I64P),
                                _ptr(rp, _I32P), _ptr(ci, _I32P), m, n)
    if rc != 0:
        raise MemoryError("oracle csr_to_csc: allocation failed")
    return col_ptr, row_idx[:nnz], perm[:nnz]


def csr_row_bins(row_ptr, per_lane: int = 8, nbins: int = 7):
    """Row-binned CSR: (perm, bin_ptr) -- rows grouped by length bin, stable
    within a bin; see lak_oracle.c for the bin rule."""
    rp = _i32(row_ptr)
    m = rp.size - 1
    perm = np.empty(max(m, 1), np.int32)
    bptr = np.empty(nbins + 1, np.int64)
    _load().orc_csr_row_bins(_ptr(rp, _I32P), m, per_lane, nbins, _ptr(perm, _I32P),
                             _ptr(bptr, _I64P))
    return perm[:m], bptr


def csr_to_sell(row_ptr, col_idx, C: int = 32, sigma: int = 1):
    """SELL-C-sigma form: (perm, slice_len, slice_ptr, cols, map) -- see
    lak_oracle.c for the layout."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    m = rp.size - 1
    mp = (m + C - 1) // C * C
    ns = mp // C
    perm = np.empty(max(mp, 1), np.int32)
    slen = np.empty(max(ns, 1), np.int32)
    sptr = np.empty(ns + 1, np.int64)
    lib = _load()
    nil = ctypes.POINTER(ctypes.c_int32)()
    total = lib.orc_csr_to_sell(_ptr(rp, _I32P), _ptr(ci, _I32P), m, C, sigma, _ptr(perm, _I32P),
                                _ptr(slen, _I32P), _ptr(sptr, _I64P), nil, nil)
    cols = np.empty(max(total, 1), np.int32)
    mp_ = np.empty(max(total, 1), np.int32)
    lib.orc_csr_to_sell(_ptr(rp, _I32P), _ptr(ci, _I32P), m, C, sigma, _ptr(perm, _I32P),
                        _ptr(slen, _I32P), _ptr(sptr, _I64P), _ptr(cols, _I32P), _ptr(mp_, _I32P))
    return perm[:mp], slen[:ns], sptr, cols[:total], mp_[:total]


def sell_spmv(perm, slice_len, slice_ptr, cols, sell_vals, x, m: int, C: int = 32) -> np.ndarray:
    """y = A x from SELL-C-sigma arrays (sell_vals in SELL slots)."""
    pm, sl, co = _i32(perm), _i32(slice_len), _i32(cols)
    sp = np.ascontiguousarray(np.asarray(slice_ptr), dtype=np.int64)
    vv, xv = widen(sell_vals), widen(x)
    y = np.zeros(m, np.float64)
    _load().orc_sell_spmv(_ptr(y, _F64P), m, C, _ptr(pm, _I32P), _ptr(sl, _I32P), _ptr(sp, _I64P),
                          _ptr(co, _I32P), _ptr(vv, _F64P), _ptr(xv, _F64P))
    return y


def dense_outer(dy, x) -> np.ndarray:
    """dA = dy x^T (m-by-n, row-major), the gradient of y = A x w.r.t. A."""
    dyv, xv = widen(dy), widen(x)
    m, n = dyv.size, xv.size
    dA = np.empty(m * n, np.float64)
    _load().orc_dense_outer(_ptr(dA, _F64P), _ptr(dyv, _F64P), _ptr(xv, _F64P), m, n, n)
    return dA.reshape(m, n)


def sampled_outer(row_ptr, col_idx, dy, x) -> np.ndarray:
    """dvals[k] = dy[row(k)] * x[col(k)]: the CSR gradient on the stored pattern."""
    rp, ci = _i32(row_ptr), _i32(col_idx)
    dyv, xv = widen(dy), widen(x)
    m = rp.size - 1
    nnz = int(rp[-1])
    out = np.empty(max(nnz, 1), np.float64)
    _load().orc_sampled_outer(_ptr(out, _F64P), _ptr(rp, _I32P), _ptr(ci, _I32P),
                              _ptr(dyv, _F64P), _ptr(xv, _F64P), m)
    return out[:nnz]


# ---- storage rounding ----------------------------------------------------------

def round_f32(v) -> np.ndarray:
    vv = widen(v)
    out = np.empty(vv.size, np.float32)
    _load().orc_round_f32(_ptr(out, _F32P), _ptr(vv, _F64P), vv.size)
    return out


def round_bf16(v_f32) -> np.ndarray:
    """FP32 values -> BF16 bit patterns (uint16), round to nearest even."""
    f = np.ascontiguousarray(np.asarray(v_f32, dtype=np.float32)).reshape(-1)
    out = np.empty(f.size, np.uint16)
    _load().orc_round_bf16(_ptr(out, _U16P), _ptr(f, _F32P), f.size)
    return out


def round_bf16_f64(v) -> np.ndarray:
    """double values -> BF16 bit patterns (uint16), one round to nearest even."""
    vv = widen(v)
    out = np.empty(vv.size, np.uint16)
    _load().orc_round_bf16_f64(_ptr(out, _U16P), _ptr(vv, _F64P), vv.size)
    return out


def round_f16(v) -> np.ndarray:
    """double values -> IEEE binary16 bit patterns (uint16), round to nearest even."""
    vv = widen(v)
    out = np.empty(vv.size, np.uint16)
    _load().orc_round_f16(_ptr(out, _U16P), _ptr(vv, _F64P), vv.size)
    return out


def widen_bf16_bits(bits) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint16)).reshape(-1)
    out = np.empty(b.size, np.float64)
    _load().orc_widen_bf16(_ptr(out, _F64P), _ptr(b, _U16P), b.size)
    return out


def widen_f16_bits(bits) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint16)).reshape(-1)
    out = np.empty(b.size, np.float64)
    _load().orc_widen_f16(_ptr(out, _F64P), _ptr(b, _U16P), b.size)
    return out


def round_to(v, storage: str) -> np.ndarray:
    """double results -> the stored values of a storage type, as float64."""
    if storage == "f64":
        return widen(v)
    if storage == "f32":
        return round_f32(v).astype(np.float64)
    if storage == "bf16":
        return widen_bf16_bits(round_bf16_f64(v))
    if storage == "f16":
        return widen_f16_bits(round_f16(v))
    raise ValueError(storage)


# ---- plain loops (the "plain CPU" baseline; not reference values) ---------------

def plain_axpy(y, z, alpha: float, out=None):
    """x = y + alpha z in the inputs' own precision (float32 or float64 arrays)."""
    suf = "f32" if y.dtype == np.float32 else "f64"
    x = np.empty_like(y) if out is None else out
    fp = _F32P if suf == "f32" else _F64P
    getattr(_load(), f"orc_plain_axpy_{suf}")(_ptr(x, fp), _ptr(y, fp), _ptr(z, fp), alpha, y.size)
    return x


def plain_dot(x, y) -> float:
    suf = "f32" if x.dtype == np.float32 else "f64"
    fp = _F32P if suf == "f32" else _F64P
    return getattr(_load(), f"orc_plain_dot_{suf}")(_ptr(x, fp), _ptr(y, fp), x.size)


def plain_gemv(A, x, m: int, n: int, lda: int, layout: str = "row", out=None):
    suf = "f32" if A.dtype == np.float32 else "f64"
    fp = _F32P if suf == "f32" else _F64P
    y = np.empty(m, A.dtype) if out is None else out
    getattr(_load(), f"orc_plain_gemv_{suf}")(_ptr(y, fp), _ptr(A, fp), _ptr(x, fp), m, n, lda,
                                              {"row": 0, "col": 1}[layout])
    return y


def plain_csr(row_ptr, col_idx, vals, x, out=None):
    suf = "f32" if vals.dtype == np.float32 else "f64"
    fp = _F32P if suf == "f32" else _F64P
    m = row_ptr.size - 1
    y = np.empty(m, vals.dtype) if out is None else out
    getattr(_load(), f"orc_plain_csr_{suf}")(_ptr(y, fp), _ptr(row_ptr, _I32P),
                                             _ptr(col_idx, _I32P), _ptr(vals, fp), _ptr(x, fp), m)
    return y


def plain_copy(y, out=None):
    x = np.empty_like(y) if out is None else out
    _load().orc_plain_copy(x.ctypes.data, y.ctypes.data, y.nbytes)
    return x
