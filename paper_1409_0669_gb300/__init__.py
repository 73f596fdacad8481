"""GB300 (sm_103a) library of memory-bandwidth-bound linear-algebra kernels.

The operations of Rupp et al., "Performance Portability Study of Linear
Algebra Kernels in OpenCL" (IWOCL'14, Sec. 2) -- vector copy, vector update
x = y + alpha*z, inner product <x, y>, dense matrix-vector product in row- and
column-major layouts -- plus the CSR sparse matrix-vector product, as
hand-written CUDA kernels behind the C ABI of ``include/lak.h``.

This module is the thin Python binding: it checks tensor devices, dtypes and
strides, turns tensors into raw device pointers and calls the C entry points of
the same names on the current CUDA stream.  Every arithmetic step runs in the
CUDA library; PyTorch only supplies device memory and streams.  Workspace for
the calls that need it is kept per (device, stream), zero-filled when first
allocated, which is the state the kernels require and leave behind.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Union

import torch

from . import _native
from ._native import DTYPES, INCREMENTS, LAYOUTS, OPS, LakCfg, LakError

__all__ = ["vec_copy", "vec_axpy", "vec_axpby", "vec_axpy_norm2", "vec_axpy_norm2_workspace",
           "dense_gemv_trans", "vec_dot", "vec_dot_workspace", "vec_dot_sparse",
           "vec_dot_sparse_workspace", "vec_dot_compensated",
           "vec_dot_noalloc", "dense_gemv",
           "dense_gemv_workspace", "csr_spmv", "dense_outer", "csr_sampled_outer",
           "csr_transpose", "vec_gather", "vec_scale_dev", "resolve_cfg", "set_default_cfg",
           "size_bucket", "SIZE_BUCKETS", "Cfg", "set_batch_default_cfg", "probe_fma_f64",
           "LakError", "storage_of", "library_path"]

_lib = _native.load()

_TORCH_TO_STORAGE = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16",
                     torch.float16: "f16"}

CfgLike = Union[None, LakCfg, Sequence[int], dict]


def library_path() -> str:
    return _native.LIB_PATH


def Cfg(block: int = 0, grid: int = 0, vec: int = 0, increment: Union[int, str] = 0) -> LakCfg:
    """A launch configuration (Sec. 2's local size, work-groups, vector
    length, increment type); zeros mean automatic."""
    inc = INCREMENTS[increment] if isinstance(increment, str) else int(increment)
    return LakCfg(int(block), int(grid), int(vec), inc)


def _cfg_ptr(cfg: CfgLike):
    if cfg is None:
        return None
    if isinstance(cfg, LakCfg):
        c = cfg
    elif isinstance(cfg, dict):
        c = Cfg(**cfg)
    else:
        c = Cfg(*cfg)
    return ctypes.byref(c)


def storage_of(t: torch.Tensor) -> str:
    try:
        return _TORCH_TO_STORAGE[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {t.dtype}; expected float32/float64/bfloat16/float16")


# The current stream's raw handle without building a torch Stream object (the
# public call costs ~3 us per launch, more than the launch itself).
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)


_current_device = getattr(torch._C, "_cuda_getDevice", None) or torch.cuda.current_device


def _stream(stream) -> int:
    if stream is None:
        if _raw_stream is not None:
            return _raw_stream(_current_device())
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        if stream.device.index != _current_device():
            raise ValueError(f"stream is on {stream.device} but the current device is "
                             f"cuda:{_current_device()}")
        return stream.cuda_stream
    return int(stream)


def _dev_ptr(t: torch.Tensor, name: str) -> int:
    """Device address of an operand.  The library launches on the current
    device (and finds per-device state such as built-in scratch through it),
    so an operand on another device is refused here rather than handed to a
    kernel running elsewhere."""
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    cur = _current_device()
    if t.device.index != cur:
        raise ValueError(f"{name} is on {t.device} but the current device is cuda:{cur}; "
                         f"call under `with torch.cuda.device({t.device.index}):`")
    return t.data_ptr()


def _on_current_device(*ts):
    """Refuse CUDA tensors on a device other than the current one (see _dev_ptr)."""
    for t in ts:
        if t is not None and t.numel() > 0:
            _dev_ptr(t, "operand")


def _vec_arg(t: torch.Tensor, name: str):
    if t.dim() != 1 or (t.numel() > 1 and t.stride(0) != 1):
        raise ValueError(f"{name} must be a contiguous 1-D tensor")
    return _dev_ptr(t, name)


def _same_storage(*ts):
    s = storage_of(ts[0])
    for t in ts[1:]:
        if t.dtype != ts[0].dtype:
            raise TypeError("all operands must share one dtype")
        if t.device != ts[0].device:
            raise ValueError("all operands must be on one device")
    return s


# ---- workspace -------------------------------------------------------------------

_workspaces = {}


def _workspace(nbytes: int, stream_handle: int, device: torch.device) -> torch.Tensor:
    """Zero-filled scratch kept per (device, stream); grown (and re-zeroed)
    when a call needs more.  Kernels leave their counters at zero."""
    key = (device.index, stream_handle)
    ws = _workspaces.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.zeros(max(nbytes, 256), dtype=torch.uint8, device=device)
        _workspaces[key] = ws
    return ws


# ---- entry points ----------------------------------------------------------------

def resolve_cfg(op: str, storage: str, m: int, n: int = 0, nnz: int = 0,
                cfg: CfgLike = None) -> LakCfg:
    """The launch configuration the library would use (lak_resolve_cfg)."""
    out = LakCfg()
    st = _lib.lak_resolve_cfg(OPS[op], DTYPES[storage], int(m), int(n), int(nnz), _cfg_ptr(cfg),
                              ctypes.byref(out))
    _native.check("lak_resolve_cfg", st)
    return out


SIZE_BUCKETS = 4


def size_bucket(op: str, storage: str, m: int, n: int = 0, nnz: int = 0) -> int:
    """The size bucket (0..3) of a call with these sizes (lak_size_bucket);
    sizes as in resolve_cfg."""
    b = _lib.lak_size_bucket(OPS[op], DTYPES[storage], int(m), int(n), int(nnz))
    if b < 0:
        _native.check("lak_size_bucket", b)
    return b


def set_default_cfg(op: str, storage: str, cfg: CfgLike, bucket: Optional[int] = None):
    """Replace (or with cfg=None restore) the default configuration of an op,
    in one size bucket or (bucket=None) in all of them."""
    b = -1 if bucket is None else int(bucket)
    _native.check("lak_set_default_cfg",
                  _lib.lak_set_default_cfg_bucket(OPS[op], DTYPES[storage], b, _cfg_ptr(cfg)))
    _dot_ws_sizes.clear()                 # workspace needs follow the defaults


# (op, storage) pairs whose batched default the caller set: the shipped
# autotuned defaults, installed when the first batch is planned, leave them alone
_user_batch_defaults = set()


def _apply_batch_default(op: str, storage: str, cfg: CfgLike):
    _native.check("lak_set_batch_default_cfg",
                  _lib.lak_set_batch_default_cfg(OPS[op], DTYPES[storage], _cfg_ptr(cfg)))


def set_batch_default_cfg(op: str, storage: str, cfg: CfgLike):
    """Replace (or with cfg=None restore the built-in shape of) the launch
    configuration that batched launches of `op` take when planned without one.
    Process-wide; takes precedence over the shipped autotuned defaults."""
    _apply_batch_default(op, storage, cfg)
    _user_batch_defaults.add((op, storage))


def probe_fma_f64(iters: int, grid: Optional[int] = None, block: int = 256,
                  out: Optional[torch.Tensor] = None, stream=None):
    """Launch the FP64 FMA throughput probe (lak_probe_fma_f64) on the current
    device; grid defaults to as many blocks as are resident at once.  Returns
    (out, flops of the launch)."""
    if grid is None:
        p = torch.cuda.get_device_properties(_current_device())
        grid = p.multi_processor_count * (p.max_threads_per_multi_processor // block)
    if out is None:
        out = torch.empty(grid * block // 32, dtype=torch.float64,
                          device=torch.device("cuda", _current_device()))
    st = _lib.lak_probe_fma_f64(_dev_ptr(out, "out"), int(iters), int(grid), int(block),
                                _stream(stream))
    _native.check("lak_probe_fma_f64", st)
    return out, int(_lib.lak_probe_fma_f64_flops(int(iters), int(grid), int(block)))


# vec_dot_workspace(n, storage) for calls without an explicit cfg, memoised
# (cleared whenever a default configuration changes)
_dot_ws_sizes = {}


def _dot_ws_need(n: int, storage: str, cfg: CfgLike) -> int:
    if cfg is not None:
        return vec_dot_workspace(n, storage, cfg)
    key = (n, storage, torch.cuda.current_device())
    need = _dot_ws_sizes.get(key)
    if need is None:
        need = _dot_ws_sizes[key] = vec_dot_workspace(n, storage)
    return need


def vec_copy(x: torch.Tensor, y: torch.Tensor, cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """x[:] = y (bit copy)."""
    s = _same_storage(x, y)
    if x.numel() != y.numel():
        raise ValueError("x and y must have the same length")
    st = _lib.vec_copy(_vec_arg(x, "x"), _vec_arg(y, "y"), x.numel(), DTYPES[s], _cfg_ptr(cfg),
                       _stream(stream))
    _native.check("vec_copy", st)
    return x


def vec_axpy(x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, alpha: float,
             cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """x[:] = y + alpha * z."""
    s = _same_storage(x, y, z)
    n = x.numel()
    if y.numel() != n or z.numel() != n:
        raise ValueError("x, y, z must have the same length")
    st = _lib.vec_axpy(_vec_arg(x, "x"), _vec_arg(y, "y"), _vec_arg(z, "z"), float(alpha), n,
                       DTYPES[s], _cfg_ptr(cfg), _stream(stream))
    _native.check("vec_axpy", st)
    return x


def vec_axpby(x: torch.Tensor, alpha: float, y: torch.Tensor, beta: float, z: torch.Tensor,
              cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """x[:] = alpha*y + beta*z; 1-D views with any (nonzero for x) strides take
    the strided kernel, contiguous ones the vectorised kernel."""
    s = _same_storage(x, y, z)
    n = x.numel()
    if y.numel() != n or z.numel() != n:
        raise ValueError("x, y, z must have the same length")
    if x.dim() != 1 or y.dim() != 1 or z.dim() != 1:
        raise ValueError("x, y, z must be 1-D")
    for t, nm in ((x, "x"), (y, "y"), (z, "z")):
        _dev_ptr(t, nm)
    if all(t.stride(0) == 1 or n <= 1 for t in (x, y, z)):
        st = _lib.vec_axpby(x.data_ptr(), float(alpha), y.data_ptr(), float(beta), z.data_ptr(),
                            n, DTYPES[s], _cfg_ptr(cfg), _stream(stream))
        _native.check("vec_axpby", st)
    else:
        st = _lib.vec_axpby_strided(x.data_ptr(), x.stride(0), float(alpha), y.data_ptr(),
                                    y.stride(0), float(beta), z.data_ptr(), z.stride(0), n,
                                    DTYPES[s], _stream(stream))
        _native.check("vec_axpby_strided", st)
    return x


def vec_axpy_norm2(x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, alpha: float,
                   out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                   cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """x[:] = y + alpha*z and returns <x, x> (one-element device tensor), in one pass."""
    s = _same_storage(x, y, z)
    n = x.numel()
    if y.numel() != n or z.numel() != n:
        raise ValueError("x, y, z must have the same length")
    odt = torch.float64 if s == "f64" else torch.float32
    if out is None:
        out = torch.empty(1, dtype=odt, device=x.device)
    sh = _stream(stream)
    need = int(_lib.vec_axpy_norm2_workspace(n, DTYPES[s], _cfg_ptr(cfg)))
    if workspace is None:
        workspace = _workspace(need, sh, x.device)
    st = _lib.vec_axpy_norm2(_vec_arg(x, "x"), _vec_arg(y, "y"), _vec_arg(z, "z"), float(alpha),
                             _dev_ptr(out, "out"), n, DTYPES[s], _dev_ptr(workspace, "workspace"),
                             workspace.numel(), _cfg_ptr(cfg), sh)
    _native.check("vec_axpy_norm2", st)
    return out


def vec_axpy_norm2_workspace(n: int, storage: str, cfg: CfgLike = None) -> int:
    return int(_lib.vec_axpy_norm2_workspace(int(n), DTYPES[storage], _cfg_ptr(cfg)))


def vec_dot_workspace(n: int, storage: str, cfg: CfgLike = None) -> int:
    return int(_lib.vec_dot_workspace(int(n), DTYPES[storage], _cfg_ptr(cfg)))


def vec_dot(x: torch.Tensor, y: torch.Tensor, out: Optional[torch.Tensor] = None,
            workspace: Optional[torch.Tensor] = None, cfg: CfgLike = None,
            stream=None) -> torch.Tensor:
    """<x, y> into a one-element device tensor (float32 for FP32/BF16/FP16
    storage, float64 for FP64)."""
    s = _same_storage(x, y)
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    odt = torch.float64 if s == "f64" else torch.float32
    if out is None:
        out = torch.empty(1, dtype=odt, device=x.device)
    elif out.dtype != odt or out.numel() < 1:
        raise TypeError(f"out must be a {odt} tensor with at least one element")
    sh = _stream(stream)
    if workspace is None:
        workspace = _workspace(_dot_ws_need(n, s, cfg), sh, x.device)
    st = _lib.vec_dot(_dev_ptr(out, "out"), _vec_arg(x, "x"), _vec_arg(y, "y"), n, DTYPES[s],
                      _dev_ptr(workspace, "workspace"), workspace.numel() * workspace.element_size(),
                      _cfg_ptr(cfg), sh)
    _native.check("vec_dot", st)
    return out


def vec_dot_sparse_workspace(nnz: int, storage: str, cfg: CfgLike = None) -> int:
    return int(_lib.vec_dot_sparse_workspace(int(nnz), DTYPES[storage], _cfg_ptr(cfg)))


def vec_dot_sparse(vals: torch.Tensor, idx: torch.Tensor, y: torch.Tensor,
                   out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                   cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """sum_k vals[k] * y[idx[k]] (idx int32, 0 <= idx < len(y)) into a
    one-element device tensor (float32 for FP32/BF16/FP16 storage, float64 for
    FP64)."""
    s = _same_storage(vals, y)
    nnz = vals.numel()
    if idx.numel() != nnz:
        raise ValueError("vals and idx must have the same length")
    if idx.dtype != torch.int32:
        raise TypeError("idx must be int32")
    odt = torch.float64 if s == "f64" else torch.float32
    if out is None:
        out = torch.empty(1, dtype=odt, device=y.device)
    elif out.dtype != odt or out.numel() < 1:
        raise TypeError(f"out must be a {odt} tensor with at least one element")
    sh = _stream(stream)
    need = vec_dot_sparse_workspace(nnz, s, cfg)
    if workspace is None:
        workspace = _workspace(need, sh, y.device)
    st = _lib.vec_dot_sparse(_dev_ptr(out, "out"), _vec_arg(vals, "vals") if nnz else None,
                             _vec_arg(idx, "idx") if nnz else None,
                             _vec_arg(y, "y") if y.numel() else None, nnz, y.numel(), DTYPES[s],
                             _dev_ptr(workspace, "workspace"),
                             workspace.numel() * workspace.element_size(), _cfg_ptr(cfg), sh)
    _native.check("vec_dot_sparse", st)
    return out


def vec_dot_compensated(x: torch.Tensor, y: torch.Tensor, out: Optional[torch.Tensor] = None,
                        workspace: Optional[torch.Tensor] = None, cfg: CfgLike = None,
                        stream=None) -> torch.Tensor:
    """<x, y> for FP32/BF16/FP16 storage with compensated (Dot2) FP32
    accumulation and an FP64 combine; the result is a one-element float64
    device tensor."""
    s = _same_storage(x, y)
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=x.device)
    elif out.dtype != torch.float64 or out.numel() < 1:
        raise TypeError("out must be a float64 tensor with at least one element")
    sh = _stream(stream)
    if workspace is None:
        workspace = _workspace(_dot_ws_need(n, s, cfg), sh, x.device)
    st = _lib.vec_dot_compensated(_dev_ptr(out, "out"), _vec_arg(x, "x"), _vec_arg(y, "y"), n,
                                  DTYPES[s], _dev_ptr(workspace, "workspace"),
                                  workspace.numel() * workspace.element_size(), _cfg_ptr(cfg), sh)
    _native.check("vec_dot_compensated", st)
    return out


def vec_dot_noalloc(x: torch.Tensor, y: torch.Tensor, out: Optional[torch.Tensor] = None,
                    cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """<x, y> like vec_dot, but using the library's built-in scratch instead of a
    workspace (for callers that cannot provide device scratch memory; calls
    must not overlap on the GPU -- see include/lak.h)."""
    s = _same_storage(x, y)
    n = x.numel()
    if y.numel() != n:
        raise ValueError("x and y must have the same length")
    odt = torch.float64 if s == "f64" else torch.float32
    if out is None:
        out = torch.empty(1, dtype=odt, device=x.device)
    elif out.dtype != odt or out.numel() < 1:
        raise TypeError(f"out must be a {odt} tensor with at least one element")
    st = _lib.vec_dot_noalloc(_dev_ptr(out, "out"), _vec_arg(x, "x"), _vec_arg(y, "y"), n,
                              DTYPES[s], _cfg_ptr(cfg), _stream(stream))
    _native.check("vec_dot_noalloc", st)
    return out


def dense_gemv_workspace(m: int, n: int, layout: str, storage: str, cfg: CfgLike = None) -> int:
    return int(_lib.dense_gemv_workspace(int(m), int(n), LAYOUTS[layout], DTYPES[storage],
                                         _cfg_ptr(cfg)))


def _matrix_layout(A: torch.Tensor):
    """(m, n, lda, layout) of a 2-D tensor viewed as a row- or column-major matrix."""
    if A.dim() != 2:
        raise ValueError("A must be 2-D (or pass m, n, lda and layout with a 1-D buffer)")
    m, n = A.shape
    s0, s1 = A.stride()
    if s1 == 1 and (m <= 1 or s0 >= max(n, 1)):
        return m, n, (s0 if m > 1 else max(n, 1)), "row"
    if s0 == 1 and (n <= 1 or s1 >= max(m, 1)):
        return m, n, (s1 if n > 1 else max(m, 1)), "col"
    raise ValueError("A must have unit stride along one dimension")


def dense_gemv(A: torch.Tensor, x: torch.Tensor, y: Optional[torch.Tensor] = None,
               m: Optional[int] = None, n: Optional[int] = None, lda: Optional[int] = None,
               layout: Optional[str] = None, workspace: Optional[torch.Tensor] = None,
               cfg: CfgLike = None, stream=None, alpha: float = 1.0,
               beta: float = 0.0) -> torch.Tensor:
    """y = alpha * A x + beta * y (y is not read when beta == 0).  A is a 2-D
    tensor (its strides give the layout and lda), or a 1-D buffer with
    explicit m, n, lda and layout ('row' or 'col')."""
    s = _same_storage(A, x)
    if A.dim() == 2 and m is None:
        m, n, lda, lay = _matrix_layout(A)
        if layout is not None and layout != lay:
            raise ValueError(f"A's strides give layout {lay!r}, not {layout!r}")
        layout = lay
    else:
        if None in (m, n, lda, layout):
            raise ValueError("a 1-D matrix buffer needs m, n, lda and layout")
    if layout not in LAYOUTS:
        raise ValueError(f"layout must be 'row' or 'col', not {layout!r}")
    if x.numel() != n:
        raise ValueError(f"x has {x.numel()} elements, expected n={n}")
    if y is None:
        y = torch.empty(m, dtype=A.dtype, device=A.device)
    elif y.dtype != A.dtype or y.numel() != m:
        raise ValueError("y must match A's dtype and have m elements")
    sh = _stream(stream)
    need = dense_gemv_workspace(m, n, layout, s, cfg)
    ws_ptr, ws_bytes = None, 0
    if need > 0:
        if workspace is None:
            workspace = _workspace(need, sh, A.device)
        ws_ptr = _dev_ptr(workspace, "workspace")
        ws_bytes = workspace.numel() * workspace.element_size()
    if alpha == 1.0 and beta == 0.0:
        st = _lib.dense_gemv(_vec_arg(y, "y"), _dev_ptr(A, "A"), _vec_arg(x, "x"), int(m), int(n),
                             int(lda), LAYOUTS[layout], DTYPES[s], ws_ptr, ws_bytes, _cfg_ptr(cfg),
                             sh)
        _native.check("dense_gemv", st)
    else:
        st = _lib.dense_gemv_axpby(_vec_arg(y, "y"), float(alpha), _dev_ptr(A, "A"),
                                   _vec_arg(x, "x"), float(beta), int(m), int(n), int(lda),
                                   LAYOUTS[layout], DTYPES[s], ws_ptr, ws_bytes, _cfg_ptr(cfg), sh)
        _native.check("dense_gemv_axpby", st)
    return y


def dense_gemv_trans(A: torch.Tensor, x: torch.Tensor, y: Optional[torch.Tensor] = None,
                     workspace: Optional[torch.Tensor] = None, cfg: CfgLike = None,
                     stream=None) -> torch.Tensor:
    """y = A^T x for a 2-D tensor A (row- or column-major), through the
    dense_gemv_trans entry point."""
    s = _same_storage(A, x)
    m, n, lda, layout = _matrix_layout(A)
    if x.numel() != m:
        raise ValueError(f"x has {x.numel()} elements, expected m={m}")
    if y is None:
        y = torch.empty(n, dtype=A.dtype, device=A.device)
    other = "col" if layout == "row" else "row"
    sh = _stream(stream)
    need = dense_gemv_workspace(n, m, other, s, cfg)
    ws_ptr, ws_bytes = None, 0
    if need > 0:
        if workspace is None:
            workspace = _workspace(need, sh, A.device)
        ws_ptr, ws_bytes = _dev_ptr(workspace, "workspace"), workspace.numel()
    st = _lib.dense_gemv_trans(_vec_arg(y, "y"), _dev_ptr(A, "A"), _vec_arg(x, "x"), m, n, lda,
                               LAYOUTS[layout], DTYPES[s], ws_ptr, ws_bytes, _cfg_ptr(cfg), sh)
    _native.check("dense_gemv_trans", st)
    return y


def csr_spmv(row_ptr: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor, x: torch.Tensor,
             y: Optional[torch.Tensor] = None, n_cols: Optional[int] = None,
             cfg: CfgLike = None, stream=None) -> torch.Tensor:
    """y = A x for A in CSR form (int32 row_ptr of m+1 entries, int32 col_idx)."""
    s = _same_storage(vals, x)
    if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32:
        raise TypeError("row_ptr and col_idx must be int32")
    m = row_ptr.numel() - 1
    if m < 0:
        raise ValueError("row_ptr needs m+1 >= 1 entries")
    nnz = vals.numel()
    if col_idx.numel() != nnz:
        raise ValueError("col_idx and vals must have nnz entries each")
    n = x.numel() if n_cols is None else int(n_cols)
    if y is None:
        y = torch.empty(m, dtype=vals.dtype, device=vals.device)
    elif y.dtype != vals.dtype or y.numel() != m:
        raise ValueError("y must match vals' dtype and have m elements")
    st = _lib.csr_spmv(_vec_arg(y, "y"), _vec_arg(row_ptr, "row_ptr"),
                       _vec_arg(col_idx, "col_idx") if nnz else None,
                       _vec_arg(vals, "vals") if nnz else None, _vec_arg(x, "x") if n else None,
                       m, n, nnz, DTYPES[s], _cfg_ptr(cfg), _stream(stream))
    _native.check("csr_spmv", st)
    return y


# ---- reverse-mode building blocks ---------------------------------------------------

def dense_outer(dy: torch.Tensor, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
    """dA = dy x^T as an (m, n) row-major tensor."""
    s = _same_storage(dy, x)
    m, n = dy.numel(), x.numel()
    if out is None:
        out = torch.empty(m, n, dtype=dy.dtype, device=dy.device)
    if out.dim() != 2 or out.shape != (m, n) or (n > 1 and out.stride(1) != 1):
        raise ValueError("out must be an (m, n) tensor with unit stride along rows")
    ldd = out.stride(0) if m > 1 else max(n, 1)
    st = _lib.dense_outer(_dev_ptr(out, "out"), _vec_arg(dy, "dy"), _vec_arg(x, "x"), m, n, ldd,
                          DTYPES[s], _stream(stream))
    _native.check("dense_outer", st)
    return out


def csr_sampled_outer(row_ptr: torch.Tensor, col_idx: torch.Tensor, dy: torch.Tensor,
                      x: torch.Tensor, out: Optional[torch.Tensor] = None,
                      stream=None) -> torch.Tensor:
    """dvals[k] = dy[row(k)] * x[col(k)] on the CSR pattern."""
    s = _same_storage(dy, x)
    m = row_ptr.numel() - 1
    nnz = col_idx.numel()
    if out is None:
        out = torch.empty(nnz, dtype=dy.dtype, device=dy.device)
    st = _lib.csr_sampled_outer(_vec_arg(out, "out") if nnz else None, _vec_arg(row_ptr, "row_ptr"),
                                _vec_arg(col_idx, "col_idx") if nnz else None, _vec_arg(dy, "dy"),
                                _vec_arg(x, "x") if x.numel() else None, m, nnz, DTYPES[s],
                                _stream(stream))
    _native.check("csr_sampled_outer", st)
    return out


def csr_transpose(row_ptr: torch.Tensor, col_idx: torch.Tensor, n_cols: int, stream=None):
    """(col_ptr, row_idx, perm) of the CSC form (int32 device tensors)."""
    m = row_ptr.numel() - 1
    nnz = col_idx.numel()
    dev = row_ptr.device
    col_ptr = torch.empty(n_cols + 1, dtype=torch.int32, device=dev)
    row_idx = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    perm = torch.empty(max(nnz, 1), dtype=torch.int32, device=dev)
    ws_bytes = int(_lib.csr_transpose_workspace(int(n_cols)))
    ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    st = _lib.csr_transpose(col_ptr.data_ptr(), row_idx.data_ptr(), perm.data_ptr(),
                            _vec_arg(row_ptr, "row_ptr"), _vec_arg(col_idx, "col_idx") if nnz else None,
                            m, int(n_cols), nnz, ws.data_ptr(), ws.numel(), _stream(stream))
    _native.check("csr_transpose", st)
    return col_ptr, row_idx[:nnz], perm[:nnz]


def vec_gather(src: torch.Tensor, idx: torch.Tensor, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
    """out[i] = src[idx[i]] (idx int32)."""
    s = storage_of(src)
    n = idx.numel()
    if out is None:
        out = torch.empty(n, dtype=src.dtype, device=src.device)
    st = _lib.vec_gather(_vec_arg(out, "out") if n else None, _vec_arg(src, "src") if src.numel() else None,
                         _vec_arg(idx, "idx") if n else None, n, DTYPES[s], _stream(stream))
    _native.check("vec_gather", st)
    return out


def vec_scale_dev(v: torch.Tensor, alpha: torch.Tensor, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """out = alpha * v with alpha a one-element device tensor (float32; float64
    for FP64 storage)."""
    s = storage_of(v)
    adt = torch.float64 if s == "f64" else torch.float32
    if alpha.dtype != adt or not alpha.is_cuda:
        raise TypeError(f"alpha must be a CUDA {adt} tensor")
    if out is None:
        out = torch.empty_like(v)
    n = v.numel()
    st = _lib.vec_scale_dev(_vec_arg(out, "out") if n else None, _vec_arg(v, "v") if n else None,
                            _dev_ptr(alpha, "alpha"), n, DTYPES[s], _stream(stream))
    _native.check("vec_scale_dev", st)
    return out
