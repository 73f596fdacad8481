"""Seeded synthetic inputs, shared by the tests, the benchmark and the oracle checks.

This module generates inputs only: vectors, dense matrices and sparse matrix
structures with the shapes and value distributions of the workloads (the
paper's vectors of two million entries and 2048x2048 matrix, Sec. 3, scaled
up to a size sweep; Laplacian and power-law CSR matrices).  It computes none of
the operations themselves, and both the oracle and the CUDA path receive the
arrays it returns; neither side regenerates them.

Every generator takes an explicit seed and draws from numpy's PCG64 stream.
Values are drawn in float64 and then rounded to the storage type: numpy's
round-to-nearest-even for float32 / float16, and torch's CPU conversion for
bfloat16 (via float32).
"""
from __future__ import annotations

import math

import numpy as np
import torch

STORAGE = ("f32", "f64", "bf16", "f16")
_TORCH = {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16,
          "f16": torch.float16}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def to_storage(v64: np.ndarray, storage: str) -> torch.Tensor:
    """float64 array -> CPU tensor of the storage type (round to nearest even)."""
    v64 = np.ascontiguousarray(v64, dtype=np.float64)
    if storage == "f64":
        return torch.from_numpy(v64.copy())
    if storage == "f32":
        return torch.from_numpy(v64.astype(np.float32))
    if storage == "f16":
        return torch.from_numpy(v64.astype(np.float16))
    if storage == "bf16":
        return torch.from_numpy(v64.astype(np.float32)).to(torch.bfloat16)
    raise ValueError(storage)


def torch_dtype(storage: str) -> torch.dtype:
    return _TORCH[storage]


# ---- vectors ------------------------------------------------------------------

def uniform(n: int, seed: int, storage: str = "f32", lo: float = -1.0, hi: float = 1.0):
    """n values ~ U(lo, hi)."""
    return to_storage(rng(seed).uniform(lo, hi, size=n), storage)


def normal(shape, seed: int, storage: str = "f32"):
    """values ~ N(0, 1) of the given shape (flattened storage)."""
    size = int(np.prod(shape))
    return to_storage(rng(seed).standard_normal(size), storage).reshape(shape)


def mixed_magnitude(n: int, seed: int, storage: str = "f32", lo_exp: float = -4.0,
                    hi_exp: float = 4.0):
    """Random signs, magnitudes log-uniform in [10^lo_exp, 10^hi_exp]."""
    g = rng(seed)
    mag = 10.0 ** g.uniform(lo_exp, hi_exp, size=n)
    sign = np.where(g.integers(0, 2, size=n) == 0, -1.0, 1.0)
    return to_storage(sign * mag, storage)


def vector_sweep_sizes():
    """n = round(10^(3 + k/3)), k = 0..15: 1,000 ... 100,000,000 (3 per decade)."""
    return [int(round(10 ** (3 + k / 3.0))) for k in range(16)]


def gemv_sweep_sizes():
    """Square GEMV orders 512 ... 16384 (the paper's 2048 among them)."""
    return [512, 1024, 2048, 4096, 8192, 16384]


# ---- sparse structures --------------------------------------------------------

def _csr_from_masked(cols: np.ndarray, mask: np.ndarray, vals: np.ndarray):
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(cols.shape[0] + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return (row_ptr.astype(np.int32), cols[mask].astype(np.int32), vals[mask])


def laplacian_2d(N: int, storage: str = "f64"):
    """5-point Laplacian on an N x N grid, Dirichlet boundary (neighbours
    outside the grid dropped), rows in lexicographic order with i fastest,
    4 on the diagonal and -1 per existing neighbour, columns sorted per row.
    Returns (row_ptr int32, col_idx int32, vals tensor of the storage type)."""
    p = np.arange(N * N, dtype=np.int64)
    i, j = p % N, p // N
    offs = np.array([-N, -1, 0, 1, N], dtype=np.int64)        # ascending columns
    cols = p[:, None] + offs[None, :]
    mask = np.stack([j > 0, i > 0, np.ones_like(i, bool), i < N - 1, j < N - 1], axis=1)
    vals = np.where(offs[None, :] == 0, 4.0, -1.0) * np.ones_like(cols, dtype=np.float64)
    rp, ci, v = _csr_from_masked(cols, mask, vals)
    return torch.from_numpy(rp), torch.from_numpy(ci), to_storage(v, storage)


def laplacian_3d(N: int, storage: str = "f64"):
    """7-point Laplacian on an N^3 grid, Dirichlet, 6 on the diagonal and -1
    per existing neighbour; rows lexicographic (i fastest), columns sorted."""
    p = np.arange(N ** 3, dtype=np.int64)
    i, j, k = p % N, (p // N) % N, p // (N * N)
    offs = np.array([-N * N, -N, -1, 0, 1, N, N * N], dtype=np.int64)
    cols = p[:, None] + offs[None, :]
    one = np.ones_like(i, bool)
    mask = np.stack([k > 0, j > 0, i > 0, one, i < N - 1, j < N - 1, k < N - 1], axis=1)
    vals = np.where(offs[None, :] == 0, 6.0, -1.0) * np.ones_like(cols, dtype=np.float64)
    rp, ci, v = _csr_from_masked(cols, mask, vals)
    return torch.from_numpy(rp), torch.from_numpy(ci), to_storage(v, storage)


def powerlaw_exponent(kmin: int = 4, kmax: int = 256, mean: float = 16.0) -> float:
    """Exponent a of P(k) ~ k^-a on [kmin, kmax] whose mean is `mean` (bisection)."""
    k = np.arange(kmin, kmax + 1, dtype=np.float64)

    def m(a):
        w = k ** (-a)
        return float((k * w).sum() / w.sum())

    lo, hi = 0.0, 6.0                      # m(0) = 130 > mean > m(6)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if m(mid) > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _distinct_sorted_cols(g, row_len: np.ndarray, n: int, lo=None, width=None):
    """Distinct, sorted random columns per row, uniform in [lo_r, lo_r + width_r)
    (default [0, n)).  Duplicates inside a row are redrawn until none remain."""
    m = row_len.size
    nnz = int(row_len.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), row_len)
    if lo is None:
        lo_e = np.zeros(nnz, np.int64)
        w_e = np.full(nnz, n, np.int64)
    else:
        lo_e = np.repeat(lo.astype(np.int64), row_len)
        w_e = np.repeat(width.astype(np.int64), row_len)
    cols = lo_e + (g.random(nnz) * w_e).astype(np.int64)
    span = np.int64(n)
    while True:
        key = rows * span + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        cols = cols[order]
        lo_e = lo_e[order]
        w_e = w_e[order]
        dup = np.zeros(nnz, bool)
        dup[1:] = key[1:] == key[:-1]
        nd = int(dup.sum())
        if nd == 0:
            break
        cols[dup] = lo_e[dup] + (g.random(nd) * w_e[dup]).astype(np.int64)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(row_len, out=row_ptr[1:])
    return row_ptr.astype(np.int32), cols.astype(np.int32)


def powerlaw_csr(m: int, n: int, seed: int, storage: str = "f32", kmin: int = 4,
                 kmax: int = 256, mean: float = 16.0):
    """Random CSR: row length k in [kmin, kmax] drawn i.i.d. from P(k) ~ k^-a
    (a fitted so E[k] = mean), distinct uniform columns sorted per row,
    values ~ N(0, 1).  Rows are in draw order (not sorted by length)."""
    g = rng(seed)
    a = powerlaw_exponent(kmin, kmax, mean)
    k = np.arange(kmin, kmax + 1)
    p = k.astype(np.float64) ** (-a)
    p /= p.sum()
    row_len = g.choice(k, size=m, p=p).astype(np.int64)
    rp, ci = _distinct_sorted_cols(g, row_len, n)
    vals = g.standard_normal(int(row_len.sum()))
    return torch.from_numpy(rp), torch.from_numpy(ci), to_storage(vals, storage)


def random_csr(m: int, n: int, seed: int, storage: str = "f64", min_len: int = 0,
               max_len: int = 8, empty_frac: float = 0.0, duplicates: bool = False):
    """Small random CSR for parity and pin tests: row lengths uniform in
    [min_len, max_len], a fraction of rows forced empty, optional repeated
    columns within a row, values ~ N(0, 1)."""
    g = rng(seed)
    row_len = g.integers(min_len, max_len + 1, size=m).astype(np.int64)
    if empty_frac > 0:
        row_len[g.random(m) < empty_frac] = 0
    if not duplicates:
        row_len = np.minimum(row_len, n)
        rp, ci = _distinct_sorted_cols(g, row_len, n)
    else:
        rp = np.zeros(m + 1, np.int64)
        np.cumsum(row_len, out=rp[1:])
        ci = g.integers(0, max(n, 1), size=int(row_len.sum()))
        rp, ci = rp.astype(np.int32), ci.astype(np.int32)
    vals = g.standard_normal(int(rp[-1]))
    return torch.from_numpy(rp), torch.from_numpy(ci), to_storage(vals, storage)


def banded_random_csr(m: int, seed: int, min_len: int = 5, max_len: int = 64,
                      storage: str = "f32"):
    """Square m x m CSR with row lengths uniform in [min_len, max_len] and
    distinct random columns anywhere in the block (batched-CSR instances)."""
    g = rng(seed)
    row_len = np.minimum(g.integers(min_len, max_len + 1, size=m), m).astype(np.int64)
    rp, ci = _distinct_sorted_cols(g, row_len, m)
    vals = g.standard_normal(int(row_len.sum()))
    return torch.from_numpy(rp), torch.from_numpy(ci), to_storage(vals, storage)


def log_uniform_ints(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integers with log-uniform distribution on [lo, hi] (batched instance sizes)."""
    g = rng(seed)
    v = np.exp(g.uniform(math.log(lo), math.log(hi + 1), size=count))
    return np.clip(np.floor(v).astype(np.int64), lo, hi)


# ---- device-side generation (large benchmark inputs) -----------------------------
#
# The full-size sweep needs ~16 GB of inputs; drawing them on the host would
# dominate the benchmark's set-up time.  These draw the same distributions on
# the GPU with torch's counter-based Philox generator, seeded explicitly.

def device_uniform_(out: torch.Tensor, seed: int, lo: float = -1.0, hi: float = 1.0):
    """Fill `out` in place with U(lo, hi) values (Philox, seeded)."""
    g = torch.Generator(device=out.device).manual_seed(seed)
    if out.dtype in (torch.float32, torch.float64):
        out.uniform_(lo, hi, generator=g)
    else:
        tmp = torch.empty(out.shape, dtype=torch.float32, device=out.device)
        tmp.uniform_(lo, hi, generator=g)
        out.copy_(tmp)
    return out


def device_normal_(out: torch.Tensor, seed: int):
    """Fill `out` in place with N(0, 1) values (Philox, seeded)."""
    g = torch.Generator(device=out.device).manual_seed(seed)
    if out.dtype in (torch.float32, torch.float64):
        out.normal_(0.0, 1.0, generator=g)
    else:
        tmp = torch.empty(out.shape, dtype=torch.float32, device=out.device)
        tmp.normal_(0.0, 1.0, generator=g)
        out.copy_(tmp)
    return out


def device_mixed_magnitude_(out: torch.Tensor, seed: int, lo_exp: float = -4.0,
                            hi_exp: float = 4.0):
    """Fill `out` in place with random signs and magnitudes log-uniform in
    [10^lo_exp, 10^hi_exp] (Philox, seeded)."""
    g = torch.Generator(device=out.device).manual_seed(seed)
    e = torch.empty(out.shape, dtype=torch.float64, device=out.device).uniform_(lo_exp, hi_exp,
                                                                                  generator=g)
    sign = torch.randint(0, 2, out.shape, generator=g, device=out.device).to(torch.float64) * 2 - 1
    out.copy_(sign * torch.pow(10.0, e))
    return out


def device_csr_block_(m: int, seed: int, min_len: int, max_len: int, dtype, device):
    """A square m x m CSR block generated on the device: row lengths uniform in
    [min_len, max_len], columns uniform in [0, m) (unsorted, repeats allowed --
    CSR sums them), values N(0, 1).  Returns (row_ptr int32, col_idx int32, vals)."""
    g = torch.Generator(device=device).manual_seed(seed)
    lens = torch.randint(min_len, max_len + 1, (m,), generator=g, device=device, dtype=torch.int32)
    rp = torch.zeros(m + 1, dtype=torch.int32, device=device)
    torch.cumsum(lens, 0, out=rp[1:])
    nnz = int(rp[-1].item())
    ci = torch.randint(0, m, (nnz,), generator=g, device=device, dtype=torch.int32)
    v = torch.empty(nnz, dtype=torch.float32, device=device).normal_(0.0, 1.0, generator=g)
    return rp, ci, v.to(dtype)


def batch_workload(device, count: int = 4096, seed: int = 4000, dtype=torch.float32,
                   families=("vec", "gemv", "csr")):
    """The batching workload's instances, drawn on the device: `count` uneven
    instances per family.
      vectors: n log-uniform in [256, 1,048,576]; y, z ~ U(-1, 1), x zeroed
        (slices of three flat buffers, each slice starting on a 64-element
        boundary);
      dense GEMV: m, n independently log-uniform in [64, 4096], A ~ N(0, 1)
        row-major, x ~ U(-1, 1), y zeroed;
      CSR: square blocks of m log-uniform in [1,000, 200,000] rows with 5..64
        entries per row (device_csr_block_), x ~ U(-1, 1), y zeroed.
    Returns {"vec": [(y, z, x)], "gemv": [(A, x, y)], "csr": [((rp, ci, v, m), x, y)]},
    with only the requested families drawn (each family's draws do not depend
    on which others are requested)."""
    out = {}
    if "vec" in families:
        out["vec"] = _batch_vectors(device, count, seed, dtype)
    if "gemv" in families:
        out["gemv"] = _batch_gemv(device, count, seed, dtype)
    if "csr" in families:
        out["csr"] = _batch_csr(device, count, seed, dtype)
    return out


def _batch_vectors(device, count, seed, dtype):
    ns = log_uniform_ints(count, 256, 1_048_576, seed)
    buf_len = int(sum((int(n) + 63) // 64 * 64 for n in ns))
    ybuf = device_uniform_(torch.empty(buf_len, dtype=dtype, device=device), seed + 1)
    zbuf = device_uniform_(torch.empty(buf_len, dtype=dtype, device=device), seed + 2)
    xbuf = torch.zeros(buf_len, dtype=dtype, device=device)
    vec, o = [], 0
    for n in ns:
        n = int(n)
        vec.append((ybuf[o:o + n], zbuf[o:o + n], xbuf[o:o + n]))
        o += (n + 63) // 64 * 64
    return vec


def _batch_gemv(device, count, seed, dtype):
    ms = log_uniform_ints(count, 64, 4096, seed + 3)
    nn = log_uniform_ints(count, 64, 4096, seed + 4)
    gemv = []
    for i, (m, n) in enumerate(zip(ms, nn)):
        m, n = int(m), int(n)
        gemv.append((device_normal_(torch.empty(m, n, dtype=dtype, device=device), seed + 10 + i),
                     device_uniform_(torch.empty(n, dtype=dtype, device=device), seed + 20000 + i),
                     torch.zeros(m, dtype=dtype, device=device)))
    return gemv


def _batch_csr(device, count, seed, dtype):
    rows = log_uniform_ints(count, 1000, 200_000, seed + 5)
    csr = []
    for i, m in enumerate(rows):
        m = int(m)
        rp, ci, v = device_csr_block_(m, seed + 40000 + i, 5, 64, dtype, device)
        csr.append(((rp, ci, v, m),
                    device_uniform_(torch.empty(m, dtype=dtype, device=device), seed + 60000 + i),
                    torch.zeros(m, dtype=dtype, device=device)))
    return csr
