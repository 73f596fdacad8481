"""Pins for the FP64 oracle: each check ties one oracle routine to something
other than the oracle itself -- a closed form, an invariant, exact rational
arithmetic (fractions.Fraction), a library routine (numpy, math.fsum, torch's
CPU conversions, scipy), brute force on tiny inputs, or a hand-worked fixture.

The checks are plain functions so that the mutation test can run the same set
against deliberately broken builds of the oracle (every planted mistake must
make at least one of them fail).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import torch

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _frac_round(fr: Fraction) -> float:
    return float(fr)                       # Fraction -> float is correctly rounded


def _ulp(v: float) -> float:
    return math.ulp(v) if v != 0 else math.ulp(0.0)


def _load_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, vals = line.split(":", 1)
            out[key.strip()] = [float(t) for t in vals.split()]
    return out


# ---- vector update (Sec. 2) ---------------------------------------------------

def pin_copy_identity():
    y = synth.uniform(1001, 3, "f64").numpy()
    assert np.array_equal(oracle.copy(y), y)


def pin_axpy_half_alpha_single_rounding():
    # alpha = 0.5 makes alpha*z exact in binary32, so y + 0.5 z rounded once
    # to binary32 equals numpy's correctly rounded float32 addition.
    y = synth.uniform(100_003, 1, "f32").numpy()
    z = synth.uniform(100_003, 2, "f32").numpy()
    got = oracle.round_f32(oracle.axpy(y, z, 0.5))
    ref = y + np.float32(0.5) * z
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def pin_axpy_special_cases():
    y = synth.uniform(4097, 4, "f64").numpy()
    z = synth.uniform(4097, 5, "f64").numpy()
    assert np.array_equal(oracle.axpy(y, z, 0.0), y)                 # alpha = 0
    zero = np.zeros_like(y)
    assert np.array_equal(oracle.axpy(zero, z, -1.75), -1.75 * z)     # y = 0
    assert np.array_equal(oracle.axpy(y, y, -1.0), zero)              # y - y


def pin_axpy_exact_rational():
    g = synth.rng(6)
    y = g.standard_normal(300) * 10.0 ** g.integers(-8, 8, 300)
    z = g.standard_normal(300) * 10.0 ** g.integers(-8, 8, 300)
    alpha = 2.0 ** -3                       # alpha*z exact: one rounding in the sum
    got = oracle.axpy(y, z, alpha)
    for i in range(y.size):
        ref = _frac_round(Fraction(y[i]) + Fraction(alpha) * Fraction(z[i]))
        assert got[i] == ref, (i, got[i], ref)


def pin_axpby_exact_rational():
    g = synth.rng(7)
    y = g.standard_normal(200)
    z = g.standard_normal(200)
    got = oracle.axpby(2.0, y, -0.5, z)     # both scalings exact
    for i in range(y.size):
        ref = _frac_round(2 * Fraction(y[i]) - Fraction(z[i]) / 2)
        assert got[i] == ref


# ---- inner product (Sec. 2) ----------------------------------------------------

def pin_dot_ones():
    n = 1_000_003
    assert oracle.dot(np.ones(n), np.ones(n)) == float(n)
    assert oracle.dot(np.ones(0), np.ones(0)) == 0.0


def pin_dot_arange_closed_forms():
    n = 100_000
    a = np.arange(1, n + 1, dtype=np.float64)
    assert oracle.dot(a, np.ones(n)) == n * (n + 1) / 2
    assert oracle.dot(a, a) == n * (n + 1) * (2 * n + 1) / 6        # < 2^53, exact
    assert oracle.dot(a, -np.ones(n)) == -(n * (n + 1) / 2)


def pin_dot_alternating_and_unit():
    s = np.where(np.arange(10_001) % 2 == 0, 1.0, -1.0)
    assert oracle.dot(s, np.ones(s.size)) == 1.0
    assert oracle.dot(s[:-1], np.ones(s.size - 1)) == 0.0
    x = synth.uniform(999, 8, "f64").numpy()
    for k in (0, 17, 998):
        e = np.zeros(999)
        e[k] = 1.0
        assert oracle.dot(x, e) == x[k]
        assert oracle.dot(e, x) == x[k]


def pin_dot_fsum_f32():
    for n, seed in ((1, 9), (3, 10), (17, 11), (1000, 12), (4099, 13)):
        x = synth.uniform(n, seed, "f32").numpy().astype(np.float64)
        y = synth.uniform(n, seed + 100, "f32").numpy().astype(np.float64)
        prods = x * y                        # exact: 24 + 24 bits <= 53
        assert oracle.dot(x, y) == math.fsum(prods)


def pin_dot_cancellation():
    big = 2.0 ** 60
    # a lost TwoSum remainder returns 0 here
    assert oracle.dot([big, 1.0, -big, 2.0 ** -30], [1.0, 1.0, 1.0, 1.0]) == 1.0 + 2.0 ** -30
    # a lost TwoProduct remainder returns 0 here: (1+2^-30)^2 - (1+2^-29) = 2^-60
    a = 1.0 + 2.0 ** -30
    assert oracle.dot([a, -1.0], [a, 1.0 + 2.0 ** -29]) == 2.0 ** -60


def pin_dot_fraction_random():
    g = synth.rng(14)
    for n in (2, 5, 33, 200):
        x = g.standard_normal(n) * 10.0 ** g.integers(-5, 5, n)
        y = g.standard_normal(n) * 10.0 ** g.integers(-5, 5, n)
        exact = sum(Fraction(a) * Fraction(b) for a, b in zip(x, y))
        hi, lo = oracle.dot(x, y, with_lo=True)
        assert hi == _frac_round(exact)
        assert abs(Fraction(hi) + Fraction(lo) - exact) <= abs(exact) * Fraction(2) ** -100


def pin_sparse_dot_fraction_and_closed_forms():
    """Sparse inner product: exact rational brute force (correctly rounded
    result), repeated indices, the ones/arange closed form, and the empty sum."""
    g = synth.rng(15)
    for nnz, n in ((1, 3), (7, 5), (64, 1000), (300, 40)):
        v = g.standard_normal(nnz) * 10.0 ** g.integers(-4, 4, nnz)
        y = g.standard_normal(n) * 10.0 ** g.integers(-4, 4, n)
        c = g.integers(0, n, nnz).astype(np.int32)        # repeats allowed
        exact = sum(Fraction(v[k]) * Fraction(y[c[k]]) for k in range(nnz))
        assert oracle.sparse_dot(v, c, y) == _frac_round(exact)
    # ones against arange: sum of the indices themselves
    c = np.array([5, 0, 5, 3, 9, 9, 9], dtype=np.int32)
    assert oracle.sparse_dot(np.ones(7), c, np.arange(10.0)) == 40.0
    # first and last stored entries both count
    assert oracle.sparse_dot(np.array([2.0, 0.0, 3.0]), np.array([1, 0, 2], np.int32),
                             np.array([0.0, 7.0, 11.0])) == 47.0
    assert oracle.sparse_dot(np.zeros(0), np.zeros(0, np.int32), np.ones(4)) == 0.0


def pin_sparse_dot_is_a_csr_row():
    """Each entry of a CSR product (brute-force dense product) is the sparse
    inner product of that row's stored entries with x."""
    rp, ci, v = synth.random_csr(40, 25, 16, "f64", 0, 9, 0.1, True)
    rp, ci, v = rp.numpy(), ci.numpy(), v.numpy()
    x = synth.uniform(25, 17, "f64").numpy()
    dense = np.zeros((40, 25))
    for i in range(40):
        for k in range(rp[i], rp[i + 1]):
            dense[i, ci[k]] += v[k]
    for i in range(40):
        a, b = rp[i], rp[i + 1]
        exact = sum(Fraction(dense[i, j]) * Fraction(x[j]) for j in range(25)) \
            if len(set(ci[a:b])) == b - a else \
            sum(Fraction(v[k]) * Fraction(x[ci[k]]) for k in range(a, b))
        assert oracle.sparse_dot(v[a:b], ci[a:b], x) == _frac_round(exact)


# ---- dense matrix-vector product (Sec. 2) -----------------------------------------

def pin_gemv_identity_and_single_entry():
    n = 37
    x = synth.uniform(n, 15, "f64").numpy()
    eye = np.eye(n)
    assert np.array_equal(oracle.gemv(eye.ravel(), x, n, n, n, "row"), x)
    assert np.array_equal(oracle.gemv(eye.ravel(), x, n, n, n, "col"), x)
    m, n2 = 5, 9
    xv = synth.uniform(n2, 16, "f64").numpy()
    for (i, j) in ((0, 0), (4, 8), (2, 3)):
        A = np.zeros((m, n2))
        A[i, j] = 1.0
        yr = oracle.gemv(A.ravel(), xv, m, n2, n2, "row")
        yc = oracle.gemv(A.T.ravel(), xv, m, n2, m, "col")
        ref = np.zeros(m)
        ref[i] = xv[j]
        assert np.array_equal(yr, ref) and np.array_equal(yc, ref)


def pin_gemv_exact_tiny():
    g = synth.rng(17)
    for m in (1, 2, 3, 7):
        for n in (1, 4, 6, 13):
            lda = n + 3
            A = np.full((m, lda), np.nan)
            A[:, :n] = g.standard_normal((m, n))
            x = g.standard_normal(n)
            y = oracle.gemv(A.ravel(), x, m, n, lda, "row")
            # column-major storage of the same matrix with padding rows
            C = np.full((n, m + 2), np.nan)
            C[:, :m] = A[:, :n].T
            yc = oracle.gemv(C.ravel(), x, m, n, m + 2, "col")
            for i in range(m):
                ref = _frac_round(sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(n)))
                assert y[i] == ref and yc[i] == ref


def pin_gemv_numpy():
    m, n = 61, 45
    A = synth.normal((m, n), 18, "f64").numpy()
    x = synth.uniform(n, 19, "f64").numpy()
    ref = A @ x
    scale = np.abs(A) @ np.abs(x)
    assert np.all(np.abs(oracle.gemv(A.ravel(), x, m, n, n, "row") - ref) <= 1e-13 * scale)
    assert np.all(np.abs(oracle.gemv(np.asfortranarray(A).ravel(order="K"), x, m, n, m, "col")
                         - ref) <= 1e-13 * scale)


def pin_gemv_linearity_and_entries():
    m, n = 33, 29
    A = synth.normal((m, n), 20, "f64").numpy().ravel()
    x1 = synth.uniform(n, 21, "f64").numpy()
    x2 = synth.uniform(n, 22, "f64").numpy()
    lhs = oracle.gemv(A, 2.0 * x1 - 0.5 * x2, m, n, n)
    rhs = 2.0 * oracle.gemv(A, x1, m, n, n) - 0.5 * oracle.gemv(A, x2, m, n, n)
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-13 * n)
    rows = [0, 5, 32]
    assert np.array_equal(oracle.gemv_entries(A, x1, rows, n, n), oracle.gemv(A, x1, m, n, n)[rows])


# ---- CSR sparse matrix-vector product -----------------------------------------------

def pin_spmv_golden():
    gd = _load_golden("laplace2d_3x3.txt")
    rp = np.array(gd["row_ptr"], np.int32)
    ci = np.array(gd["col_idx"], np.int32)
    v = np.array(gd["vals"])
    assert np.array_equal(oracle.csr_spmv(rp, ci, v, np.ones(9)), gd["A_times_ones"])
    assert np.array_equal(oracle.csr_spmv(rp, ci, v, gd["x"]), gd["A_times_x"])
    grp, gci, gv = synth.laplacian_2d(3)
    assert np.array_equal(grp.numpy(), rp) and np.array_equal(gci.numpy(), ci)
    assert np.array_equal(gv.numpy(), v)


def pin_spmv_laplacian_ones():
    N = 256
    rp, ci, v = synth.laplacian_2d(N)
    y = oracle.csr_spmv(rp, ci, v, np.ones(N * N)).reshape(N, N)
    assert np.all(y[1:-1, 1:-1] == 0.0)
    assert y[0, 0] == y[0, -1] == y[-1, 0] == y[-1, -1] == 2.0
    assert np.all(y[0, 1:-1] == 1.0) and np.all(y[1:-1, 0] == 1.0)
    assert y.sum() == 4 * N
    N3 = 24
    rp, ci, v = synth.laplacian_3d(N3)
    y3 = oracle.csr_spmv(rp, ci, v, np.ones(N3 ** 3))
    assert y3.sum() == 6 * N3 * N3


def _eig2(N, p, q):
    i = np.arange(1, N + 1)
    sx = np.sin(p * np.pi * i / (N + 1))
    sy = np.sin(q * np.pi * i / (N + 1))
    x = (sy[:, None] * sx[None, :]).ravel()          # row index = i + N*j, i fastest
    lam = 4 - 2 * np.cos(p * np.pi / (N + 1)) - 2 * np.cos(q * np.pi / (N + 1))
    return x, lam


def pin_spmv_eigen_2d():
    N = 64
    rp, ci, v = synth.laplacian_2d(N)
    for p, q in ((1, 1), (3, 5), (64, 2)):
        x, lam = _eig2(N, p, q)
        y = oracle.csr_spmv(rp, ci, v, x)
        assert np.max(np.abs(y - lam * x)) <= 1e-13


def pin_spmv_eigen_3d():
    N = 20
    rp, ci, v = synth.laplacian_3d(N)
    i = np.arange(1, N + 1)
    p, q, r = 2, 3, 7
    sx = np.sin(p * np.pi * i / (N + 1))
    sy = np.sin(q * np.pi * i / (N + 1))
    sz = np.sin(r * np.pi * i / (N + 1))
    x = (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]).ravel()
    lam = 6 - 2 * (np.cos(p * np.pi / (N + 1)) + np.cos(q * np.pi / (N + 1))
                   + np.cos(r * np.pi / (N + 1)))
    y = oracle.csr_spmv(rp, ci, v, x)
    assert np.max(np.abs(y - lam * x)) <= 1e-13


def pin_spmv_dense_bruteforce():
    m, n = 23, 17
    rp, ci, v = synth.random_csr(m, n, 23, "f64", min_len=0, max_len=9, empty_frac=0.25,
                                 duplicates=True)
    rp, ci, v = rp.numpy(), ci.numpy(), v.numpy()
    assert np.any(np.diff(rp) == 0)
    dense = [[Fraction(0)] * n for _ in range(m)]
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            dense[i][ci[k]] += Fraction(v[k])
    x = synth.uniform(n, 24, "f64").numpy()
    y = oracle.csr_spmv(rp, ci, v, x)
    for i in range(m):
        ref = _frac_round(sum(dense[i][j] * Fraction(x[j]) for j in range(n)))
        assert y[i] == ref


def pin_spmv_rows():
    rp, ci, v = synth.powerlaw_csr(3000, 2500, 25, "f64")
    x = synth.uniform(2500, 26, "f64").numpy()
    y = oracle.csr_spmv(rp, ci, v, x)
    rows = [0, 1, 1234, 2999]
    assert np.array_equal(oracle.csr_rows(rp, ci, v, x, rows), y[rows])
    sp = _scipy_sparse()
    if sp is not None:
        A = sp.csr_matrix((v.numpy(), ci.numpy(), rp.numpy()), shape=(3000, 2500))
        ref = A @ x
        scale = abs(A) @ np.abs(x)
        assert np.all(np.abs(y - ref) <= 1e-13 * scale)


def _scipy_sparse():
    try:
        import scipy.sparse as sp
        return sp
    except ImportError:
        return None


def pin_csc_transpose():
    m, n = 41, 29
    rp, ci, v = synth.random_csr(m, n, 27, "f64", min_len=0, max_len=7, empty_frac=0.2)
    rp, ci, v = rp.numpy(), ci.numpy(), v.numpy()
    cp, ri, perm = oracle.csr_to_csc(rp, ci, n)
    # brute force: walk the dense pattern column by column
    pattern = {}
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            pattern.setdefault(int(ci[k]), []).append((i, k))
    q = 0
    for j in range(n):
        ents = sorted(pattern.get(j, []))
        assert cp[j] == q and cp[j + 1] == q + len(ents)
        for (i, k) in ents:
            assert ri[q] == i and perm[q] == k
            q += 1
    # A^T x through the CSC arrays equals the dense transpose product
    D = np.zeros((m, n))
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            D[i, ci[k]] += v[k]
    w = synth.uniform(m, 28, "f64").numpy()
    got = oracle.csr_spmv(cp, ri, v[perm], w)
    assert np.allclose(got, D.T @ w, rtol=0, atol=1e-14 * m)
    sp = _scipy_sparse()
    if sp is not None:
        C = sp.csr_matrix((v, ci, rp), shape=(m, n)).tocsc()
        C.sort_indices()
        assert np.array_equal(C.indptr, cp) and np.array_equal(C.indices, ri)
        assert np.array_equal(C.data, v[perm])


# ---- SELL-C-sigma --------------------------------------------------------------------

def pin_sell_layout_bruteforce():
    m, n = 203, 150
    rp, ci, v = synth.random_csr(m, n, 40, "f64", 0, 12, 0.15, True)
    rp, ci = rp.numpy(), ci.numpy()
    lens = np.diff(rp)
    for sigma in (1, 32, 64, 256):
        perm, slen, sptr, cols, mp = oracle.csr_to_sell(rp, ci, 32, sigma)
        mpad = (m + 31) // 32 * 32
        assert perm.size == mpad
        assert sorted(int(p) for p in perm if p >= 0) == list(range(m))
        assert np.all(perm[m:] == -1) if sigma == 1 else np.sum(perm < 0) == mpad - m
        win = max(sigma, 1)
        for w0 in range(0, mpad, win):
            blk = perm[w0:w0 + win]
            assert set(int(p) for p in blk if p >= 0) == set(range(w0, min(w0 + win, m)))
            if sigma > 1:
                key = [(-lens[p], p) if p >= 0 else (1, 10 ** 9 + q) for q, p in enumerate(blk)]
                assert key == sorted(key)
        total = 0
        for s_ in range(mpad // 32):
            L = max([lens[p] if p >= 0 else 0 for p in perm[32 * s_:32 * s_ + 32]])
            assert slen[s_] == L and sptr[s_] == total
            total += 32 * L
            for r in range(32):
                i = perm[32 * s_ + r]
                li = lens[i] if i >= 0 else 0
                for j in range(L):
                    slot = sptr[s_] + 32 * j + r
                    if j < li:
                        assert cols[slot] == ci[rp[i] + j] and mp[slot] == rp[i] + j
                    else:
                        assert cols[slot] == -1 and mp[slot] == -1
        assert sptr[-1] == total == cols.size


def pin_sell_spmv_matches_csr_and_eigen():
    for (rp, ci, v), n in ((synth.random_csr(500, 300, 41, "f64", 0, 20, 0.1, True), 300),
                           (synth.powerlaw_csr(2000, 1500, 42, "f64"), 1500)):
        x = synth.uniform(n, 43, "f64").numpy()
        ref = oracle.csr_spmv(rp, ci, v, x)
        for sigma in (1, 128):
            perm, slen, sptr, cols, mp = oracle.csr_to_sell(rp, ci, 32, sigma)
            sv = np.where(mp >= 0, v.numpy()[np.maximum(mp, 0)], 0.0)
            y = oracle.sell_spmv(perm, slen, sptr, cols, sv, x, rp.numel() - 1)
            assert np.array_equal(y, ref)             # same entries, same order per row
    N = 30
    rp, ci, v = synth.laplacian_2d(N)
    x, lam = _eig2(N, 2, 9)
    perm, slen, sptr, cols, mp = oracle.csr_to_sell(rp, ci, 32, 64)
    sv = np.where(mp >= 0, v.numpy()[np.maximum(mp, 0)], 0.0)
    y = oracle.sell_spmv(perm, slen, sptr, cols, sv, x, N * N)
    assert np.max(np.abs(y - lam * x)) <= 1e-13


# ---- derivatives --------------------------------------------------------------------

def pin_csr_row_bins_bruteforce():
    """Row-binned CSR layout against an independent statement of the rule: bin =
    ceil(log2(L / per_lane)) clipped to [0, nbins-1] (exact integer form), rows
    listed bin by bin in increasing index -- checked as a permutation, per-bin
    length bounds, stability and counts, on patterns with empty rows and rows
    at every bin edge."""
    for seed, per_lane, nbins in ((60, 8, 7), (61, 4, 7), (62, 8, 3), (63, 1, 2)):
        g = synth.rng(seed)
        lens = list(g.integers(0, 300, 400))
        edges = [0, per_lane, per_lane + 1] + [per_lane << k for k in range(nbins)] + \
                [(per_lane << k) + 1 for k in range(nbins)]
        lens = edges + lens
        rp = np.zeros(len(lens) + 1, np.int64)
        rp[1:] = np.cumsum(lens)
        perm, bptr = oracle.csr_row_bins(rp.astype(np.int32), per_lane, nbins)

        def bin_of(L):
            b = 0
            while per_lane * (1 << b) < L:          # smallest b with L <= per_lane * 2^b
                b += 1
            return min(b, nbins - 1)
        want = sorted(range(len(lens)), key=lambda i: (bin_of(lens[i]), i))
        assert list(perm) == want
        assert sorted(perm) == list(range(len(lens)))
        for b in range(nbins):
            rows = perm[bptr[b]:bptr[b + 1]]
            assert list(rows) == sorted(rows)
            assert all(bin_of(lens[r]) == b for r in rows)
        assert bptr[0] == 0 and bptr[nbins] == len(lens)
    # degenerate: no rows
    perm, bptr = oracle.csr_row_bins(np.zeros(1, np.int32), 8, 7)
    assert perm.size == 0 and list(bptr) == [0] * 8


def pin_dense_outer_fd():
    # L(A) = <w, A x>  =>  dL/dA = w x^T; central differences are exact up to
    # rounding for a linear map.
    m, n = 6, 5
    A = synth.normal((m, n), 29, "f64").numpy()
    x = synth.uniform(n, 30, "f64").numpy()
    w = synth.uniform(m, 31, "f64").numpy()
    G = oracle.dense_outer(w, x)
    assert G.shape == (m, n)
    for i in range(m):
        for j in range(n):
            h = 1e-6 * max(1.0, abs(A[i, j]))
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h
            Am[i, j] -= h
            lp = oracle.dot(w, oracle.gemv(Ap.ravel(), x, m, n, n))
            lm = oracle.dot(w, oracle.gemv(Am.ravel(), x, m, n, n))
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[i, j]) <= 1e-6 * max(1.0, abs(G[i, j]))
    assert np.array_equal(G, np.outer(w, x))


def pin_sampled_outer_fd():
    m = n = 30
    rp, ci, v = synth.random_csr(m, n, 32, "f64", min_len=0, max_len=6, empty_frac=0.1)
    rp, ci, v = rp.numpy(), ci.numpy(), v.numpy()
    x = synth.uniform(n, 33, "f64").numpy()
    w = synth.uniform(m, 34, "f64").numpy()
    G = oracle.sampled_outer(rp, ci, w, x)
    for k in range(0, v.size, max(1, v.size // 25)):
        h = 1e-6 * max(1.0, abs(v[k]))
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        fd = (oracle.dot(w, oracle.csr_spmv(rp, ci, vp, x))
              - oracle.dot(w, oracle.csr_spmv(rp, ci, vm, x))) / (2 * h)
        assert abs(fd - G[k]) <= 1e-6 * max(1.0, abs(G[k]))


def pin_scale_dot_gradient():
    n = 50
    x = synth.uniform(n, 35, "f64").numpy()
    y = synth.uniform(n, 36, "f64").numpy()
    ds = 1.75
    gx = oracle.scale(y, ds)                # d(ds * <x, y>)/dx = ds * y
    for i in (0, 13, 49):
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        fd = ds * (oracle.dot(xp, y) - oracle.dot(xm, y)) / (2 * h)
        assert abs(fd - gx[i]) <= 1e-7
    assert np.array_equal(gx, ds * y)


# ---- storage rounding --------------------------------------------------------------

def _bf16_cases():
    g = synth.rng(37)
    rnd = (g.standard_normal(20000) * 10.0 ** g.integers(-40, 38, 20000)).astype(np.float32)
    bits = g.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32)
    ties = (bits & np.uint32(0xFFFF0000)) | np.uint32(0x8000)       # exact half-way
    special = np.array([0.0, -0.0, np.inf, -np.inf, 3.3895314e38, 1e-45, -1e-45,
                        1.17549435e-38, 65504.0, 1.0, -1.0], np.float32)
    vals = np.concatenate([rnd, bits.view(np.float32), ties.view(np.float32), special])
    return vals[np.isfinite(vals) | np.isinf(vals)]


def pin_round_bf16():
    v = _bf16_cases()
    got = oracle.round_bf16(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    nan = np.isnan(v)
    assert np.array_equal(got[~nan], ref[~nan])
    w = oracle.widen_bf16_bits(got)
    assert np.all(np.isnan(w[nan]))
    assert np.array_equal(w[~nan], torch.from_numpy(ref[~nan].view(np.int16)).view(
        torch.bfloat16).to(torch.float64).numpy())


def _bf16_nearest_bits(v: float) -> int:
    """Correctly rounded BF16 (nearest, ties to even) of a finite double, by
    exact rational arithmetic on the BF16 grid: 8 significant bits, exponents
    down to -126, subnormal spacing 2^-133, overflow to infinity at and above
    (2 - 2^-8) * 2^127."""
    from fractions import Fraction
    sign = 0x8000 if math.copysign(1.0, v) < 0 else 0
    a = Fraction(abs(v))
    if a >= Fraction(2 ** 9 - 1, 2 ** 8) * 2 ** 127:
        return sign | 0x7F80
    if a == 0:
        return sign
    e = math.floor(math.log2(abs(v)))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = Fraction(2) ** (max(e, -126) - 7)
    k = a / q
    lo = math.floor(k)
    rem = k - lo
    r = lo + 1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and lo % 2 == 1) else lo
    h = r * q
    if h < Fraction(2) ** -126:
        return sign | r
    he = max(e, -126)
    if h >= Fraction(2) ** (he + 1):                   # carried into the next binade
        he += 1
        r //= 2
    return sign | ((he + 127) << 7) | (r - 128)


def pin_round_bf16_f64():
    """Direct FP64 -> BF16 rounding: equals torch's conversion on FP32 values
    (one rounding either way), equals an exact rational rounding on random
    doubles, and differs from rounding through FP32 where that route lands on a
    BF16 midpoint (1 + 2^-8 + 2^-40 must go up to 1 + 2^-7)."""
    f32 = _bf16_cases()
    f32 = f32[~np.isnan(f32)]
    assert np.array_equal(oracle.round_bf16_f64(f32.astype(np.float64)), oracle.round_bf16(f32))
    g = synth.rng(41)
    rnd = g.standard_normal(3000) * 2.0 ** g.integers(-140, 128, 3000)
    mid = (2 * g.integers(128, 256, 1000) + 1) * 2.0 ** g.integers(-130, 120, 1000)
    nudged = np.concatenate([mid * (1 + 2.0 ** -40), mid * (1 - 2.0 ** -40), mid])
    big = np.array([(2 - 2.0 ** -8) * 2.0 ** 127, np.nextafter((2 - 2.0 ** -8) * 2.0 ** 127, 0),
                    2.0 ** -133, 2.0 ** -134, 3 * 2.0 ** -135, 2.0 ** -126, -0.0, 1e-300])
    v = np.concatenate([rnd, nudged, -nudged, big])
    v = v[np.isfinite(v)]
    got = oracle.round_bf16_f64(v)
    ref = np.array([_bf16_nearest_bits(float(t)) for t in v], np.uint16)
    assert np.array_equal(got, ref)
    trap = 1.0 + 2.0 ** -8 + 2.0 ** -40
    assert oracle.widen_bf16_bits(oracle.round_bf16_f64([trap]))[0] == 1.0 + 2.0 ** -7
    assert oracle.widen_bf16_bits(oracle.round_bf16(np.float32(trap)))[0] == 1.0
    assert np.array_equal(oracle.round_to([trap], "bf16"), [1.0 + 2.0 ** -7])


def pin_round_f16():
    g = synth.rng(38)
    rnd = g.standard_normal(20000) * 10.0 ** g.uniform(-9, 5, 20000)
    e = g.integers(-24, 16, 5000)
    k = g.integers(0, 2048, 5000)
    ties = (2 * k + 1) * np.exp2(e - 11.0)                          # half-way points
    special = np.array([0.0, -0.0, 65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -24,
                        2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -14, 6.1e-5, np.inf, -np.inf])
    v = np.concatenate([rnd, ties, -ties, special])
    got = oracle.round_f16(v)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16).view(np.uint16)
    assert np.array_equal(got, ref)
    assert np.array_equal(oracle.widen_f16_bits(got), ref.view(np.float16).astype(np.float64))


def pin_round_f32():
    g = synth.rng(39)
    v = g.standard_normal(50000) * 10.0 ** g.uniform(-44, 38, 50000)
    assert np.array_equal(oracle.round_f32(v).view(np.uint32), v.astype(np.float32).view(np.uint32))


PINS = [
    pin_copy_identity, pin_axpy_half_alpha_single_rounding, pin_axpy_special_cases,
    pin_axpy_exact_rational, pin_axpby_exact_rational,
    pin_dot_ones, pin_dot_arange_closed_forms, pin_dot_alternating_and_unit, pin_dot_fsum_f32,
    pin_dot_cancellation, pin_dot_fraction_random,
    pin_sparse_dot_fraction_and_closed_forms, pin_sparse_dot_is_a_csr_row,
    pin_gemv_identity_and_single_entry, pin_gemv_exact_tiny, pin_gemv_numpy,
    pin_gemv_linearity_and_entries,
    pin_spmv_golden, pin_spmv_laplacian_ones, pin_spmv_eigen_2d, pin_spmv_eigen_3d,
    pin_spmv_dense_bruteforce, pin_spmv_rows, pin_csc_transpose,
    pin_sell_layout_bruteforce, pin_sell_spmv_matches_csr_and_eigen,
    pin_csr_row_bins_bruteforce,
    pin_dense_outer_fd, pin_sampled_outer_fd, pin_scale_dot_gradient,
    pin_round_bf16, pin_round_bf16_f64, pin_round_f16, pin_round_f32,
]
