/*
 * Plain FP64 CPU oracle for the bandwidth-bound linear-algebra operations of
 * Rupp et al., "Performance Portability Study of Linear Algebra Kernels in
 * OpenCL" (IWOCL'14).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark load it.  It shares no header, helper or
 * constant with the CUDA path.
 *
 * Every routine is the plain textbook definition, written as loops in the
 * order the definition states.  Inputs arrive already widened to double (the
 * Python wrapper widens FP32 / BF16 / FP16 storage exactly), so the oracle is
 * a function of the stored values.  Sums use the compensated Dot2 scheme of
 * Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005): each product is
 * split exactly into value + error with an FMA (TwoProduct) and the running
 * sum is split exactly with Knuth's TwoSum, so the result is as accurate as if
 * it were computed in twice double precision and then rounded.
 *
 * Must be compiled with -ffp-contract=off: TwoSum and TwoProduct rely on
 * every + and * being rounded separately (GCC contracts a*b+c into an FMA by
 * default on aarch64, which would silently break them).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- error-free transformations ------------------------------------------ */

/* Knuth's TwoSum: s + e == a + b exactly, s = fl(a + b). */
static void two_sum(double a, double b, double *s, double *e)
{
    double sum = a + b;
    double bv = sum - a;
    double av = sum - bv;
    *s = sum;
    *e = (a - av) + (b - bv);
}

/* TwoProduct via a fused multiply-add: p + e == a * b exactly. */
static void two_prod(double a, double b, double *p, double *e)
{
    double prod = a * b;
    *p = prod;
    *e = fma(a, b, -prod);
}

/* Dot2 accumulator: the running sum is (s + c). */
typedef struct { double s, c; } orc_acc;

static void acc_add_prod(orc_acc *acc, double a, double b)
{
    double p, pe, s, se;
    two_prod(a, b, &p, &pe);
    two_sum(acc->s, p, &s, &se);
    acc->s = s;
    acc->c += se + pe;
}

static double acc_value(const orc_acc *acc, double *lo)
{
    double hi, e;
    two_sum(acc->s, acc->c, &hi, &e);
    if (lo) *lo = e;
    return hi;
}

/* ---- BLAS-1 ------------------------------------------------------------- */

/* Vector copy x <- y (paper Sec. 2, the "archetype" operation). */
void orc_copy(double *x, const double *y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) x[i] = y[i];
}

/*
 * Vector update x <- alpha*y + beta*z (paper Sec. 2, with alpha, beta != 0 in
 * the paper's study).  The library's vec_axpy is the beta = 1 instance
 * x = y + alpha*z, called here with alpha_y = 1.  Each term is rounded
 * separately: fl(fl(alpha_y*y) + fl(alpha_z*z)).
 */
void orc_axpby(double *x, double alpha_y, const double *y, double alpha_z,
               const double *z, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        double ay = alpha_y * y[i];
        double az = alpha_z * z[i];
        x[i] = ay + az;
    }
}

/* x <- y + alpha*z, the vector update the library exports. */
void orc_axpy(double *x, const double *y, const double *z, double alpha, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        double az = alpha * z[i];
        x[i] = y[i] + az;
    }
}

/*
 * Inner product s = <x, y> = sum_i x_i y_i (paper Sec. 2).  Returns the
 * double nearest the compensated sum; *lo (if not NULL) receives the
 * remainder, so hi + lo carries about 106 bits.
 */
double orc_dot(const double *x, const double *y, int64_t n, double *lo)
{
    orc_acc acc = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) acc_add_prod(&acc, x[i], y[i]);
    return acc_value(&acc, lo);
}

/*
 * Inner product of a sparse vector with a dense one: s = sum_k v_k y_{c_k},
 * where the sparse vector holds nnz stored values v_k at positions c_k
 * (paper Sec. 2's inner product with one operand given by its nonzeros; each
 * row of a CSR product y = A x is one such sum).  Compensated sum in
 * increasing k, as in orc_dot.
 */
double orc_sparse_dot(const double *v, const int32_t *c, const double *y, int64_t nnz)
{
    orc_acc acc = {0.0, 0.0};
    for (int64_t k = 0; k < nnz; ++k) acc_add_prod(&acc, v[k], y[c[k]]);
    return acc_value(&acc, NULL);
}

/* Scaling out <- s * v (the backward of the inner product: d<x,y>/dx = y). */
void orc_scale(double *out, const double *v, double s, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = s * v[i];
}

/* ---- BLAS-2: dense matrix-vector product -------------------------------- */

/*
 * y <- A x for an m-by-n matrix A (paper Sec. 2: entry i of the result is the
 * inner product of row i of A with the right-hand side).  layout 0 = row
 * major, A(i,j) = A[i*lda + j]; layout 1 = column major, A(i,j) = A[i + j*lda].
 * Each entry is a compensated sum over j in increasing order, independent of
 * the layout.
 */
void orc_gemv(double *y, const double *A, const double *x, int64_t m, int64_t n,
              int64_t lda, int layout)
{
    for (int64_t i = 0; i < m; ++i) {
        orc_acc acc = {0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            double a = (layout == 0) ? A[i * lda + j] : A[i + j * lda];
            acc_add_prod(&acc, a, x[j]);
        }
        y[i] = acc_value(&acc, NULL);
    }
}

/* One entry of y = A x: the sampled form used on outputs too large to recompute. */
double orc_gemv_entry(const double *A, const double *x, int64_t i, int64_t n,
                      int64_t lda, int layout)
{
    orc_acc acc = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        double a = (layout == 0) ? A[i * lda + j] : A[i + j * lda];
        acc_add_prod(&acc, a, x[j]);
    }
    return acc_value(&acc, NULL);
}

/* ---- sparse matrix-vector product (CSR) ---------------------------------- */

/*
 * y <- A x for A in compressed sparse row form: row i owns the stored entries
 * k = row_ptr[i] .. row_ptr[i+1]-1 with column col_idx[k] and value vals[k];
 * y_i = sum_k vals[k] * x[col_idx[k]].  Repeated columns within a row are
 * summed, which is the standard meaning of the format.  The paper leaves
 * sparse operations out (Sec. 1); this is the textbook definition.
 */
void orc_csr_spmv(double *y, const int32_t *row_ptr, const int32_t *col_idx,
                  const double *vals, const double *x, int64_t m)
{
    for (int64_t i = 0; i < m; ++i) {
        orc_acc acc = {0.0, 0.0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            acc_add_prod(&acc, vals[k], x[col_idx[k]]);
        y[i] = acc_value(&acc, NULL);
    }
}

/* One row of the CSR product (sampled checks at full size). */
double orc_csr_row(const int32_t *row_ptr, const int32_t *col_idx,
                   const double *vals, const double *x, int64_t i)
{
    orc_acc acc = {0.0, 0.0};
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
        acc_add_prod(&acc, vals[k], x[col_idx[k]]);
    return acc_value(&acc, NULL);
}

/*
 * Transpose of an m-by-n CSR matrix, returned as the CSR form of A^T (that is,
 * the CSC form of A): col_ptr (n+1), row_idx (nnz), and perm (nnz) with
 * perm[q] = the CSR position of the q-th CSC entry.  A stable counting sort by
 * column: entries are placed while walking the rows in order, so the entries
 * of each column stay in increasing row order.  Returns 0, or -1 if the
 * cursor array cannot be allocated.
 */
int orc_csr_to_csc(int32_t *col_ptr, int32_t *row_idx, int64_t *perm,
                   const int32_t *row_ptr, const int32_t *col_idx, int64_t m,
                   int64_t n)
{
    int64_t *cursor = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!cursor) return -1;
    for (int64_t j = 0; j <= n; ++j) col_ptr[j] = 0;
    for (int64_t k = 0; k < row_ptr[m]; ++k) col_ptr[col_idx[k] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) col_ptr[j + 1] += col_ptr[j];
    for (int64_t j = 0; j < n; ++j) cursor[j] = col_ptr[j];
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t q = cursor[col_idx[k]]++;
            perm[q] = k;
            row_idx[q] = (int32_t)i;
        }
    }
    free(cursor);
    return 0;
}

/* ---- sliced ELLPACK (SELL-C-sigma) ----------------------------------------- */

/*
 * Row-binned CSR: the rows of an m-row CSR pattern grouped by length.  Row i
 * with L = row_ptr[i+1] - row_ptr[i] stored entries falls in bin b, the
 * smallest b < nbins - 1 with L <= per_lane * 2^b, else in the last bin (rows
 * longer than per_lane * 2^(nbins-2)).  perm lists the rows bin by bin, in
 * increasing row index within a bin (a stable sort by bin); bin_ptr[b] is the
 * position of bin b's first row (bin_ptr[nbins] = m).  The product over the
 * binned rows is the CSR product itself (orc_csr_spmv).
 */
static int64_t row_bin(int64_t len, int64_t per_lane, int64_t nbins)
{
    int64_t b = 0;
    while (b < nbins - 1 && len > (per_lane << b)) ++b;
    return b;
}

void orc_csr_row_bins(const int32_t *row_ptr, int64_t m, int64_t per_lane, int64_t nbins,
                      int32_t *perm, int64_t *bin_ptr)
{
    for (int64_t b = 0; b <= nbins; ++b) bin_ptr[b] = 0;
    /* bin of every row, counted */
    for (int64_t i = 0; i < m; ++i)
        bin_ptr[row_bin((int64_t)row_ptr[i + 1] - row_ptr[i], per_lane, nbins) + 1] += 1;
    for (int64_t b = 0; b < nbins; ++b) bin_ptr[b + 1] += bin_ptr[b];
    /* place rows in increasing index order within each bin */
    int64_t *next = (int64_t *)malloc((size_t)(nbins > 0 ? nbins : 1) * sizeof(int64_t));
    if (!next) return;
    for (int64_t b = 0; b < nbins; ++b) next[b] = bin_ptr[b];
    for (int64_t i = 0; i < m; ++i) {
        int64_t b = row_bin((int64_t)row_ptr[i + 1] - row_ptr[i], per_lane, nbins);
        perm[next[b]++] = (int32_t)i;
    }
    free(next);
}

/*
 * SELL-C-sigma layout of an m-row CSR pattern with slices of C rows: within
 * every window of `sigma` consecutive rows (sigma a multiple of C, or 1 for no
 * sorting) rows are ordered by decreasing length, ties by increasing row index;
 * position p of that order holds original row perm[p] (-1 past the last row,
 * positions padded to a multiple of C).  Slice s (positions s*C .. s*C+C-1) is
 * padded to its longest row: slice_len[s]; its entries start at slice_ptr[s]
 * and entry j of the row at position s*C + r sits at slice_ptr[s] + j*C + r
 * (column-major inside the slice).  cols holds the column, or -1 for padding;
 * map holds the CSR position of the entry, or -1.  Returns the padded size
 * when cols is NULL (first call), else fills the arrays and returns it.
 */
int64_t orc_csr_to_sell(const int32_t *row_ptr, const int32_t *col_idx, int64_t m, int64_t C,
                        int64_t sigma, int32_t *perm, int32_t *slice_len, int64_t *slice_ptr,
                        int32_t *cols, int32_t *map)
{
    int64_t mp = (m + C - 1) / C * C;
    int64_t nslices = mp / C;
    int64_t win = sigma > 1 ? sigma : 1;
    /* order within windows: insertion sort of (length desc, index asc) */
    for (int64_t w0 = 0; w0 < mp; w0 += win) {
        int64_t w1 = w0 + win < mp ? w0 + win : mp;
        for (int64_t p = w0; p < w1; ++p) perm[p] = p < m ? (int32_t)p : -1;
        if (win > 1) {
            for (int64_t p = w0 + 1; p < w1; ++p) {
                int32_t r = perm[p];
                int64_t lr = r >= 0 ? row_ptr[r + 1] - row_ptr[r] : -1;
                int64_t q = p - 1;
                while (q >= w0) {
                    int32_t o = perm[q];
                    int64_t lo = o >= 0 ? row_ptr[o + 1] - row_ptr[o] : -1;
                    if (lo > lr || (lo == lr && (o >= 0 ? o : m + q) < (r >= 0 ? r : m + p))) break;
                    perm[q + 1] = perm[q];
                    --q;
                }
                perm[q + 1] = r;
            }
        }
    }
    int64_t total = 0;
    for (int64_t s = 0; s < nslices; ++s) {
        int64_t L = 0;
        for (int64_t r = 0; r < C; ++r) {
            int32_t i = perm[s * C + r];
            int64_t l = i >= 0 ? row_ptr[i + 1] - row_ptr[i] : 0;
            if (l > L) L = l;
        }
        slice_len[s] = (int32_t)L;
        slice_ptr[s] = total;
        total += L * C;
    }
    slice_ptr[nslices] = total;
    if (!cols) return total;
    for (int64_t s = 0; s < nslices; ++s) {
        for (int64_t r = 0; r < C; ++r) {
            int32_t i = perm[s * C + r];
            int64_t l = i >= 0 ? row_ptr[i + 1] - row_ptr[i] : 0;
            for (int64_t j = 0; j < slice_len[s]; ++j) {
                int64_t slot = slice_ptr[s] + j * C + r;
                if (j < l) {
                    cols[slot] = col_idx[row_ptr[i] + j];
                    map[slot] = (int32_t)(row_ptr[i] + j);
                } else {
                    cols[slot] = -1;
                    map[slot] = -1;
                }
            }
        }
    }
    return total;
}

/* y = A x from the SELL-C-sigma arrays above (vals in SELL slots; padding
 * skipped); each row a compensated sum over its entries in stored order. */
void orc_sell_spmv(double *y, int64_t m, int64_t C, const int32_t *perm,
                   const int32_t *slice_len, const int64_t *slice_ptr, const int32_t *cols,
                   const double *vals, const double *x)
{
    int64_t nslices = (m + C - 1) / C;
    for (int64_t s = 0; s < nslices; ++s) {
        for (int64_t r = 0; r < C; ++r) {
            int32_t i = perm[s * C + r];
            if (i < 0) continue;
            orc_acc acc = {0.0, 0.0};
            for (int64_t j = 0; j < slice_len[s]; ++j) {
                int64_t slot = slice_ptr[s] + j * C + r;
                if (cols[slot] >= 0) acc_add_prod(&acc, vals[slot], x[cols[slot]]);
            }
            y[i] = acc_value(&acc, NULL);
        }
    }
}

/* ---- gradients of the products (reverse mode) ---------------------------- */

/* Dense y = A x:  dA = dy x^T, an m-by-n row-major outer product. */
void orc_dense_outer(double *dA, const double *dy, const double *x, int64_t m,
                     int64_t n, int64_t ldd)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) dA[i * ldd + j] = dy[i] * x[j];
}

/* CSR y = A x:  dvals[k] = dy[row(k)] * x[col(k)] on the stored pattern only. */
void orc_sampled_outer(double *dvals, const int32_t *row_ptr, const int32_t *col_idx,
                       const double *dy, const double *x, int64_t m)
{
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            dvals[k] = dy[i] * x[col_idx[k]];
}

/* ---- storage rounding (reduced-precision storage of the same data) ------- */

/*
 * FP32 -> BF16 with round-to-nearest-even, on the bit pattern: BF16 keeps the
 * top 16 bits of an IEEE binary32.  NaNs are kept quiet NaNs.
 */
void orc_round_bf16(uint16_t *out, const float *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &in[i], sizeof u);
        if ((u & 0x7fffffffu) > 0x7f800000u) {          /* NaN */
            out[i] = (uint16_t)((u >> 16) | 0x0040u);
            continue;
        }
        uint32_t keep = u >> 16;
        uint32_t rest = u & 0xffffu;
        if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
        out[i] = (uint16_t)keep;
    }
}

/*
 * double -> BF16 bit patterns with round-to-nearest-even, in one rounding of
 * the double itself (not through FP32, whose own rounding can move a value
 * onto a BF16 midpoint).  BF16 is FP32's layout with 7 fraction bits: normal
 * values 1.f * 2^e for e in [-126, 127], subnormal spacing 2^-133; values at
 * or above (2 - 2^-8) * 2^127 round to infinity.
 */
void orc_round_bf16_f64(uint16_t *out, const double *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = in[i];
        uint16_t sign = signbit(v) ? 0x8000u : 0u;
        double a = fabs(v);
        if (isnan(v)) { out[i] = (uint16_t)(sign | 0x7fc0u); continue; }
        if (a >= ldexp(2.0 - ldexp(1.0, -8), 127)) { out[i] = (uint16_t)(sign | 0x7f80u); continue; }
        int e;
        frexp(a, &e);                     /* a = f * 2^e, f in [0.5, 1) */
        int exp_unb = e - 1;              /* a = 1.x * 2^exp_unb */
        double quantum = (exp_unb < -126) ? ldexp(1.0, -133) : ldexp(1.0, exp_unb - 7);
        double r = nearbyint(a / quantum);   /* exact scaling; nearest-even */
        double h = r * quantum;
        uint16_t bits;
        if (h == 0.0) {
            bits = 0;
        } else if (h < ldexp(1.0, -126)) {
            bits = (uint16_t)r;           /* subnormal: fraction = r */
        } else {
            int he;
            double hf = frexp(h, &he);    /* h = hf * 2^he */
            int biased = he - 1 + 127;
            uint32_t frac = (uint32_t)((hf * 2.0 - 1.0) * 128.0);
            bits = (uint16_t)((biased << 7) | frac);
        }
        out[i] = (uint16_t)(sign | bits);
    }
}

/* BF16 -> double, exact. */
void orc_widen_bf16(double *out, const uint16_t *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u = (uint32_t)in[i] << 16;
        float f;
        memcpy(&f, &u, sizeof f);
        out[i] = (double)f;
    }
}

/*
 * double -> IEEE binary16 with round-to-nearest-even, written from the format:
 * 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits; subnormals have
 * spacing 2^-24; values at or above 65520 round to infinity.
 */
void orc_round_f16(uint16_t *out, const double *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = in[i];
        uint16_t sign = signbit(v) ? 0x8000u : 0u;
        double a = fabs(v);
        if (isnan(v)) { out[i] = (uint16_t)(sign | 0x7e00u); continue; }
        if (a >= 65520.0) { out[i] = (uint16_t)(sign | 0x7c00u); continue; }
        int e;
        frexp(a, &e);                     /* a = f * 2^e, f in [0.5, 1) */
        int exp_unb = e - 1;              /* a = 1.x * 2^exp_unb */
        double quantum = (exp_unb < -14) ? ldexp(1.0, -24) : ldexp(1.0, exp_unb - 10);
        double q = a / quantum;           /* exact: a power-of-two scaling */
        double r = nearbyint(q);          /* default rounding mode: nearest-even */
        /* r * quantum is representable; recompose the bit pattern */
        double h = r * quantum;
        uint16_t bits;
        if (h == 0.0) {
            bits = 0;
        } else if (h < ldexp(1.0, -14)) {
            bits = (uint16_t)r;           /* subnormal: fraction = r */
        } else {
            int he;
            double hf = frexp(h, &he);    /* h = hf * 2^he */
            int biased = he - 1 + 15;
            uint32_t frac = (uint32_t)((hf * 2.0 - 1.0) * 1024.0);
            bits = (uint16_t)((biased << 10) | frac);
        }
        out[i] = (uint16_t)(sign | bits);
    }
}

/* IEEE binary16 -> double, exact. */
void orc_widen_f16(double *out, const uint16_t *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        uint16_t h = in[i];
        int s = (h >> 15) & 1;
        int e = (h >> 10) & 0x1f;
        int f = h & 0x3ff;
        double v;
        if (e == 0) v = ldexp((double)f, -24);
        else if (e == 31) v = f ? NAN : INFINITY;
        else v = ldexp((double)(1024 + f), e - 25);
        out[i] = s ? -v : v;
    }
}

/* double -> float, round-to-nearest-even (C conversion rule). */
void orc_round_f32(float *out, const double *in, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) out[i] = (float)in[i];
}

/* ---- plain loops: the "plain CPU" baseline, not reference values ----------
 *
 * The benchmark times these beside the oracle: the same operations as the
 * straightforward loops a CPU programmer would write, in the storage type's own
 * arithmetic (FP32 sums for FP32 data), with no compensation.  Nothing checks a
 * kernel against them; a CPU test checks them against the oracle above.
 */
#define ORC_PLAIN(T, SUF)                                                          \
void orc_plain_axpy_##SUF(T *x, const T *y, const T *z, T alpha, int64_t n)        \
{                                                                                  \
    for (int64_t i = 0; i < n; ++i) x[i] = y[i] + alpha * z[i];                   \
}                                                                                  \
double orc_plain_dot_##SUF(const T *x, const T *y, int64_t n)                      \
{                                                                                  \
    T s = 0;                                                                       \
    for (int64_t i = 0; i < n; ++i) s += x[i] * y[i];                              \
    return (double)s;                                                              \
}                                                                                  \
void orc_plain_gemv_##SUF(T *y, const T *A, const T *x, int64_t m, int64_t n,      \
                          int64_t lda, int layout)                                 \
{                                                                                  \
    if (layout == 0) {                                                             \
        for (int64_t i = 0; i < m; ++i) {                                          \
            T s = 0;                                                               \
            for (int64_t j = 0; j < n; ++j) s += A[i * lda + j] * x[j];            \
            y[i] = s;                                                              \
        }                                                                          \
    } else {                                                                       \
        for (int64_t i = 0; i < m; ++i) y[i] = 0;                                  \
        for (int64_t j = 0; j < n; ++j)                                            \
            for (int64_t i = 0; i < m; ++i) y[i] += A[i + j * lda] * x[j];         \
    }                                                                              \
}                                                                                  \
void orc_plain_csr_##SUF(T *y, const int32_t *row_ptr, const int32_t *col_idx,     \
                         const T *vals, const T *x, int64_t m)                     \
{                                                                                  \
    for (int64_t i = 0; i < m; ++i) {                                              \
        T s = 0;                                                                   \
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)                      \
            s += vals[k] * x[col_idx[k]];                                          \
        y[i] = s;                                                                  \
    }                                                                              \
}

ORC_PLAIN(float, f32)
ORC_PLAIN(double, f64)

void orc_plain_copy(void *dst, const void *src, int64_t nbytes)
{
    memcpy(dst, src, (size_t)nbytes);
}
