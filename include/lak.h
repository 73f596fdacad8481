/*
 * lak.h -- C ABI of a GB300 (sm_103a) library of memory-bandwidth-bound
 * linear-algebra kernels: the vector copy, vector update, inner product and
 * dense matrix-vector product studied by Rupp, Tillet, Rudolf, Weinbub,
 * Grasser and Juengel, "Performance Portability Study of Linear Algebra
 * Kernels in OpenCL" (IWOCL'14), plus the CSR sparse matrix-vector product,
 * all run under one shared launch-size configuration (lak_cfg).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Every array argument is DEVICE memory owned by the caller (for
 *   instance a PyTorch CUDA tensor's data pointer) on the current CUDA device.
 *   The library allocates nothing and frees nothing; where a kernel needs
 *   scratch memory the caller passes it in ("workspace"), sized by the matching
 *   *_workspace() query for the same arguments.
 * Workspace layout.  Every workspace begins with a counter area of
 *   LAK_WS_COUNTER_BYTES that must be zero-filled before the workspace is first
 *   used; kernels touch it only with self-resetting arrival counters, so every
 *   completed call leaves it zero again.  Scratch data follows it.  One
 *   workspace (256-byte aligned, as large as the largest query) can therefore
 *   serve any sequence of calls of any op and shape on one stream; calls that
 *   share a workspace must not run concurrently on the device.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *   default stream).  Every call is asynchronous on that stream: no call
 *   synchronises the host, and scalar results (vec_dot) stay on the device.
 * Storage types (lak_dtype).  LAK_F32 and LAK_F64 compute in their own
 *   precision; LAK_BF16 and LAK_F16 are reduced-precision STORAGE with FP32
 *   arithmetic.  Results are rounded to the storage type with
 *   round-to-nearest-even.
 * Alignment.  Any element-aligned pointer is accepted.  Wide (up to 32-byte)
 *   vector loads are used when the pointers of one call share their offset
 *   modulo the load width; otherwise the call runs the same kernel with
 *   one-element accesses.  Misalignment is never an error.
 * Errors.  Arguments are checked on the host before anything is launched; a
 *   failed check returns a negative lak_status and launches nothing.  A
 *   launch that CUDA rejects returns LAK_ECUDA.  lak_last_error() gives a
 *   human-readable message for the calling thread's last failure.  The
 *   library never calls exit/abort and never traps on the device.
 * Sizes.  Element counts and leading dimensions are int64_t; all device
 *   index arithmetic is 64-bit.  CSR index arrays are int32 (nnz < 2^31).
 * Aliasing.  vec_axpy allows x == y or x == z (in place); vec_dot allows
 *   x == y.  Outputs of dense_gemv and csr_spmv must not overlap any input.
 */
#ifndef LAK_H
#define LAK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LAK_API __attribute__((visibility("default")))
#else
#define LAK_API
#endif

typedef enum {
    LAK_OK = 0,
    LAK_EINVAL = -1,      /* bad size, pointer, leading dimension or config */
    LAK_EDTYPE = -2,      /* unknown or unsupported storage type */
    LAK_ELAYOUT = -3,     /* unknown matrix layout */
    LAK_ECUDA = -4,       /* the CUDA runtime rejected a launch or query */
    LAK_EWORKSPACE = -5   /* workspace missing or smaller than the query said */
} lak_status;

typedef enum { LAK_F32 = 0, LAK_F64 = 1, LAK_BF16 = 2, LAK_F16 = 3 } lak_dtype;

/* Size of the zero-filled counter area at the start of every workspace. */
#define LAK_WS_COUNTER_BYTES 65536

typedef enum { LAK_ROW_MAJOR = 0, LAK_COL_MAJOR = 1 } lak_layout;

/* Loop skeletons of Sec. 2: the index advances by the whole grid ("global
 * increment") or each block walks one contiguous range ("local increment"). */
typedef enum { LAK_INC_GLOBAL = 0, LAK_INC_LOCAL = 1 } lak_increment;

typedef enum {
    LAK_OP_COPY = 0, LAK_OP_AXPY = 1, LAK_OP_DOT = 2,
    LAK_OP_GEMV_ROW = 3, LAK_OP_GEMV_COL = 4, LAK_OP_SPMV = 5,
    LAK_OP_COUNT = 6
} lak_op;

/*
 * Kernel configuration (Sec. 1 defines a configuration as source variant +
 * local work size + global work size; Sec. 2 parameterises it by increment
 * type, vector length, local size and number of work-groups).
 *   block      threads per block, a multiple of 32 in [32, 512]    (0 = auto;
 *              512 is also the largest local size the paper studies)
 *   grid       number of blocks, >= 1                              (0 = auto)
 *   vec        elements per thread per access group: 1, 2, 4, 8 or 16
 *              (0 = auto).  Per op: copy/axpy/dot and row-major GEMV read
 *              `vec` consecutive elements per thread per step; column-major
 *              GEMV gives each thread `vec` consecutive rows; CSR SpMV issues
 *              `vec` independent nonzero loads per thread per step.
 *   increment  LAK_INC_GLOBAL or LAK_INC_LOCAL (ignored when block = 0)
 * A NULL cfg, or one whose block is 0, takes the library default for the op,
 * storage type and size bucket (set by lak_set_default_cfg[_bucket], e.g. from
 * an autotuning cache, else built in); a zero grid or vec in an otherwise
 * explicit cfg is filled in by the library.
 */
typedef struct {
    int32_t block;
    int32_t grid;
    int32_t vec;
    int32_t increment;
} lak_cfg;

/* Message for the calling thread's most recent failed call ("" if none).
 * Library infrastructure: no counterpart in the paper. */
LAK_API const char *lak_last_error(void);

/* ABI version of this header (bumped on any incompatible change).  Library
 * infrastructure: no counterpart in the paper. */
LAK_API int32_t lak_abi_version(void);

/*
 * Size buckets.  Defaults are kept per (op, dtype, size bucket): the bucket is
 * fixed by the call's algorithmic bytes B (operands read once + results
 * written; copy/dot 2n*s, axpy 3n*s, dense_gemv (mn + m + n)*s, csr_spmv
 * nnz*(s + 4) + (m + 1)*4 + (m + n)*s, s = bytes per stored value):
 *   0: B < 8 MiB    1: B < 64 MiB    2: B < 512 MiB    3: otherwise.
 * The paper tunes one configuration per device and operation (Sec. 3); on
 * GB300 the best launch shape for a call that moves a few MB (launch-latency
 * bound) differs from the one for a call that streams GBs, so the autotuner
 * fills one entry per bucket.
 */
#define LAK_SIZE_BUCKETS 4

/*
 * The size bucket (0 .. LAK_SIZE_BUCKETS-1) a call of `op` with these sizes
 * falls in (sizes as in lak_resolve_cfg), or a negative lak_status.  The
 * buckets refine the paper's one configuration per device and operation
 * (Sec. 3).
 */
LAK_API int32_t lak_size_bucket(lak_op op, lak_dtype dtype, int64_t m, int64_t n, int64_t nnz);

/*
 * Replace the default configuration used for (op, dtype) in size bucket
 * `bucket` (-1: every bucket) when a call passes no explicit cfg; cfg = NULL
 * restores the built-in default.  Process-wide; not synchronised against
 * concurrent calls that read it.  (Sec. 3.4: the configuration chosen for a
 * device, here per size bucket.)
 */
LAK_API lak_status lak_set_default_cfg_bucket(lak_op op, lak_dtype dtype, int32_t bucket,
                                              const lak_cfg *cfg);

/* lak_set_default_cfg_bucket(op, dtype, -1, cfg): every size bucket (the
 * paper's single configuration per device and operation, Sec. 3.4). */
LAK_API lak_status lak_set_default_cfg(lak_op op, lak_dtype dtype, const lak_cfg *cfg);

/*
 * The configuration (Sec. 1: local and global work size, with Sec. 2's vector
 * length and increment) a call of `op` would launch with on the current device,
 * after defaults and automatic fields are filled in.  Sizes: for the vector
 * ops m = n = the vector length; for dense_gemv the matrix is m-by-n; for
 * csr_spmv m rows, n columns and nnz stored entries (nnz is ignored by the
 * other ops).  `vec` in *out is the vector width the call would actually use
 * for aligned pointers.  Writes *out; returns LAK_OK or a negative status.
 */
LAK_API lak_status lak_resolve_cfg(lak_op op, lak_dtype dtype, int64_t m, int64_t n,
                                   int64_t nnz, const lak_cfg *cfg, lak_cfg *out);

/*
 * vec_copy: x[i] = y[i] for 0 <= i < n  (Sec. 2, the copy operation x <- y,
 * which the paper uses as the archetype whose good configurations carry over
 * to the other operations, Sec. 3.2 and Sec. 4).  A bit copy of n elements of
 * `dtype`; x and y must not overlap unless x == y.  n = 0 is a no-op.
 */
LAK_API lak_status vec_copy(void *x, const void *y, int64_t n, lak_dtype dtype,
                            const lak_cfg *cfg, void *stream);

/*
 * vec_axpy: x[i] = y[i] + alpha * z[i] for 0 <= i < n  (Sec. 2's scaled
 * vector addition x <- alpha*y + beta*z, taken with the first coefficient 1).
 * alpha is rounded to the arithmetic type (FP32 for F32/BF16/F16 storage, FP64
 * for F64) and each element is one fused multiply-add rounded once to the
 * storage type.  x may equal y or z.  n = 0 is a no-op.
 */
LAK_API lak_status vec_axpy(void *x, const void *y, const void *z, double alpha,
                            int64_t n, lak_dtype dtype, const lak_cfg *cfg,
                            void *stream);

/*
 * vec_axpby: x[i] = alpha * y[i] + beta * z[i]  (Sec. 2's scaled vector
 * addition in its general form).  alpha and beta are rounded to the arithmetic
 * type; each element is fl(alpha*y + fl(beta*z)) (one product rounded, then one
 * fused multiply-add), rounded once more to the storage type for BF16/FP16.
 * x may equal y or z.  Launch configuration as for vec_axpy.
 */
LAK_API lak_status vec_axpby(void *x, double alpha, const void *y, double beta, const void *z,
                             int64_t n, lak_dtype dtype, const lak_cfg *cfg, void *stream);

/*
 * vec_axpby_strided: the same on strided vectors -- element i of x is
 * x[i*incx] (likewise y, z); increments are in elements, may be negative (the
 * pointer then addresses element 0, the highest address) and must not make x
 * overlap itself (incx != 0).  Scalar accesses: the paper notes that its wide
 * vector types suit strided access poorly (Sec. 2).
 */
LAK_API lak_status vec_axpby_strided(void *x, int64_t incx, double alpha, const void *y,
                                     int64_t incy, double beta, const void *z, int64_t incz,
                                     int64_t n, lak_dtype dtype, void *stream);

/*
 * vec_axpy_norm2: x[i] = y[i] + alpha * z[i] and *out = sum_i x[i]^2 of the
 * stored x, in one pass (Sec. 2's vector update fused with Sec. 2's inner
 * product of its result with itself: 3n elements moved instead of 5n for vec_axpy then vec_dot).
 * Reduction, `out` type and workspace rules as for vec_dot; the workspace size
 * comes from vec_axpy_norm2_workspace.
 */
LAK_API size_t vec_axpy_norm2_workspace(int64_t n, lak_dtype dtype, const lak_cfg *cfg);
LAK_API lak_status vec_axpy_norm2(void *x, const void *y, const void *z, double alpha, void *out,
                                  int64_t n, lak_dtype dtype, void *workspace, size_t ws_bytes,
                                  const lak_cfg *cfg, void *stream);

/*
 * Workspace bytes vec_dot (Sec. 2's inner product) needs for these arguments on
 * the current device (a partial sum per block and one arrival counter).  0 on
 * invalid input.
 */
LAK_API size_t vec_dot_workspace(int64_t n, lak_dtype dtype, const lak_cfg *cfg);

/*
 * vec_dot: *out = sum_i x[i] * y[i]  (Sec. 2's inner product, reduced in
 * on-chip memory per work-group; the paper leaves the cross-group combine
 * open).  Single pass: each thread accumulates in the arithmetic type, warps
 * reduce with shuffles, each block's partial is combined in FP64 and written
 * to the workspace, and the last block to arrive adds the partials in FP64 in
 * block order, so the result is deterministic for a fixed configuration.
 * `out` is one device element: float for F32/BF16/F16, double for F64.
 * `workspace`: >= vec_dot_workspace() bytes, 256-byte aligned, laid out as
 * described at the top of this header.  n = 0 writes 0.
 */
LAK_API lak_status vec_dot(void *out, const void *x, const void *y, int64_t n,
                           lak_dtype dtype, void *workspace, size_t ws_bytes,
                           const lak_cfg *cfg, void *stream);

/*
 * Row-binned CSR (an SpMV format variant; the paper leaves sparse formats out,
 * Sec. 1).  The CSR arrays are used as they are; a row permutation groups the
 * rows by length.  Row i with L stored entries falls in bin b, the smallest
 * b < LAK_CSR_BINS - 1 with L <= LAK_CSR_BIN_PER_LANE * 2^b, else in the last
 * bin.  perm (m int32, device) lists the rows bin by bin, in increasing row
 * index within a bin; bin_ptr (LAK_CSR_BINS + 1 int64, device) holds each
 * bin's first position, bin_ptr[LAK_CSR_BINS] = m.
 *
 * csr_bin_build computes perm and bin_ptr from row_ptr on the device (three
 * kernels; workspace >= csr_bin_workspace(m) bytes, 256-byte aligned, no
 * zeroing needed).  csr_bin_spmv computes y = A x in one launch: rows of bin b
 * get 2^min(b, 5) lanes each (all of a bin's rows need one step of at most
 * LAK_CSR_BIN_PER_LANE loads per lane, except the last bin's, which loop), so
 * every warp serves rows of similar length.  Each y[i] is written once; the
 * result is deterministic.  cfg: block and grid only (0 = automatic).
 * Requirements the library does not check on the device: perm and bin_ptr
 * from csr_bin_build for this row_ptr, and the CSR requirements of csr_spmv.
 */
#define LAK_CSR_BINS 7
#define LAK_CSR_BIN_PER_LANE 4
LAK_API size_t csr_bin_workspace(int64_t m);
LAK_API lak_status csr_bin_build(int32_t *perm, int64_t *bin_ptr, const int32_t *row_ptr,
                                 int64_t m, void *workspace, size_t ws_bytes, void *stream);
LAK_API lak_status csr_bin_spmv(void *y, const int32_t *row_ptr, const int32_t *col_idx,
                                const void *vals, const void *x, const int32_t *perm,
                                const int64_t *bin_ptr, int64_t m, int64_t n, int64_t nnz,
                                lak_dtype dtype, const lak_cfg *cfg, void *stream);

/*
 * vec_dot_sparse: *out = sum_{k<nnz} vals[k] * y[idx[k]] -- the inner product
 * of Sec. 2 with one operand given by its nonzeros: a sparse vector of nnz
 * stored values `vals` at positions `idx` (int32) times a dense vector y of n
 * elements (the sparse BLAS "usdot").  Every row of a CSR product is one such
 * sum, so its time on a matrix's own (vals, col_idx) is the floor that the
 * x gather sets for any CSR kernel on that matrix.  Values and indices stream
 * in packs, y is gathered through L1, and the reduction is vec_dot's (same
 * configuration, workspace and determinism).  `out` is one device element:
 * float for F32/BF16/F16, double for F64.  Requirement the library does not
 * check on the device: 0 <= idx[k] < n; repeated indices are summed.
 * nnz = 0 writes 0.
 */
LAK_API size_t vec_dot_sparse_workspace(int64_t nnz, lak_dtype dtype, const lak_cfg *cfg);
LAK_API lak_status vec_dot_sparse(void *out, const void *vals, const int32_t *idx, const void *y,
                                  int64_t nnz, int64_t n, lak_dtype dtype, void *workspace,
                                  size_t ws_bytes, const lak_cfg *cfg, void *stream);

/*
 * vec_dot_compensated: *out = sum_i x[i] * y[i] for FP32, BF16 or FP16 storage,
 * accumulated with compensated FP32 arithmetic (the inner product of Sec. 2;
 * the scheme is Ogita, Rump and Oishi's Dot2, 2005): each product is split
 * exactly with one FMA and each running sum with TwoSum, the error terms are
 * carried alongside, and the per-thread (sum, error) pairs are combined in FP64.
 * The result behaves as if accumulated in about twice FP32 precision, so
 * cancellation among terms of widely different magnitude costs far less
 * accuracy than in vec_dot.  `out` is one DEVICE double.  Workspace as for
 * vec_dot (vec_dot_workspace gives its size).  F64 storage returns LAK_EDTYPE
 * (vec_dot already accumulates FP64 data in FP64).  n = 0 writes 0.
 */
LAK_API lak_status vec_dot_compensated(double *out, const void *x, const void *y, int64_t n,
                                       lak_dtype dtype, void *workspace, size_t ws_bytes,
                                       const lak_cfg *cfg, void *stream);

/*
 * vec_dot_noalloc: the same inner product as vec_dot (same kernel, result and
 * tolerance), for callers that cannot give the library scratch memory -- for
 * instance a host application whose own memory manager owns every device
 * buffer and hands out only the operands, or a binding from another language
 * that has no device allocator at hand.  The paper has no counterpart; this is
 * an interface convenience of this library.
 *   Scratch: a fixed array of LAK_WS_COUNTER_BYTES + 8 * LAK_DOT_NOALLOC_MAX_BLOCKS
 *     bytes (about 128 KiB) compiled into the library; every GPU that loads the
 *     library holds it until the process exits.  The call allocates nothing.
 *   Limit: the launch may use at most LAK_DOT_NOALLOC_MAX_BLOCKS blocks (one
 *     partial sum each); a configuration asking for more is rejected with
 *     LAK_EINVAL and launches nothing.  Default configurations stay far below.
 *   First call per device: looks up the array's device address (and may load
 *     the library's GPU code onto the device); make it before any stream
 *     capture starts.
 *   Sharing: all calls on a device use the same array.  Calls that overlap on
 *     the GPU (e.g. on different streams) race and give wrong results; each call
 *     clears the arrival counter before its kernel runs.
 * Arguments as for vec_dot, without the workspace.  n = 0 writes 0.
 */
#define LAK_DOT_NOALLOC_MAX_BLOCKS 8192
LAK_API lak_status vec_dot_noalloc(void *out, const void *x, const void *y, int64_t n,
                                   lak_dtype dtype, const lak_cfg *cfg, void *stream);

/*
 * Workspace bytes dense_gemv (Sec. 2's matrix-vector product) needs
 * (column-major split-K partials and per-tile counters; 0 for row-major) on the
 * current device.
 */
LAK_API size_t dense_gemv_workspace(int64_t m, int64_t n, lak_layout layout,
                                    lak_dtype dtype, const lak_cfg *cfg);

/*
 * dense_gemv: y = A x for an m-by-n matrix  (Sec. 2's matrix-vector product,
 * where work-group i forms the inner product of row i with the right-hand
 * side; the column-major layout is this library's addition).
 *   LAK_ROW_MAJOR: A(i,j) = A[i*lda + j], lda >= max(1, n).  A group of
 *     threads per row (sized from n) reduces with shuffles.
 *   LAK_COL_MAJOR: A(i,j) = A[i + j*lda], lda >= max(1, m).  Each thread owns
 *     `vec` consecutive rows and sweeps columns; wide matrices are split over
 *     columns (split-K), the partials land in `workspace` and the last block
 *     of each row tile adds them in split order (deterministic).  Called on
 *     the storage of a row-major matrix B (n-by-m) with layout COL_MAJOR this
 *     computes B^T x.
 * y has m elements, x has n.  `workspace` (>= dense_gemv_workspace() bytes,
 * 256-byte aligned, laid out as described at the top of this header) may be
 * NULL when the query returns 0.  m = 0 is a no-op; n = 0 writes y = 0.
 */
LAK_API lak_status dense_gemv(void *y, const void *A, const void *x, int64_t m,
                              int64_t n, int64_t lda, lak_layout layout,
                              lak_dtype dtype, void *workspace, size_t ws_bytes,
                              const lak_cfg *cfg, void *stream);

/*
 * dense_gemv_axpby: y = alpha * A x + beta * y, same layouts, workspace and
 * configuration as dense_gemv (Sec. 2's matrix-vector product and vector update
 * fused: y is read only when beta != 0).  dense_gemv is the alpha = 1, beta = 0 case.
 */
LAK_API lak_status dense_gemv_axpby(void *y, double alpha, const void *A, const void *x,
                                    double beta, int64_t m, int64_t n, int64_t lda,
                                    lak_layout layout, lak_dtype dtype, void *workspace,
                                    size_t ws_bytes, const lak_cfg *cfg, void *stream);

/*
 * dense_gemv_trans: y = A^T x for the m-by-n matrix A stored as for dense_gemv
 * (y has n elements, x has m): Sec. 2's matrix-vector product in the other
 * layout of the same storage.  Workspace: dense_gemv_workspace(n, m, <the other layout>, ...).
 */
LAK_API lak_status dense_gemv_trans(void *y, const void *A, const void *x, int64_t m, int64_t n,
                                    int64_t lda, lak_layout layout, lak_dtype dtype,
                                    void *workspace, size_t ws_bytes, const lak_cfg *cfg,
                                    void *stream);

/*
 * csr_spmv: y[i] = sum_{k=row_ptr[i]}^{row_ptr[i+1]-1} vals[k] * x[col_idx[k]]
 * for an m-by-n CSR matrix with nnz stored entries (textbook CSR product; the
 * paper leaves sparse formats out of its study, Sec. 1).  Three variants,
 * chosen by the mean row length nnz/m (rounded up):
 *   mean <= 12 (short, regular rows such as stencils): one lane per row (two
 *     for means 9..12); the lane issues `vec` independent loads of its row at a
 *     time through L1, so a warp keeps 32 rows in flight;
 *   13 <= mean <= 64: warp-segmented -- a warp owns 32 consecutive rows, whose
 *     entries are contiguous; each lane takes `vec` consecutive entries
 *     (16-byte loads when col_idx and vals are 16-byte aligned), accumulates
 *     them with one fused multiply-add each and splits at row ends; rows
 *     crossing lanes are joined by a segmented warp scan, deterministically and
 *     without atomics;
 *   mean > 64: a power-of-two group of lanes per row (up to a warp) strides
 *     through the row and reduces with shuffles.
 * The environment variables LAK_SPMV_SEG_MIN_MEAN / LAK_SPMV_SEG_MAX_MEAN
 * (read once) move the bounds of the middle range.
 * Requirements the library does not check
 * on the device: row_ptr[0] = 0, row_ptr non-decreasing, row_ptr[m] = nnz,
 * 0 <= col_idx[k] < n.  Repeated columns in a row are summed.  m = 0 is a
 * no-op; empty rows give 0.
 */
LAK_API lak_status csr_spmv(void *y, const int32_t *row_ptr, const int32_t *col_idx,
                            const void *vals, const void *x, int64_t m, int64_t n,
                            int64_t nnz, lak_dtype dtype, const lak_cfg *cfg,
                            void *stream);

/* ------------------------------------------------------------------------
 * SELL-C-sigma (sliced ELLPACK, C = 32): a format variant of the CSR product
 * (an extension of this library; the paper leaves sparse formats out, Sec. 1).
 * Rows are ordered by decreasing length within windows of `sigma` rows
 * (sigma = 1: no reordering; else a multiple of 32, at most 4096), ties by row
 * index; position p holds original row perm[p] (-1 past the last row);
 * positions are padded to mp = 32 * ceil(m / 32).  Slice s (positions
 * 32s..32s+31) is padded to its longest row, slice_len[s] entries per row,
 * stored column-major from slice_ptr[s]: entry j of the row at position
 * 32s + r is slot slice_ptr[s] + 32j + r.  cols[slot] is the column or -1
 * (padding); map[slot] the CSR position or -1.  The product runs one warp per
 * slice with coalesced 32-slot loads and adds each row in its CSR order.
 * Conversion, one time per pattern:
 *   1. csr_to_sell_count writes perm (mp), slice_len (mp/32) and slice_ptr
 *      (mp/32 + 1; slice_ptr[mp/32] = total slots);
 *   2. with total read back, csr_to_sell_fill writes cols and map (total each);
 *   3. sell_pack_values puts CSR values into SELL slots (again whenever the
 *      values change).
 * ---------------------------------------------------------------------- */
LAK_API lak_status csr_to_sell_count(const int32_t *row_ptr, int64_t m, int32_t sigma,
                                     int32_t *perm, int32_t *slice_len, int64_t *slice_ptr,
                                     void *stream);
LAK_API lak_status csr_to_sell_fill(const int32_t *row_ptr, const int32_t *col_idx, int64_t m,
                                    const int32_t *perm, const int32_t *slice_len,
                                    const int64_t *slice_ptr, int32_t *cols, int32_t *map,
                                    void *stream);
LAK_API lak_status sell_pack_values(void *sell_vals, const void *csr_vals, const int32_t *map,
                                    int64_t total, lak_dtype dtype, void *stream);
/* The SELL-C-sigma product (outside the paper, Sec. 1, like every sparse
 * format): y[perm[p]] = sum over the row at position p, for the m rows.  cfg: block
 * (warps of it each take a slice), grid (0 = one warp per slice), vec (slots
 * loaded per lane per step), increment; NULL = (256, 0, 4, global). */
LAK_API lak_status sell_spmv(void *y, const int64_t *slice_ptr, const int32_t *slice_len,
                             const int32_t *perm, const int32_t *cols, const void *vals,
                             const void *x, int64_t m, lak_dtype dtype, const lak_cfg *cfg,
                             void *stream);

/* ------------------------------------------------------------------------
 * Reverse-mode building blocks for the products above (an extension of this
 * library; the paper studies forward operations only).  For y = A x:
 * dA = dy x^T (dense_outer; on a CSR pattern csr_sampled_outer) and
 * dx = A^T dy (dense_gemv on the same storage with the other layout; for CSR a
 * csr_spmv on the transpose from csr_transpose, with the values brought into
 * its order by vec_gather).  For s = <x, y>: dx = ds * y (vec_scale_dev, the
 * scale read from device memory so that no host synchronisation is needed).
 * ---------------------------------------------------------------------- */

/* dA[i*ldd + j] = dy[i] * x[j] for i < m, j < n (ldd >= n); one product
 * rounded once to the storage type.  Derivative building block: no counterpart
 * in the paper. */
LAK_API lak_status dense_outer(void *dA, const void *dy, const void *x, int64_t m, int64_t n,
                               int64_t ldd, lak_dtype dtype, void *stream);

/* dvals[k] = dy[i] * x[col_idx[k]] for every stored entry k of row i of an
 * m-row CSR pattern with nnz entries (the gradient of the CSR product with
 * respect to its values; no counterpart in the paper). */
LAK_API lak_status csr_sampled_outer(void *dvals, const int32_t *row_ptr, const int32_t *col_idx,
                                     const void *dy, const void *x, int64_t m, int64_t nnz,
                                     lak_dtype dtype, void *stream);

/* Workspace bytes csr_transpose needs for a matrix with n columns (derivative
 * building block; no counterpart in the paper). */
LAK_API size_t csr_transpose_workspace(int64_t n);

/* The CSC form of an m-by-n CSR pattern (derivative building block; no
 * counterpart in the paper): col_ptr (n+1), row_idx (nnz) and
 * perm (nnz), perm[q] = the CSR position of the q-th CSC entry, entries of
 * each column in increasing CSR position (the result of a stable counting
 * sort; deterministic).  (col_ptr, row_idx) with values vals[perm] is A^T in
 * CSR form.  Workspace: csr_transpose_workspace(n) bytes, 256-byte aligned, no
 * initial contents required. */
LAK_API lak_status csr_transpose(int32_t *col_ptr, int32_t *row_idx, int32_t *perm,
                                 const int32_t *row_ptr, const int32_t *col_idx, int64_t m,
                                 int64_t n, int64_t nnz, void *workspace, size_t ws_bytes,
                                 void *stream);

/* dst[i] = src[idx[i]] for i < n (a bit copy of elements of `dtype`; derivative
 * building block, no counterpart in the paper). */
LAK_API lak_status vec_gather(void *dst, const void *src, const int32_t *idx, int64_t n,
                              lak_dtype dtype, void *stream);

/* out[i] = alpha * v[i], alpha ONE DEVICE element: float for F32/BF16/F16,
 * double for F64 (the type vec_dot writes).  Derivative building block (the
 * inner product's gradient); no counterpart in the paper. */
LAK_API lak_status vec_scale_dev(void *out, const void *v, const void *alpha, int64_t n,
                                 lak_dtype dtype, void *stream);

/* ------------------------------------------------------------------------
 * Batched operations: many independent instances of uneven sizes in one
 * persistent launch (an extension of this library; the paper runs one
 * operation at a time).
 *
 * Two steps, so that the launch itself reads nothing from the host and can be
 * replayed (for instance from a CUDA graph) as often as wanted:
 *   1. lak_batch_plan (host only, no CUDA call): from the caller's instance
 *      descriptors (in HOST memory) it writes a work table into a caller host
 *      buffer -- a header, per-instance prefix offsets of work units and the
 *      descriptors with their per-instance launch details -- and fills a
 *      lak_batch_info.  Called with table = NULL it only fills the info
 *      (table and workspace sizes).  Work units hold about the same number of
 *      bytes, so uneven instances are balanced across the persistent grid.
 *   2. The caller copies the table to device memory (any 8-byte aligned
 *      buffer) and calls lak_batch_run with it and a workspace of
 *      info->workspace_bytes (laid out like every workspace: zero-filled counter
 *      area first).  Pointers inside the descriptors must stay valid and the
 *      operands must not overlap across instances.
 * Ops: LAK_OP_AXPY (lak_axpy_desc), LAK_OP_DOT (lak_dot_desc; `out` is float
 * for F32/BF16/F16, double for F64), LAK_OP_GEMV_ROW (lak_gemv_desc, row-major
 * instances), LAK_OP_SPMV (lak_csr_desc, warp-segmented rows; its warps take
 * 32-row blocks in order from a ticket counter in the workspace, so cfg.increment
 * does not apply to it).  The dot and CSR batches keep counters in the
 * workspace: one run of a batch at a time per workspace.  Per instance
 * the results equal those of the single-instance calls up to the order of
 * floating-point summation (axpy: identical).  The dot keeps at most
 * LAK_WS_COUNTER_BYTES / 4 instances (one arrival counter each).  A NULL cfg
 * (or block 0) takes the batched default for (op, dtype): the configuration
 * installed with lak_set_batch_default_cfg (the autotuner's cache), else the
 * batched kernels' built-in launch shape -- never the per-size defaults of the
 * single-instance calls.  Batched GEMV takes at most 128 threads per block
 * (LAK_EINVAL otherwise).
 * ---------------------------------------------------------------------- */
typedef struct { void *x; const void *y; const void *z; int64_t n; double alpha; } lak_axpy_desc;
typedef struct { void *out; const void *x; const void *y; int64_t n; } lak_dot_desc;
typedef struct { void *y; const void *A; const void *x; int64_t m; int64_t n; int64_t lda; } lak_gemv_desc;
typedef struct {
    void *y; const int32_t *row_ptr; const int32_t *col_idx; const void *vals; const void *x;
    int64_t m; int64_t n; int64_t nnz;
} lak_csr_desc;

typedef struct {
    int64_t count;          /* instances */
    int64_t total_units;    /* work units over all instances */
    int64_t unit_elems;     /* elements (or rows, for GEMV / SpMV) per unit */
    size_t table_bytes;     /* size of the work table */
    size_t workspace_bytes; /* device workspace lak_batch_run needs */
    lak_cfg cfg;            /* resolved launch configuration */
    int32_t op;
    int32_t dtype;
} lak_batch_info;

/* Plan a batch on the host, then run it (see above; no counterpart in the
 * paper, which runs one operation at a time). */
LAK_API lak_status lak_batch_plan(lak_op op, lak_dtype dtype, const void *host_descs, int64_t count,
                                  const lak_cfg *cfg, void *host_table, size_t table_bytes,
                                  lak_batch_info *info);

LAK_API lak_status lak_batch_run(const lak_batch_info *info, const void *dev_table, void *workspace,
                                 size_t ws_bytes, void *stream);

/*
 * Default launch configuration of lak_batch_plan for (op, dtype) when it is
 * given no cfg (the batched form of Sec. 2's tuning parameters, chosen by this
 * library's autotuner over the batching workload).  cfg = NULL or block 0
 * removes the entry (back to the built-in shape).  block: 32..512 in steps of
 * 32 (batched GEMV: at most 128); grid >= 0 (0 = the SM count times the blocks
 * of `block` threads an SM holds by thread count, 2048 / block; capped at the
 * batch's work units); vec 0 (the built-in width) or 1, 2, 4, 8, 16 (CSR uses 4 or
 * 8 entries per lane and clamps to that range).  Host only; process-wide;
 * plans made earlier keep their configuration.
 */
LAK_API lak_status lak_set_batch_default_cfg(lak_op op, lak_dtype dtype, const lak_cfg *cfg);

/* ------------------------------------------------------------------------
 * Measurement aid (no counterpart in the paper, whose roofs are the devices'
 * nominal memory bandwidths, Sec. 3): the FP64 FMA throughput of the device.
 * On GB300 the FP64 dense and sparse products are bound by the FP64 pipe, so
 * their roof is this measured rate.
 *
 * lak_probe_fma_f64 launches `grid` blocks of `block` threads; every thread
 * runs 8 independent chains of `iters` dependent FMAs (a <- a*b + c with
 * values that stay normal), then the chains are summed and reduced over each
 * warp and lane 0 writes one double to out[warp index], so `out` (device) must
 * hold grid * block / 32 doubles.  lak_probe_fma_f64_flops gives the floating-
 * point operations of such a launch (2 per FMA).  Time it with events on
 * `stream`.  Errors: LAK_EINVAL for iters < 1, grid < 1, block outside
 * 32..1024 or not a multiple of 32, or a NULL / misaligned out.
 * ---------------------------------------------------------------------- */
LAK_API lak_status lak_probe_fma_f64(double *out, int64_t iters, int32_t grid, int32_t block,
                                     void *stream);
LAK_API int64_t lak_probe_fma_f64_flops(int64_t iters, int32_t grid, int32_t block);

#ifdef __cplusplus
}
#endif

#endif /* LAK_H */
