// Dense matrix-vector product y = A x (Rupp et al., IWOCL'14, Sec. 2: entry i
// of the result is the inner product of row i of A with the right-hand side,
// computed by one work-group and reduced in on-chip memory).
//
// Row-major: a group of G threads (G a power of two, from 1 up to the whole
// block) owns one row; each thread reads V consecutive matrix entries per step
// with wide streamed loads (after a short per-row head that brings the row to
// the access width, so any leading dimension takes the wide path) and the
// matching V entries of x with cached loads (x is re-read by every row, so it
// lives in L1/L2), then the group reduces with shuffles (and shared memory
// across warps when G > 32).  G grows with
// the row length, so long rows use a whole block -- the paper's one
// work-group per row -- and short rows pack several rows per warp.
//
// Column-major (this library's addition): A(i,j) = A[i + j*lda].  A block owns
// a tile of 32*V consecutive rows; lane l holds V consecutive rows and every
// warp walks a strided subset of the columns, so each warp-wide load reads
// 32*V consecutive entries of one column.  The warps' partial sums are added
// in shared memory.  Wide matrices are split over columns (grid.y splits);
// each split stores its partial tile in the workspace and the last split to
// arrive at a row tile adds the partials in split order -- deterministic and
// free of floating-point atomics.
#include "gemv_row.cuh"
#include "lak_internal.cuh"

namespace lak {
namespace {

// y = alpha * t + beta * y; y is not read when beta == 0 (it may hold anything)
template <typename T>
__device__ __forceinline__ T gemv_epilogue(typename Acc<T>::type t, typename Acc<T>::type alpha,
                                           typename Acc<T>::type beta, const T *yold) {
    using Ac = typename Acc<T>::type;
    if (beta == Ac(0)) return narrow<T>(alpha * t);
    return narrow<T>(fma_acc(alpha, t, beta * widen(*yold)));
}

// the same with the old y value already loaded (prefetched before the row's
// dot product, so the epilogue adds no dependent load)
template <typename T>
__device__ __forceinline__ T gemv_epilogue_v(typename Acc<T>::type t, typename Acc<T>::type alpha,
                                             typename Acc<T>::type beta,
                                             typename Acc<T>::type yold) {
    using Ac = typename Acc<T>::type;
    if (beta == Ac(0)) return narrow<T>(alpha * t);
    return narrow<T>(fma_acc(alpha, t, beta * yold));
}

template <typename T, int V>
__global__ void __launch_bounds__(512)
gemv_row_kernel(T *__restrict__ y, const T *__restrict__ A, const T *__restrict__ x, int64_t m,
                int64_t n, int64_t lda, int G, int inc, typename Acc<T>::type alpha,
                typename Acc<T>::type beta) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    __shared__ Ac red[32];
    const int R = blockDim.x / G;                  // rows per block step
    const int grp = threadIdx.x / G;
    const int lg = threadIdx.x % G;

    int64_t row0, row_end, step;
    if (inc == LAK_INC_GLOBAL) {
        row0 = (int64_t)blockIdx.x * R;
        row_end = m;
        step = (int64_t)gridDim.x * R;
    } else {
        int64_t per = (m + gridDim.x - 1) / gridDim.x;
        per = (per + R - 1) / R * R;
        row0 = (int64_t)blockIdx.x * per;
        row_end = row0 + per < m ? row0 + per : m;
        step = R;
    }
    for (int64_t rb = row0; rb < row_end; rb += step) {   // block-uniform trip count
        const int64_t row = rb + grp;
        Ac acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = Ac(0);
        Ac yold = Ac(0);
        if (beta != Ac(0) && lg == 0 && row < row_end) yold = widen(y[row]);
        if (row < row_end) row_group_dot<T, V>(acc, A + row * lda, x, n, lg, G);
        if constexpr (!gemv_one_chain<T>) {
#pragma unroll
            for (int w = 1; w < V; w <<= 1) {
#pragma unroll
                for (int v = 0; v + w < V; v += 2 * w) acc[v] += acc[v + w];
            }
        }
        Ac s = acc[0];
        if (G <= 32) {
            s = group_sum(s, G);
            if (lg == 0 && row < row_end) y[row] = gemv_epilogue_v<T>(s, alpha, beta, yold);
        } else {
            s = group_sum(s, 32);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
            __syncthreads();
            if (lg == 0 && row < row_end) {
                const int wpg = G >> 5;
                Ac t = Ac(0);
                for (int w = 0; w < wpg; ++w) t += red[grp * wpg + w];
                y[row] = gemv_epilogue_v<T>(t, alpha, beta, yold);
            }
            __syncthreads();
        }
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(512)
gemv_col_kernel(T *__restrict__ y, const T *__restrict__ A, const T *__restrict__ x, int64_t m,
                int64_t n, int64_t lda, int64_t cols_per_split,
                typename Acc<T>::type *__restrict__ partials, unsigned int *__restrict__ tickets,
                typename Acc<T>::type alpha, typename Acc<T>::type beta) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Ac *red = reinterpret_cast<Ac *>(smem_raw);    // [nwarps][32*V]
    __shared__ int am_last;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    constexpr int TILE = 32 * V;
    const int64_t tile0 = (int64_t)blockIdx.x * TILE;
    const int64_t r0 = tile0 + (int64_t)lane * V;
    const int split = blockIdx.y;
    const int nsplit = gridDim.y;
    const int64_t c0 = (int64_t)split * cols_per_split;
    const int64_t c1 = c0 + cols_per_split < n ? c0 + cols_per_split : n;

    Ac acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = Ac(0);
    if (r0 + V <= m) {
#pragma unroll 4
        for (int64_t j = c0 + warp; j < c1; j += nwarps) {
            Pack<T, V> pa;
            load_pack<T, V, STREAM>(pa, A + j * lda + r0);
            const T xj = ld_cached(x + j);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fma_wide(pa.e[v], xj, acc[v]);
        }
    } else if (r0 < m) {
        for (int64_t j = c0 + warp; j < c1; j += nwarps) {
            const T xj = ld_cached(x + j);
#pragma unroll
            for (int v = 0; v < V; ++v)
                if (r0 + v < m) acc[v] = fma_wide(A[j * lda + r0 + v], xj, acc[v]);
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) red[warp * TILE + lane * V + v] = acc[v];
    __syncthreads();

    for (int rr = threadIdx.x; rr < TILE; rr += blockDim.x) {
        Ac t = Ac(0);
        for (int w = 0; w < nwarps; ++w) t += red[w * TILE + rr];
        const int64_t row = tile0 + rr;
        if (row < m) {
            if (nsplit == 1)
                y[row] = gemv_epilogue<T>(t, alpha, beta, y + row);
            else
                partials[(int64_t)split * m + row] = t;
        }
    }
    if (nsplit == 1) return;

    __threadfence();                 // every writer publishes its partials
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int ticket = atomicInc(tickets + blockIdx.x, (unsigned int)nsplit - 1);
        am_last = (ticket == (unsigned int)nsplit - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    for (int rr = threadIdx.x; rr < TILE; rr += blockDim.x) {
        const int64_t row = tile0 + rr;
        if (row < m) {
            Ac t = Ac(0);
            for (int s2 = 0; s2 < nsplit; ++s2) t += __ldcg(partials + (int64_t)s2 * m + row);
            y[row] = gemv_epilogue<T>(t, alpha, beta, y + row);
        }
    }
}

template <typename T>
lak_status gemv_row_t(void *y, const void *A, const void *x, int64_t m, int64_t n, int64_t lda,
                      const Launch &L, int G, double alpha, double beta, cudaStream_t s) {
    using Ac = typename Acc<T>::type;
    T *yp = static_cast<T *>(y);
    const T *Ap = static_cast<const T *>(A);
    const T *xp = static_cast<const T *>(x);
#define LAK_ROW(VV) \
    launch_k(gemv_row_kernel<T, VV>, L.grid, L.block, 0, s, yp, Ap, xp, m, n, lda, G, L.inc, (Ac)alpha, \
                                                      (Ac)beta)
    switch (L.vec) {
    case 1: LAK_ROW(1); break;
    case 2: LAK_ROW(2); break;
    case 4: LAK_ROW(4); break;
    case 8: LAK_ROW(8); break;
    case 16: LAK_ROW(16); break;
    default: return fail(LAK_EINVAL, "dense_gemv: unsupported vec %d", L.vec);
    }
#undef LAK_ROW
    return check_launch("dense_gemv (row-major)");
}

template <typename T>
lak_status gemv_col_t(void *y, const void *A, const void *x, int64_t m, int64_t n, int64_t lda,
                      const Launch &L, int splits, void *ws, double alpha, double beta,
                      cudaStream_t s) {
    using Ac = typename Acc<T>::type;
    T *yp = static_cast<T *>(y);
    const T *Ap = static_cast<const T *>(A);
    const T *xp = static_cast<const T *>(x);
    const int64_t tiles = ceil_div(m, 32LL * L.vec);
    const int64_t cps = splits > 1 ? ceil_div(n, splits) : (n > 0 ? n : 1);
    unsigned int *tickets = static_cast<unsigned int *>(ws);     // counter area
    Ac *partials = nullptr;
    if (splits > 1)
        partials = reinterpret_cast<Ac *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
    const dim3 grid((unsigned)tiles, (unsigned)splits);
    const size_t smem = (size_t)(L.block / 32) * 32 * L.vec * sizeof(Ac);
#define LAK_COL(VV)                                                                          \
    do {                                                                                      \
        if (smem > 48 * 1024) {                                                               \
            const cudaError_t e = cudaFuncSetAttribute(                                       \
                gemv_col_kernel<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            if (e != cudaSuccess)                                                             \
                return fail(LAK_ECUDA, "dense_gemv: shared memory %zu: %s", smem,             \
                            cudaGetErrorString(e));                                           \
        }                                                                                     \
        launch_k(gemv_col_kernel<T, VV>, grid, L.block, smem, s, yp, Ap, xp, m, n, lda, cps,        \
                                                           partials, tickets, (Ac)alpha,      \
                                                           (Ac)beta);                         \
    } while (0)
    switch (L.vec) {
    case 1: LAK_COL(1); break;
    case 2: LAK_COL(2); break;
    case 4: LAK_COL(4); break;
    case 8: LAK_COL(8); break;
    case 16: LAK_COL(16); break;
    default: return fail(LAK_EINVAL, "dense_gemv: unsupported vec %d", L.vec);
    }
#undef LAK_COL
    return check_launch("dense_gemv (column-major)");
}

}  // namespace

lak_status launch_gemv_row(lak_dtype dt, void *y, const void *A, const void *x, int64_t m,
                           int64_t n, int64_t lda, const Launch &L, int group, double alpha,
                           double beta, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return gemv_row_t<float>(y, A, x, m, n, lda, L, group, alpha, beta, s);
    case LAK_F64: return gemv_row_t<double>(y, A, x, m, n, lda, L, group, alpha, beta, s);
    case LAK_BF16: return gemv_row_t<__nv_bfloat16>(y, A, x, m, n, lda, L, group, alpha, beta, s);
    case LAK_F16: return gemv_row_t<__half>(y, A, x, m, n, lda, L, group, alpha, beta, s);
    }
    return fail(LAK_EDTYPE, "dense_gemv: unknown dtype %d", (int)dt);
}

lak_status launch_gemv_col(lak_dtype dt, void *y, const void *A, const void *x, int64_t m,
                           int64_t n, int64_t lda, const Launch &L, int splits, void *ws,
                           double alpha, double beta, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return gemv_col_t<float>(y, A, x, m, n, lda, L, splits, ws, alpha, beta, s);
    case LAK_F64: return gemv_col_t<double>(y, A, x, m, n, lda, L, splits, ws, alpha, beta, s);
    case LAK_BF16:
        return gemv_col_t<__nv_bfloat16>(y, A, x, m, n, lda, L, splits, ws, alpha, beta, s);
    case LAK_F16: return gemv_col_t<__half>(y, A, x, m, n, lda, L, splits, ws, alpha, beta, s);
    }
    return fail(LAK_EDTYPE, "dense_gemv: unknown dtype %d", (int)dt);
}

}  // namespace lak
