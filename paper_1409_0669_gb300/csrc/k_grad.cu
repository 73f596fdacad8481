// Kernels for the reverse-mode derivatives of the products, and their C ABI:
//   dense_outer        dA = dy x^T                (gradient of y = A x w.r.t. A)
//   csr_sampled_outer  dvals[k] = dy[row(k)] * x[col(k)]   (same, on a CSR pattern)
//   csr_transpose      CSC form of a CSR pattern (+ the value permutation), so
//                      that A^T dy is a CSR product with no atomics
//   vec_gather         dst[i] = src[idx[i]]       (values into CSC order)
//   vec_scale_dev      out = alpha * v, alpha read from device memory
//                      (gradient of <x, y>: dx = ds * y without a host sync)
#include "lak_internal.cuh"

namespace lak {
namespace {

// ---- dense outer product --------------------------------------------------------

// Grid (column blocks) x (row groups): each block owns a contiguous range of
// rows and each thread a V-wide chunk of columns; the thread keeps its chunk
// of x in registers and writes dy[i] times it into every row of the range, so
// the row loop holds no dependent global load (dy[i] is one broadcast L1 hit)
// and is bound by the stores alone.
template <typename T, int V>
__global__ void __launch_bounds__(512)
outer_kernel(T *__restrict__ dA, const T *__restrict__ dy, const T *__restrict__ x, int64_t m,
             int64_t n, int64_t ldd, bool vec_ok) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    const int64_t rows_per = (m + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per;
    const int64_t r1 = r0 + rows_per < m ? r0 + rows_per : m;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tstride = (int64_t)gridDim.x * blockDim.x;
    if (vec_ok) {
        const int64_t nch = n / V;
        for (int64_t c = t; c < nch; c += tstride) {
            Pack<T, V> px;
            load_pack<T, V, CACHED>(px, x + c * V);
            A xv[V];
#pragma unroll
            for (int v = 0; v < V; ++v) xv[v] = widen(px.e[v]);
#pragma unroll 4
            for (int64_t i = r0; i < r1; ++i) {
                const A d = widen(__ldg(dy + i));
                Pack<T, V> po;
#pragma unroll
                for (int v = 0; v < V; ++v) po.e[v] = narrow<T>(d * xv[v]);
                store_pack<T, V>(dA + i * ldd + c * V, po);
            }
        }
        for (int64_t j = nch * V + t; j < n; j += tstride) {
            const A xj = widen(x[j]);
            for (int64_t i = r0; i < r1; ++i) dA[i * ldd + j] = narrow<T>(widen(dy[i]) * xj);
        }
    } else {
        for (int64_t j = t; j < n; j += tstride) {
            const A xj = widen(x[j]);
            for (int64_t i = r0; i < r1; ++i) dA[i * ldd + j] = narrow<T>(widen(dy[i]) * xj);
        }
    }
}

// ---- CSR sampled outer product ------------------------------------------------------

// A group of G lanes per row (G from the mean row length): the lanes of a
// group write consecutive entries of the row, so the stores and the col_idx
// loads of a warp stay contiguous.
template <typename T, int G>
__global__ void __launch_bounds__(512)
sampled_outer_kernel(T *__restrict__ dvals, const int32_t *__restrict__ rp,
                     const int32_t *__restrict__ ci, const T *__restrict__ dy,
                     const T *__restrict__ x, int64_t m) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    const int lg = threadIdx.x % G;
    const int64_t groups = ((int64_t)gridDim.x * blockDim.x) / G;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < m; i += groups) {
        const A d = widen(dy[i]);
        const int64_t k1 = __ldg(rp + i + 1);
        for (int64_t k = __ldg(rp + i) + lg; k < k1; k += G)
            dvals[k] = narrow<T>(d * widen(ld_cached(x + __ldg(ci + k))));
    }
}

// ---- CSR -> CSC ---------------------------------------------------------------------

__global__ void count_cols_kernel(int32_t *__restrict__ counts, const int32_t *__restrict__ ci,
                                  int64_t nnz) {
    LAK_PDL_ENTRY();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + __ldg(ci + k), 1);      // integer: order-independent
}

constexpr int kScanBlock = 512;
constexpr int kScanPer = 8;                         // elements per thread
constexpr int64_t kScanTile = (int64_t)kScanBlock * kScanPer;

// Inclusive scan of v[0..len) in tiles; tile totals to sums[tile].
__global__ void __launch_bounds__(kScanBlock)
scan_tiles_kernel(int32_t *__restrict__ v, int64_t len, int32_t *__restrict__ sums) {
    LAK_PDL_ENTRY();
    __shared__ int32_t warp_tot[kScanBlock / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int32_t loc[kScanPer];
    int32_t run = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        const int64_t k = base + e;
        run += k < len ? v[k] : 0;
        loc[e] = run;
    }
    // exclusive scan of the per-thread totals across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t t = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t up = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += up;
    }
    if (lane == 31) warp_tot[warp] = t;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < kScanBlock / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t up = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += up;
        }
        if (lane < kScanBlock / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    const int32_t before = (t - run) + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
        const int64_t k = base + e;
        if (k < len) v[k] = loc[e] + before;
    }
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = before + run;
}

// Adds the inclusive prefix of earlier tiles' totals (sums already scanned).
__global__ void add_tile_offsets_kernel(int32_t *__restrict__ v, int64_t len,
                                        const int32_t *__restrict__ sums_scanned) {
    LAK_PDL_ENTRY();
    const int64_t tile = blockIdx.x;
    if (tile == 0) return;
    const int32_t off = sums_scanned[tile - 1];
    for (int64_t k = tile * kScanTile + threadIdx.x; k < (tile + 1) * kScanTile && k < len;
         k += blockDim.x)
        v[k] += off;
}

__global__ void copy_i32_kernel(int32_t *__restrict__ dst, const int32_t *__restrict__ src,
                                int64_t len) {
    LAK_PDL_ENTRY();
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < len;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[k];
}

__global__ void scatter_kernel(int32_t *__restrict__ row_idx, int32_t *__restrict__ perm,
                               int32_t *__restrict__ cursor, const int32_t *__restrict__ rp,
                               const int32_t *__restrict__ ci, int64_t m) {
    LAK_PDL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k1 = rp[i + 1];
        for (int64_t k = rp[i]; k < k1; ++k) {
            const int32_t q = atomicAdd(cursor + ci[k], 1);
            row_idx[q] = (int32_t)i;
            perm[q] = (int32_t)k;
        }
    }
}

// Orders every column's entries by CSR position (= by row, and by position
// inside a row): the result of a stable counting sort, independent of the
// order in which the scatter's atomics were served.
__global__ void sort_columns_kernel(int32_t *__restrict__ row_idx, int32_t *__restrict__ perm,
                                    const int32_t *__restrict__ cp, int64_t n) {
    LAK_PDL_ENTRY();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = cp[j], b = cp[j + 1];
        for (int64_t q = a + 1; q < b; ++q) {
            const int32_t pk = perm[q], rk = row_idx[q];
            int64_t t = q - 1;
            while (t >= a && perm[t] > pk) {
                perm[t + 1] = perm[t];
                row_idx[t + 1] = row_idx[t];
                --t;
            }
            perm[t + 1] = pk;
            row_idx[t + 1] = rk;
        }
    }
}

// ---- gather and device-scalar scaling ---------------------------------------------

template <typename E>
__global__ void gather_kernel(E *__restrict__ dst, const E *__restrict__ src,
                              const int32_t *__restrict__ idx, int64_t n) {
    LAK_PDL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[__ldg(idx + i)];
}

template <typename T, typename S>
__global__ void scale_dev_kernel(T *__restrict__ out, const T *__restrict__ v,
                                 const S *__restrict__ alpha, int64_t n) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    const A a = static_cast<A>(*alpha);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = narrow<T>(a * widen(v[i]));
}

int grid_for(int64_t work, int block) {
    const DeviceInfo *di = device_info();
    int64_t cap = di ? (int64_t)di->sms * (di->max_threads_per_sm / block) : 1024;
    int64_t g = (work + block - 1) / block;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T>
lak_status outer_t(void *dA, const void *dy, const void *x, int64_t m, int64_t n, int64_t ldd,
                   cudaStream_t s) {
    constexpr int V = 32 / (int)sizeof(T) > 8 ? 8 : 32 / (int)sizeof(T);
    const int w = V * (int)sizeof(T);
    const bool vec_ok = (uintptr_t)dA % w == 0 && (uintptr_t)x % w == 0 &&
                        (ldd * (int64_t)sizeof(T)) % w == 0;
    // a few column blocks per row, and enough row groups to fill the GPU about
    // twice; every block then walks many rows (long-lived blocks)
    const int block = 256;
    int64_t gx = (n / V + block - 1) / block;
    if (gx < 1) gx = 1;
    if (gx > 64) gx = 64;
    const DeviceInfo *di = device_info();
    const int64_t cap = di ? 2LL * di->sms * (di->max_threads_per_sm / block) : 2048;
    int64_t gy = cap / gx;
    if (gy < 1) gy = 1;
    if (gy > m) gy = m;
    if (gy > 65535) gy = 65535;
    launch_k(outer_kernel<T, V>, dim3((unsigned)gx, (unsigned)gy), block, 0, s, 
        static_cast<T *>(dA), static_cast<const T *>(dy), static_cast<const T *>(x), m, n, ldd,
        vec_ok);
    return check_launch("dense_outer");
}

bool valid_dt(lak_dtype dt) { return dt == LAK_F32 || dt == LAK_F64 || dt == LAK_BF16 || dt == LAK_F16; }

}  // namespace
}  // namespace lak

using namespace lak;

extern "C" {

LAK_API lak_status dense_outer(void *dA, const void *dy, const void *x, int64_t m, int64_t n,
                               int64_t ldd, lak_dtype dtype, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "dense_outer: unknown dtype %d", (int)dtype);
    if (m < 0 || n < 0) return fail(LAK_EINVAL, "dense_outer: negative size");
    if (ldd < (n > 1 ? n : 1)) return fail(LAK_EINVAL, "dense_outer: ldd=%lld < n", (long long)ldd);
    if (m == 0 || n == 0) return LAK_OK;
    if (!dA || !dy || !x) return fail(LAK_EINVAL, "dense_outer: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
    case LAK_F32: return outer_t<float>(dA, dy, x, m, n, ldd, s);
    case LAK_F64: return outer_t<double>(dA, dy, x, m, n, ldd, s);
    case LAK_BF16: return outer_t<__nv_bfloat16>(dA, dy, x, m, n, ldd, s);
    case LAK_F16: return outer_t<__half>(dA, dy, x, m, n, ldd, s);
    }
    return LAK_EDTYPE;
}

LAK_API lak_status csr_sampled_outer(void *dvals, const int32_t *row_ptr, const int32_t *col_idx,
                                     const void *dy, const void *x, int64_t m, int64_t nnz,
                                     lak_dtype dtype, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "csr_sampled_outer: unknown dtype %d", (int)dtype);
    if (m < 0 || nnz < 0) return fail(LAK_EINVAL, "csr_sampled_outer: negative size");
    if (m == 0 || nnz == 0) return LAK_OK;
    if (!dvals || !row_ptr || !col_idx || !dy || !x)
        return fail(LAK_EINVAL, "csr_sampled_outer: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    const int64_t mean = (nnz + m - 1) / m;
    // short rows (stencils): a thread per row reads its few col_idx from one
    // cache line; longer rows: a group of about half the mean row length
    const int G = mean <= 12 ? 1 : mean <= 16 ? 8 : mean <= 32 ? 16 : 32;
    const int grid = grid_for(m * G, block);
#define LAK_SOG(T, GG)                                                                         \
    launch_k(sampled_outer_kernel<T, GG>, grid, block, 0, s, static_cast<T *>(dvals), row_ptr, col_idx, \
                                                       static_cast<const T *>(dy),              \
                                                       static_cast<const T *>(x), m)
#define LAK_SO(T)                     \
    switch (G) {                      \
    case 1: LAK_SOG(T, 1); break;     \
    case 8: LAK_SOG(T, 8); break;     \
    case 16: LAK_SOG(T, 16); break;   \
    default: LAK_SOG(T, 32); break;   \
    }
    switch (dtype) {
    case LAK_F32: LAK_SO(float); break;
    case LAK_F64: LAK_SO(double); break;
    case LAK_BF16: LAK_SO(__nv_bfloat16); break;
    case LAK_F16: LAK_SO(__half); break;
    }
#undef LAK_SO
#undef LAK_SOG
    return check_launch("csr_sampled_outer");
}

LAK_API size_t csr_transpose_workspace(int64_t n) {
    if (n < 0) return 0;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    // cursor (n) + tile sums + sums of tile sums, all int32, 256-byte sections
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const int64_t tiles2 = (tiles + kScanTile - 1) / kScanTile;
    return up((size_t)n * 4) + up((size_t)tiles * 4) + up((size_t)tiles2 * 4) + 256;
}

LAK_API lak_status csr_transpose(int32_t *col_ptr, int32_t *row_idx, int32_t *perm,
                                 const int32_t *row_ptr, const int32_t *col_idx, int64_t m,
                                 int64_t n, int64_t nnz, void *workspace, size_t ws_bytes,
                                 void *stream) {
    if (m < 0 || n < 0 || nnz < 0 || nnz > 0x7fffffffLL)
        return fail(LAK_EINVAL, "csr_transpose: bad sizes");
    if (!col_ptr) return fail(LAK_EINVAL, "csr_transpose: NULL col_ptr");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(col_ptr, 0, (size_t)(n + 1) * 4, s);
    if (e != cudaSuccess) return fail(LAK_ECUDA, "csr_transpose: memset: %s", cudaGetErrorString(e));
    if (n == 0 || nnz == 0) return LAK_OK;
    if (!row_ptr || !col_idx || !row_idx || !perm)
        return fail(LAK_EINVAL, "csr_transpose: NULL pointer");
    const size_t need = csr_transpose_workspace(n);
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "csr_transpose: workspace of %zu bytes needed, %zu given", need,
                    workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "csr_transpose: workspace not 256-byte aligned");
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    const int64_t tiles2 = (tiles + kScanTile - 1) / kScanTile;
    char *w = static_cast<char *>(workspace);
    int32_t *cursor = reinterpret_cast<int32_t *>(w);
    int32_t *sums = reinterpret_cast<int32_t *>(w + up((size_t)n * 4));
    int32_t *sums2 = reinterpret_cast<int32_t *>(w + up((size_t)n * 4) + up((size_t)tiles * 4));
    if (tiles2 > kScanTile)
        return fail(LAK_EINVAL, "csr_transpose: n = %lld is beyond the two-level scan",
                    (long long)n);
    const int block = 256;
    // counts land in col_ptr[1..n]
    launch_k(count_cols_kernel, grid_for(nnz, block), block, 0, s, col_ptr + 1, col_idx, nnz);
    // inclusive scan of col_ptr[1..n] -> col_ptr[j+1] = entries in columns <= j
    launch_k(scan_tiles_kernel, (unsigned)tiles, kScanBlock, 0, s, col_ptr + 1, n, sums);
    if (tiles > 1) {
        launch_k(scan_tiles_kernel, (unsigned)tiles2, kScanBlock, 0, s, sums, tiles, sums2);
        if (tiles2 > 1) {
            launch_k(scan_tiles_kernel, 1, kScanBlock, 0, s, sums2, tiles2, sums2 + tiles2);
            launch_k(add_tile_offsets_kernel, (unsigned)tiles2, 256, 0, s, sums, tiles, sums2);
        }
        launch_k(add_tile_offsets_kernel, (unsigned)tiles, 256, 0, s, col_ptr + 1, n, sums);
    }
    launch_k(copy_i32_kernel, grid_for(n, block), block, 0, s, cursor, col_ptr, n);
    launch_k(scatter_kernel, grid_for(m, block), block, 0, s, row_idx, perm, cursor, row_ptr, col_idx, m);
    launch_k(sort_columns_kernel, grid_for(n, block), block, 0, s, row_idx, perm, col_ptr, n);
    return check_launch("csr_transpose");
}

LAK_API lak_status vec_gather(void *dst, const void *src, const int32_t *idx, int64_t n,
                              lak_dtype dtype, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "vec_gather: unknown dtype %d", (int)dtype);
    if (n < 0) return fail(LAK_EINVAL, "vec_gather: n < 0");
    if (n == 0) return LAK_OK;
    if (!dst || !src || !idx) return fail(LAK_EINVAL, "vec_gather: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    const int grid = grid_for(n, block);
    switch (esize(dtype)) {
    case 2: launch_k(gather_kernel<uint16_t>, grid, block, 0, s, (uint16_t *)dst, (const uint16_t *)src, idx, n); break;
    case 4: launch_k(gather_kernel<uint32_t>, grid, block, 0, s, (uint32_t *)dst, (const uint32_t *)src, idx, n); break;
    case 8: launch_k(gather_kernel<uint64_t>, grid, block, 0, s, (uint64_t *)dst, (const uint64_t *)src, idx, n); break;
    }
    return check_launch("vec_gather");
}

LAK_API lak_status vec_scale_dev(void *out, const void *v, const void *alpha, int64_t n,
                                 lak_dtype dtype, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "vec_scale_dev: unknown dtype %d", (int)dtype);
    if (n < 0) return fail(LAK_EINVAL, "vec_scale_dev: n < 0");
    if (n == 0) return LAK_OK;
    if (!out || !v || !alpha) return fail(LAK_EINVAL, "vec_scale_dev: NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    const int grid = grid_for(n, block);
    switch (dtype) {
    case LAK_F32: launch_k(scale_dev_kernel<float, float>, grid, block, 0, s, (float *)out, (const float *)v, (const float *)alpha, n); break;
    case LAK_F64: launch_k(scale_dev_kernel<double, double>, grid, block, 0, s, (double *)out, (const double *)v, (const double *)alpha, n); break;
    case LAK_BF16: launch_k(scale_dev_kernel<__nv_bfloat16, float>, grid, block, 0, s, (__nv_bfloat16 *)out, (const __nv_bfloat16 *)v, (const float *)alpha, n); break;
    case LAK_F16: launch_k(scale_dev_kernel<__half, float>, grid, block, 0, s, (__half *)out, (const __half *)v, (const float *)alpha, n); break;
    }
    return check_launch("vec_scale_dev");
}

}  // extern "C"
