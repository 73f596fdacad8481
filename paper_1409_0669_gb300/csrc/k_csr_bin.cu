// Row-binned CSR: the CSR arrays stay as they are; a row permutation groups
// the rows by length so that each group can be served by a lane group of the
// right width (rows of power-law length distributions otherwise put a 4-entry
// and a 256-entry row in one warp).
//
// Bin b of LAK_CSR_BINS holds the rows with L stored entries, where b is the
// smallest bin with L <= LAK_CSR_BIN_PER_LANE * 2^b, the last bin taking every
// longer row.  Within a bin rows keep their original order (a stable sort by
// bin), so the permutation is unique and the product's result does not depend
// on how the build was scheduled.
//
//   csr_bin_build  three passes over row_ptr: per-tile bin counts (integer
//                  shared-memory counters), one block scanning the counts in
//                  bin-major order, and a stable scatter using warp ballots.
//   csr_bin_spmv   one launch: every warp takes 32/G rows of one bin, G =
//                  2^min(b, 5) lanes per row; in bins 0..LAK_CSR_BINS-2 each
//                  lane needs at most LAK_CSR_BIN_PER_LANE entries, read in one
//                  step of independent loads; the last bin loops.  Lanes of a
//                  group reduce with shuffles; FP64 keeps one accumulator chain
//                  per lane (the FP64 pipe, not latency, limits it on GB300).
#include "lak_internal.cuh"

namespace lak {
namespace {

constexpr int kNB = LAK_CSR_BINS;
constexpr int kE = LAK_CSR_BIN_PER_LANE;
constexpr int kTile = 1024;                        // rows per build tile (one block)

__device__ __forceinline__ int row_bin(int64_t len) {
    int b = 0;
    while (b < kNB - 1 && len > ((int64_t)kE << b)) ++b;
    return b;
}

__global__ void __launch_bounds__(kTile)
bin_count_kernel(const int32_t *__restrict__ rp, int64_t m, int32_t *__restrict__ counts) {
    LAK_PDL_ENTRY();
    __shared__ int32_t c[kNB];
    if (threadIdx.x < kNB) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kTile + threadIdx.x;
    if (i < m) atomicAdd(&c[row_bin((int64_t)__ldg(rp + i + 1) - __ldg(rp + i))], 1);
    __syncthreads();
    if (threadIdx.x < kNB) counts[(int64_t)blockIdx.x * kNB + threadIdx.x] = c[threadIdx.x];
}

// One block: offsets[t][b] = start of bin b + rows of bin b in tiles before t,
// and bin_ptr[0..kNB].
__global__ void __launch_bounds__(1024)
bin_scan_kernel(const int32_t *__restrict__ counts, int64_t tiles, int32_t *__restrict__ offsets,
                int64_t *__restrict__ bin_ptr) {
    LAK_PDL_ENTRY();
    __shared__ int64_t total[kNB];
    __shared__ int64_t warp_sum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (threadIdx.x < kNB) total[threadIdx.x] = 0;
    __syncthreads();
    // totals per bin
    for (int b = 0; b < kNB; ++b) {
        int64_t s = 0;
        for (int64_t t = threadIdx.x; t < tiles; t += blockDim.x) s += counts[t * kNB + b];
        s = group_sum(s, 32);
        if (lane == 0) warp_sum[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t a = 0;
            for (int w = 0; w < nwarps; ++w) a += warp_sum[w];
            total[b] = a;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int64_t a = 0;
        for (int b = 0; b < kNB; ++b) {
            bin_ptr[b] = a;
            a += total[b];
        }
        bin_ptr[kNB] = a;
    }
    __syncthreads();
    // exclusive scan over tiles, bin by bin, in chunks of blockDim tiles
    for (int b = 0; b < kNB; ++b) {
        if (threadIdx.x == 0) carry = bin_ptr[b];
        __syncthreads();
        for (int64_t t0 = 0; t0 < tiles; t0 += blockDim.x) {
            const int64_t t = t0 + threadIdx.x;
            const int64_t v = t < tiles ? counts[t * kNB + b] : 0;
            int64_t incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t up = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += up;
            }
            if (lane == 31) warp_sum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                int64_t w = lane < nwarps ? warp_sum[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int64_t up = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += up;
                }
                if (lane < nwarps) warp_sum[lane] = w;     // inclusive prefix of warp sums
            }
            __syncthreads();
            const int64_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + incl - v;
            if (t < tiles) offsets[t * kNB + b] = (int32_t)before;
            __syncthreads();
            if (threadIdx.x == 0) carry += warp_sum[nwarps - 1];
            __syncthreads();
        }
    }
}

// Stable scatter: within a tile, row i's rank among the tile's rows of its
// bin counts the rows before it (earlier warps via per-warp counts, the same
// warp via a ballot).
__global__ void __launch_bounds__(kTile)
bin_scatter_kernel(const int32_t *__restrict__ rp, int64_t m, const int32_t *__restrict__ offsets,
                   int32_t *__restrict__ perm) {
    LAK_PDL_ENTRY();
    __shared__ int32_t wc[kTile / 32][kNB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kTile + threadIdx.x;
    const bool valid = i < m;
    const int b = valid ? row_bin((int64_t)__ldg(rp + i + 1) - __ldg(rp + i)) : -1;
    int my_rank_in_warp = 0;
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
        const unsigned bal = __ballot_sync(0xffffffffu, b == q);
        if (b == q) my_rank_in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wc[warp][q] = __popc(bal);
    }
    __syncthreads();
    if (valid) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wc[w][b];
        perm[offsets[(int64_t)blockIdx.x * kNB + b] + before + my_rank_in_warp] = (int32_t)i;
    }
}

// One step of a lane over its row: up to kE entries k, k + G, ... below k1,
// all loads issued before any is used.  Entry indices are unsigned 32-bit:
// nnz < 2^31 (checked on the host), so k + G * kE stays below 2^32.
template <typename T>
__device__ __forceinline__ void bin_row_step(typename Acc<T>::type (&acc)[kE], uint32_t k, uint32_t k1,
                                             int G, const int32_t *__restrict__ ci,
                                             const T *__restrict__ vals, const T *__restrict__ x) {
    using Ac = typename Acc<T>::type;
    constexpr bool one_chain = sizeof(Ac) == 8;
    int32_t col[kE];
    T val[kE];
#pragma unroll
    for (int u = 0; u < kE; ++u) {
        const uint32_t kk = k + (uint32_t)(u * G);
        if (kk < k1) {
            ld_raw<4, CACHED>(&col[u], ci + kk);
            ld_raw<(int)sizeof(T), CACHED>(&val[u], vals + kk);
        }
    }
#pragma unroll
    for (int u = 0; u < kE; ++u) {
        const uint32_t kk = k + (uint32_t)(u * G);
        if (kk < k1) {
            Ac &a = one_chain ? acc[0] : acc[u];
            a = fma_acc(widen(val[u]), widen(ld_cached(x + col[u])), a);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256, 8)
bin_spmv_kernel(T *__restrict__ y, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                const T *__restrict__ vals, const T *__restrict__ x,
                const int32_t *__restrict__ perm, const int64_t *__restrict__ bin_ptr) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    __shared__ int32_t sb[kNB + 1];
    __shared__ int32_t wpre[kNB + 1];     // first warp task of every bin
    if (threadIdx.x == 0) {
        int32_t w = 0;
        for (int b = 0; b <= kNB; ++b) sb[b] = (int32_t)bin_ptr[b];
        for (int b = 0; b < kNB; ++b) {
            wpre[b] = w;
            const int rpw = 32 >> (b < 5 ? b : 5);
            w += (sb[b + 1] - sb[b] + rpw - 1) / rpw;
        }
        wpre[kNB] = w;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int32_t wpb = blockDim.x >> 5;
    const int32_t nw = gridDim.x * wpb;
    const int32_t total_w = wpre[kNB];
    for (int64_t w = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); w < total_w; w += nw) {
        int b = 0;
        while (b < kNB - 1 && w >= wpre[b + 1]) ++b;          // warp-uniform
        const int lgG = b < 5 ? b : 5;
        const int G = 1 << lgG;
        const int lg = lane & (G - 1);
        const int32_t pos = sb[b] + (((int32_t)w - wpre[b]) << (5 - lgG)) + (lane >> lgG);
        const bool valid = pos < sb[b + 1];
        Ac acc[kE];
#pragma unroll
        for (int u = 0; u < kE; ++u) acc[u] = Ac(0);
        int32_t row = 0;
        if (valid) {
            row = __ldg(perm + pos);
            const uint32_t k1 = (uint32_t)__ldg(rp + row + 1);
            for (uint32_t k = (uint32_t)__ldg(rp + row) + (uint32_t)lg; k < k1; k += (uint32_t)(G * kE))
                bin_row_step<T>(acc, k, k1, G, ci, vals, x);
        }
        if constexpr (sizeof(Ac) != 8) {
#pragma unroll
            for (int s = 1; s < kE; s <<= 1) {
#pragma unroll
                for (int u = 0; u + s < kE; u += 2 * s) acc[u] += acc[u + s];
            }
        }
        const Ac sum = group_sum(acc[0], G);
        if (lg == 0 && valid) y[row] = narrow<T>(sum);
    }
}

int64_t tiles_of(int64_t m) { return (m + kTile - 1) / kTile; }

bool valid_dt(lak_dtype dt) {
    return dt == LAK_F32 || dt == LAK_F64 || dt == LAK_BF16 || dt == LAK_F16;
}

}  // namespace
}  // namespace lak

using namespace lak;

extern "C" {

LAK_API size_t csr_bin_workspace(int64_t m) {
    if (m < 0) return 0;
    const size_t t = (size_t)tiles_of(m);
    return (2 * t * kNB * sizeof(int32_t) + 255) / 256 * 256 + 256;
}

LAK_API lak_status csr_bin_build(int32_t *perm, int64_t *bin_ptr, const int32_t *row_ptr,
                                 int64_t m, void *workspace, size_t ws_bytes, void *stream) {
    if (m < 0 || m > 0x7fffffffLL) return fail(LAK_EINVAL, "csr_bin_build: bad m");
    if (!bin_ptr || !row_ptr) return fail(LAK_EINVAL, "csr_bin_build: NULL pointer");
    if ((uintptr_t)bin_ptr % 8) return fail(LAK_EINVAL, "csr_bin_build: bin_ptr not 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0) {
        const cudaError_t e = cudaMemsetAsync(bin_ptr, 0, (kNB + 1) * sizeof(int64_t), s);
        if (e != cudaSuccess)
            return fail(LAK_ECUDA, "csr_bin_build: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    if (!perm) return fail(LAK_EINVAL, "csr_bin_build: NULL perm");
    const size_t need = csr_bin_workspace(m);
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "csr_bin_build: workspace of %zu bytes needed, %zu given", need,
                    workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "csr_bin_build: workspace not 256-byte aligned");
    const int64_t tiles = tiles_of(m);
    if (tiles > 0x7fffffffLL) return fail(LAK_EINVAL, "csr_bin_build: too many rows");
    int32_t *counts = static_cast<int32_t *>(workspace);
    int32_t *offsets = counts + tiles * kNB;
    launch_k(bin_count_kernel, (unsigned)tiles, kTile, 0, s, row_ptr, m, counts);
    launch_k(bin_scan_kernel, 1, 1024, 0, s, counts, tiles, offsets, bin_ptr);
    launch_k(bin_scatter_kernel, (unsigned)tiles, kTile, 0, s, row_ptr, m, offsets, perm);
    return check_launch("csr_bin_build");
}

LAK_API lak_status csr_bin_spmv(void *y, const int32_t *row_ptr, const int32_t *col_idx,
                                const void *vals, const void *x, const int32_t *perm,
                                const int64_t *bin_ptr, int64_t m, int64_t n, int64_t nnz,
                                lak_dtype dtype, const lak_cfg *cfg, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "csr_bin_spmv: unknown dtype %d", (int)dtype);
    if (m < 0 || n < 0 || nnz < 0 || nnz > 0x7fffffffLL)
        return fail(LAK_EINVAL, "csr_bin_spmv: bad sizes");
    if (cfg && cfg->block != 0 && (cfg->block < 32 || cfg->block > 512 || cfg->block % 32 ||
                                   cfg->grid < 0))
        return fail(LAK_EINVAL, "csr_bin_spmv: invalid cfg");
    if (m == 0) return LAK_OK;
    if (!y || !row_ptr || !perm || !bin_ptr || (nnz > 0 && (!col_idx || !vals || !x)))
        return fail(LAK_EINVAL, "csr_bin_spmv: NULL pointer");
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int block = cfg && cfg->block ? cfg->block : 256;
    if (block > 256) return fail(LAK_EINVAL, "csr_bin_spmv: block %d > 256", block);
    cudaStream_t s = (cudaStream_t)stream;
    // every warp strides over equal shares of the tasks, so an automatic grid is
    // exactly the blocks that fit on the GPU at once (a second, partial wave
    // would run its equal shares at a fraction of the occupancy)
    auto launch = [&](auto kernel, auto *yp, auto *vp, auto *xp) -> lak_status {
        int grid = cfg && cfg->block && cfg->grid ? cfg->grid : 0;
        if (grid == 0) {
            int per_sm = 0;
            const cudaError_t e =
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
            if (e != cudaSuccess || per_sm < 1)
                return fail(LAK_ECUDA, "csr_bin_spmv: occupancy query failed");
            grid = per_sm * di->sms;
        }
        launch_k(kernel, grid, block, 0, s, yp, row_ptr, col_idx, vp, xp, perm, bin_ptr);
        return check_launch("csr_bin_spmv");
    };
#define LAK_BIN(T)                                                                               \
    return launch(bin_spmv_kernel<T>, static_cast<T *>(y), static_cast<const T *>(vals),          \
                  static_cast<const T *>(x))
    switch (dtype) {
    case LAK_F32: LAK_BIN(float);
    case LAK_F64: LAK_BIN(double);
    case LAK_BF16: LAK_BIN(__nv_bfloat16);
    case LAK_F16: LAK_BIN(__half);
    }
#undef LAK_BIN
    return LAK_EDTYPE;
}

}  // extern "C"
