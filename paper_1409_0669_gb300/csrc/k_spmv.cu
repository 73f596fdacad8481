// CSR sparse matrix-vector product y = A x (the textbook product; the paper
// leaves sparse formats out of its study, Sec. 1).  Two kernels, three
// variants chosen on the host from the mean row length:
//
// Group per row (spmv_kernel): a group of G lanes (a power of two <= 32) owns
// one row; the lanes stride through the row's stored entries G at a time,
// each issuing U independent loads per step before using any of them,
// multiply by the gathered x[col] (cached load: neighbouring rows share x
// entries), and the group reduces with shuffles.  Short rows (stencils, mean
// <= 12) take one or two lanes per row with U covering the row, so a warp
// keeps 16-32 rows' loads in flight; their col_idx / vals loads are strided
// across the warp and go through L1 (one miss brings the lines the next lanes
// need).  Long rows (mean > 64) take more lanes per row and stream col_idx /
// vals past L1.  In FP64 each lane keeps one accumulator chain.
//
// Warp-segmented (spmv_seg_kernel, 13 <= mean <= 64): a warp owns 32
// consecutive rows, whose entries are contiguous, and walks them in chunks of
// 32*U entries with coalesced (16-byte when aligned) loads; rows that cross
// lanes are joined by a segmented shuffle scan, rows that cross chunks in a
// per-warp shared accumulator with one writer per row per chunk -- no atomics,
// deterministic (the body lives in spmv_seg.cuh, shared with the batched
// kernel).
#include "lak_internal.cuh"
#include "spmv_seg.cuh"

namespace lak {
namespace {

template <typename T, int U, int P>
__global__ void __launch_bounds__(512)
spmv_kernel(T *__restrict__ y, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
            const T *__restrict__ vals, const T *__restrict__ x, int64_t m, int G, int inc) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    const int R = blockDim.x / G;
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
        Ac acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) acc[u] = Ac(0);
        if (row < row_end) {
            const int64_t k0 = __ldg(rp + row);
            const int64_t k1 = __ldg(rp + row + 1);
            for (int64_t k = k0 + lg; k < k1; k += (int64_t)G * U) {
                int32_t col[U];
                T val[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t kk = k + (int64_t)u * G;
                    if (kk < k1) {
                        ld_raw<4, P>(&col[u], ci + kk);
                        ld_raw<(int)sizeof(T), P>(&val[u], vals + kk);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t kk = k + (int64_t)u * G;
                    // FP64: one chain (GB300's FP64 pipe, not latency, is the limit,
                    // and U partial sums would cost U - 1 extra adds per row)
                    constexpr bool one_chain = sizeof(Ac) == 8;
                    if (kk < k1) {
                        Ac &a = one_chain ? acc[0] : acc[u];
                        a = fma_acc(widen(val[u]), widen(ld_cached(x + col[u])), a);
                    }
                }
            }
        }
        if constexpr (sizeof(Ac) != 8) {
#pragma unroll
            for (int w = 1; w < U; w <<= 1) {
#pragma unroll
                for (int u = 0; u + w < U; u += 2 * w) acc[u] += acc[u + w];
            }
        }
        const Ac s = group_sum(acc[0], G);
        if (lg == 0 && row < row_end) y[row] = narrow<T>(s);
    }
}

// Warp-segmented variant: the 32-row block body lives in spmv_seg.cuh (shared
// with the batched kernel); this kernel hands each warp its 32-row blocks.
template <typename T, int U, bool VLOAD, int WMAX = 16>
__global__ void __launch_bounds__(512)
spmv_seg_kernel(T *__restrict__ y, const int32_t *__restrict__ rp,
                const int32_t *__restrict__ ci, const T *__restrict__ vals,
                const T *__restrict__ x, int64_t m, int inc) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    uint32_t *rs_w;
    Ac *racc_w;
    if constexpr (sizeof(Ac) == 8) {
        __shared__ uint32_t rs_all[WMAX][33];
        __shared__ Ac racc_all[WMAX][32];
        rs_w = rs_all[warp];
        racc_w = racc_all[warp];
    } else {
        // sized to the block's warps (the launch passes the bytes), which leaves
        // more of the unified L1 to the x gathers: FP32 power-law 142.0 -> 140.0-
        // 141.0 us.  FP64 keeps static arrays, sized for WMAX warps (2 for its
        // 64-thread default blocks: 178.8 -> 176.8 us); the dynamic form cost it
        // two registers and 2 % (178.9 -> 182.9 us).
        extern __shared__ __align__(16) unsigned char seg_smem[];
        racc_w = reinterpret_cast<Ac *>(seg_smem) + (size_t)warp * 32;
        rs_w = reinterpret_cast<uint32_t *>(seg_smem + (size_t)wpb * 32 * sizeof(Ac)) + (size_t)warp * 33;
    }
    const int64_t nrb = (m + 31) / 32;               // 32-row blocks
    const int64_t gw = (int64_t)blockIdx.x * wpb + warp;
    const int64_t nw = (int64_t)gridDim.x * wpb;
    int64_t b0, b_end, b_step;
    if (inc == LAK_INC_GLOBAL) {
        b0 = gw;
        b_end = nrb;
        b_step = nw;
    } else {
        const int64_t per = (nrb + nw - 1) / nw;
        b0 = gw * per;
        b_end = b0 + per < nrb ? b0 + per : nrb;
        b_step = 1;
    }
    const int64_t nnz = __ldg(rp + m);
    for (int64_t b = b0; b < b_end; b += b_step)     // warp-uniform trip count
        seg_rows32<T, U, VLOAD>(y, rp, ci, vals, x, m, nnz, b, rs_w, racc_w);
}

template <typename T, int U>
lak_status spmv_seg_launch(T *yp, const int32_t *rp, const int32_t *ci, const T *vp,
                           const T *xp, int64_t m, const Launch &L, cudaStream_t s) {
    const bool vload = U % 4 == 0 && (uintptr_t)ci % 16 == 0 && (uintptr_t)vp % 16 == 0;
    using Ac = typename Acc<T>::type;
    const size_t smem = sizeof(Ac) == 8 ? 0 : (size_t)(L.block / 32) * (32 * sizeof(Ac) + 33 * 4);
    if constexpr (U % 4 == 0) {
        if (vload) {
            if (sizeof(Ac) == 8 && L.block <= 64)
                launch_k(spmv_seg_kernel<T, U, true, 2>, L.grid, L.block, smem, s, yp, rp, ci, vp, xp, m, L.inc);
            else
                launch_k(spmv_seg_kernel<T, U, true>, L.grid, L.block, smem, s, yp, rp, ci, vp, xp, m, L.inc);
            return check_launch("csr_spmv (warp-segmented)");
        }
    }
    launch_k(spmv_seg_kernel<T, U, false>, L.grid, L.block, smem, s, yp, rp, ci, vp, xp, m, L.inc);
    return check_launch("csr_spmv (warp-segmented)");
}

template <typename T>
lak_status spmv_t(void *y, const int32_t *rp, const int32_t *ci, const void *vals, const void *x,
                  int64_t m, const Launch &L, int G, cudaStream_t s) {
    T *yp = static_cast<T *>(y);
    const T *vp = static_cast<const T *>(vals);
    const T *xp = static_cast<const T *>(x);
    if (G == 0) {
        switch (L.vec) {
        case 1: return spmv_seg_launch<T, 1>(yp, rp, ci, vp, xp, m, L, s);
        case 2: return spmv_seg_launch<T, 2>(yp, rp, ci, vp, xp, m, L, s);
        case 4: return spmv_seg_launch<T, 4>(yp, rp, ci, vp, xp, m, L, s);
        case 8: return spmv_seg_launch<T, 8>(yp, rp, ci, vp, xp, m, L, s);
        case 16: return spmv_seg_launch<T, 16>(yp, rp, ci, vp, xp, m, L, s);
        default: return fail(LAK_EINVAL, "csr_spmv: unsupported vec %d", L.vec);
        }
    }
#define LAK_SPMV(UU)                                                                      \
    do {                                                                                  \
        if (G <= 4)                                                                       \
            launch_k(spmv_kernel<T, UU, CACHED>, L.grid, L.block, 0, s, yp, rp, ci, vp, xp, m, G, \
                                                                  L.inc);                 \
        else                                                                              \
            launch_k(spmv_kernel<T, UU, STREAM>, L.grid, L.block, 0, s, yp, rp, ci, vp, xp, m, G, \
                                                                  L.inc);                 \
    } while (0)
    switch (L.vec) {
    case 1: LAK_SPMV(1); break;
    case 2: LAK_SPMV(2); break;
    case 4: LAK_SPMV(4); break;
    case 8: LAK_SPMV(8); break;
    case 16: LAK_SPMV(16); break;
    default: return fail(LAK_EINVAL, "csr_spmv: unsupported vec %d", L.vec);
    }
#undef LAK_SPMV
    return check_launch("csr_spmv");
}

}  // namespace

lak_status launch_spmv(lak_dtype dt, void *y, const int32_t *rp, const int32_t *ci,
                       const void *vals, const void *x, int64_t m, const Launch &L, int group,
                       cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return spmv_t<float>(y, rp, ci, vals, x, m, L, group, s);
    case LAK_F64: return spmv_t<double>(y, rp, ci, vals, x, m, L, group, s);
    case LAK_BF16: return spmv_t<__nv_bfloat16>(y, rp, ci, vals, x, m, L, group, s);
    case LAK_F16: return spmv_t<__half>(y, rp, ci, vals, x, m, L, group, s);
    }
    return fail(LAK_EDTYPE, "csr_spmv: unknown dtype %d", (int)dt);
}

}  // namespace lak
