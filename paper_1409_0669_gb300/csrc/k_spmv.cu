// CSR sparse matrix-vector product y = A x (the textbook product; the paper
// leaves sparse formats out of its study, Sec. 1).
//
// A group of G lanes (G a power of two <= 32, chosen on the host from the mean
// row length) owns one row: the lanes stride through the row's stored entries
// G at a time, each issuing U independent loads per step, multiply by the
// gathered x[col] (cached load: neighbouring rows share x entries), and the
// group reduces with shuffles.  Short rows (the Laplacian stencils) use a few
// lanes so that one warp covers several consecutive rows and its loads of
// col_idx / vals stay contiguous; long rows use the whole warp.
#include "lak_internal.cuh"

namespace lak {
namespace {

template <typename T, int U>
__global__ void __launch_bounds__(512)
spmv_kernel(T *__restrict__ y, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
            const T *__restrict__ vals, const T *__restrict__ x, int64_t m, int G, int inc) {
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
                        ld_raw<4, STREAM>(&col[u], ci + kk);
                        ld_raw<(int)sizeof(T), STREAM>(&val[u], vals + kk);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int64_t kk = k + (int64_t)u * G;
                    if (kk < k1) acc[u] = fma_acc(widen(val[u]), widen(ld_cached(x + col[u])), acc[u]);
                }
            }
        }
#pragma unroll
        for (int w = 1; w < U; w <<= 1) {
#pragma unroll
            for (int u = 0; u + w < U; u += 2 * w) acc[u] += acc[u + w];
        }
        const Ac s = group_sum(acc[0], G);
        if (lg == 0 && row < row_end) y[row] = narrow<T>(s);
    }
}

template <typename T>
lak_status spmv_t(void *y, const int32_t *rp, const int32_t *ci, const void *vals, const void *x,
                  int64_t m, const Launch &L, int G, cudaStream_t s) {
    T *yp = static_cast<T *>(y);
    const T *vp = static_cast<const T *>(vals);
    const T *xp = static_cast<const T *>(x);
#define LAK_SPMV(UU) spmv_kernel<T, UU><<<L.grid, L.block, 0, s>>>(yp, rp, ci, vp, xp, m, G, L.inc)
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
