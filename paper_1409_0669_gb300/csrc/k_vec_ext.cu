// Vector-operation variants built on the same loop skeletons as k_vec.cu:
//   vec_axpby          x = alpha*y + beta*z      (Sec. 2's scaled vector addition
//                                                 in its general form)
//   vec_axpby_strided  the same on strided vectors (element i at p + i*inc)
//   vec_axpy_norm2     x = y + alpha*z and s = <x, x> in one pass (the update
//                      and the squared norm of its result, reading y and z once
//                      and never re-reading x)
//   vec_dot_sparse     s = sum_k vals[k] * y[idx[k]]: the inner product of a
//                      sparse vector (stored values and their indices) with a
//                      dense one -- the gather-bound core of every CSR row
#include "lak_internal.cuh"
#include "vec_loop.cuh"

namespace lak {
namespace {

template <typename T, int V>
__global__ void __launch_bounds__(512)
axpby_kernel(T *x, typename Acc<T>::type alpha, const T *y, typename Acc<T>::type beta,
             const T *z, int64_t n, int64_t head, int64_t nchunks, int inc) {
    LAK_PDL_ENTRY();
    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        const int64_t o = head + c * V;
        Pack<T, V> py, pz, px;
        load_pack<T, V, COHERENT>(py, y + o);
        load_pack<T, V, COHERENT>(pz, z + o);
#pragma unroll
        for (int v = 0; v < V; ++v)
            px.e[v] = narrow<T>(fma_acc(alpha, widen(py.e[v]), beta * widen(pz.e[v])));
        store_pack<T, V>(x + o, px);
    }
    const int64_t body_end = head + nchunks * V;
    const int64_t nextra = head + (n - body_end);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nextra) {
        const int64_t i = extra_index(t, head, body_end);
        x[i] = narrow<T>(fma_acc(alpha, widen(y[i]), beta * widen(z[i])));
    }
}

template <typename T>
__global__ void __launch_bounds__(512)
axpby_strided_kernel(T *x, int64_t incx, typename Acc<T>::type alpha, const T *y, int64_t incy,
                     typename Acc<T>::type beta, const T *z, int64_t incz, int64_t n) {
    LAK_PDL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i * incx] = narrow<T>(fma_acc(alpha, widen(y[i * incy]), beta * widen(z[i * incz])));
}

// x = y + alpha*z; s = sum x_i^2 of the STORED x (after rounding to the storage
// type), reduced like dot_kernel: per-thread accumulators, warp shuffles, FP64
// block partials, last block combines in block order.
template <typename T, int V>
__global__ void __launch_bounds__(512, 2)     // two 512-thread blocks per SM
axpy_norm2_kernel(T *x, const T *y, const T *z, typename Acc<T>::type alpha, void *out,
                  int64_t n, int64_t head, int64_t nchunks, int inc, unsigned int *counter,
                  double *partials) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    A acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = A(0);
    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        const int64_t o = head + c * V;
        Pack<T, V> py, pz, px;
        load_pack<T, V, COHERENT>(py, y + o);
        load_pack<T, V, COHERENT>(pz, z + o);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            px.e[v] = narrow<T>(fma_acc(alpha, widen(pz.e[v]), widen(py.e[v])));
            const A xv = widen(px.e[v]);
            acc[v] = fma_acc(xv, xv, acc[v]);
        }
        store_pack<T, V>(x + o, px);
    }
    {
        const int64_t body_end = head + nchunks * V;
        const int64_t nextra = head + (n - body_end);
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (t < nextra) {
            const int64_t i = extra_index(t, head, body_end);
            const T xi = narrow<T>(fma_acc(alpha, widen(z[i]), widen(y[i])));
            x[i] = xi;
            acc[0] = fma_acc(widen(xi), widen(xi), acc[0]);
        }
    }
#pragma unroll
    for (int w = 1; w < V; w <<= 1) {
#pragma unroll
        for (int v = 0; v + w < V; v += 2 * w) acc[v] += acc[v + w];
    }
    if constexpr (sizeof(A) == 8)
        grid_sum_last_block(acc[0], static_cast<double *>(out), counter, partials);
    else
        grid_sum_last_block(acc[0], static_cast<float *>(out), counter, partials);
}

// Sparse inner product: the values and indices stream in V-wide packs (the
// loop skeleton of dot_kernel), each index gathers one element of y through
// L1, and the sum is finished like dot_kernel's.
template <typename T, int V>
__global__ void __launch_bounds__(512)
dot_sparse_kernel(void *out, const T *__restrict__ vals, const int32_t *__restrict__ idx,
                  const T *__restrict__ y, int64_t nnz, int64_t head, int64_t nchunks, int inc,
                  unsigned int *counter, double *partials) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    A acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = A(0);
    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        const int64_t o = head + c * V;
        Pack<T, V> pv;
        Pack<int32_t, V> pi;
        load_pack<T, V, STREAM>(pv, vals + o);
        load_pack<int32_t, V, STREAM>(pi, idx + o);
#pragma unroll
        for (int v = 0; v < V; ++v)
            acc[v] = fma_acc(widen(pv.e[v]), widen(ld_cached(y + pi.e[v])), acc[v]);
    }
    {
        const int64_t body_end = head + nchunks * V;
        const int64_t nextra = head + (nnz - body_end);
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (t < nextra) {
            const int64_t k = extra_index(t, head, body_end);
            acc[0] = fma_acc(widen(vals[k]), widen(ld_cached(y + idx[k])), acc[0]);
        }
    }
#pragma unroll
    for (int w = 1; w < V; w <<= 1) {
#pragma unroll
        for (int v = 0; v + w < V; v += 2 * w) acc[v] += acc[v + w];
    }
    if constexpr (sizeof(A) == 8)
        grid_sum_last_block(acc[0], static_cast<double *>(out), counter, partials);
    else
        grid_sum_last_block(acc[0], static_cast<float *>(out), counter, partials);
}

template <typename T>
lak_status dot_sparse_t(void *out, const void *vals, const int32_t *idx, const void *y,
                        int64_t nnz, int64_t head, void *ws, const Launch &L, cudaStream_t s) {
    const T *vp = static_cast<const T *>(vals);
    const T *yp = static_cast<const T *>(y);
    unsigned int *counter = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
    const int64_t nchunks = (nnz - head) / L.vec;
#define LAK_SD(VV)                                                                        \
    launch_k(dot_sparse_kernel<T, VV>, L.grid, L.block, 0, s, out, vp, idx, yp, nnz, head,       \
                                                        nchunks, L.inc, counter, partials)
    switch (L.vec) {
    case 1: LAK_SD(1); break;
    case 2: LAK_SD(2); break;
    case 4: LAK_SD(4); break;
    case 8: LAK_SD(8); break;
    default: return fail(LAK_EINVAL, "vec_dot_sparse: unsupported vec %d", L.vec);
    }
#undef LAK_SD
    return check_launch("vec_dot_sparse");
}

template <typename T>
lak_status axpby_t(void *x, double alpha, const void *y, double beta, const void *z, int64_t n,
                   int64_t head, const Launch &L, cudaStream_t s) {
    using A = typename Acc<T>::type;
    T *xp = static_cast<T *>(x);
    const T *yp = static_cast<const T *>(y);
    const T *zp = static_cast<const T *>(z);
    const int64_t nchunks = (n - head) / L.vec;
#define LAK_AB(VV)                                                                        \
    launch_k(axpby_kernel<T, VV>, L.grid, L.block, 0, s, xp, (A)alpha, yp, (A)beta, zp, n, head, \
                                                   nchunks, L.inc)
    switch (L.vec) {
    case 1: LAK_AB(1); break;
    case 2: LAK_AB(2); break;
    case 4: LAK_AB(4); break;
    case 8: LAK_AB(8); break;
    case 16: LAK_AB(16); break;
    default: return fail(LAK_EINVAL, "vec_axpby: unsupported vec %d", L.vec);
    }
#undef LAK_AB
    return check_launch("vec_axpby");
}

template <typename T>
lak_status axpby_strided_t(void *x, int64_t incx, double alpha, const void *y, int64_t incy,
                           double beta, const void *z, int64_t incz, int64_t n, int grid,
                           int block, cudaStream_t s) {
    using A = typename Acc<T>::type;
    launch_k(axpby_strided_kernel<T>, grid, block, 0, s, static_cast<T *>(x), incx, (A)alpha,
                                                   static_cast<const T *>(y), incy, (A)beta,
                                                   static_cast<const T *>(z), incz, n);
    return check_launch("vec_axpby_strided");
}

template <typename T>
lak_status axpy_norm2_t(void *x, const void *y, const void *z, double alpha, void *out, int64_t n,
                        int64_t head, void *ws, const Launch &L, cudaStream_t s) {
    using A = typename Acc<T>::type;
    T *xp = static_cast<T *>(x);
    const T *yp = static_cast<const T *>(y);
    const T *zp = static_cast<const T *>(z);
    unsigned int *counter = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
    const int64_t nchunks = (n - head) / L.vec;
#define LAK_AN(VV)                                                                          \
    launch_k(axpy_norm2_kernel<T, VV>, L.grid, L.block, 0, s, xp, yp, zp, (A)alpha, out, n, head,   \
                                                        nchunks, L.inc, counter, partials)
    switch (L.vec) {
    case 1: LAK_AN(1); break;
    case 2: LAK_AN(2); break;
    case 4: LAK_AN(4); break;
    case 8: LAK_AN(8); break;
    case 16: LAK_AN(16); break;
    default: return fail(LAK_EINVAL, "vec_axpy_norm2: unsupported vec %d", L.vec);
    }
#undef LAK_AN
    return check_launch("vec_axpy_norm2");
}

}  // namespace

lak_status launch_axpby(lak_dtype dt, void *x, double alpha, const void *y, double beta,
                        const void *z, int64_t n, const Launch &L, int64_t head, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return axpby_t<float>(x, alpha, y, beta, z, n, head, L, s);
    case LAK_F64: return axpby_t<double>(x, alpha, y, beta, z, n, head, L, s);
    case LAK_BF16: return axpby_t<__nv_bfloat16>(x, alpha, y, beta, z, n, head, L, s);
    case LAK_F16: return axpby_t<__half>(x, alpha, y, beta, z, n, head, L, s);
    }
    return fail(LAK_EDTYPE, "vec_axpby: unknown dtype %d", (int)dt);
}

lak_status launch_axpby_strided(lak_dtype dt, void *x, int64_t incx, double alpha, const void *y,
                                int64_t incy, double beta, const void *z, int64_t incz, int64_t n,
                                int grid, int block, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return axpby_strided_t<float>(x, incx, alpha, y, incy, beta, z, incz, n, grid, block, s);
    case LAK_F64: return axpby_strided_t<double>(x, incx, alpha, y, incy, beta, z, incz, n, grid, block, s);
    case LAK_BF16: return axpby_strided_t<__nv_bfloat16>(x, incx, alpha, y, incy, beta, z, incz, n, grid, block, s);
    case LAK_F16: return axpby_strided_t<__half>(x, incx, alpha, y, incy, beta, z, incz, n, grid, block, s);
    }
    return fail(LAK_EDTYPE, "vec_axpby_strided: unknown dtype %d", (int)dt);
}

lak_status launch_dot_sparse(lak_dtype dt, void *out, const void *vals, const int32_t *idx,
                             const void *y, int64_t nnz, void *ws, const Launch &L, int64_t head,
                             cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return dot_sparse_t<float>(out, vals, idx, y, nnz, head, ws, L, s);
    case LAK_F64: return dot_sparse_t<double>(out, vals, idx, y, nnz, head, ws, L, s);
    case LAK_BF16: return dot_sparse_t<__nv_bfloat16>(out, vals, idx, y, nnz, head, ws, L, s);
    case LAK_F16: return dot_sparse_t<__half>(out, vals, idx, y, nnz, head, ws, L, s);
    }
    return fail(LAK_EDTYPE, "vec_dot_sparse: unknown dtype %d", (int)dt);
}

lak_status launch_axpy_norm2(lak_dtype dt, void *x, const void *y, const void *z, double alpha,
                             void *out, int64_t n, void *ws, const Launch &L, int64_t head,
                             cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return axpy_norm2_t<float>(x, y, z, alpha, out, n, head, ws, L, s);
    case LAK_F64: return axpy_norm2_t<double>(x, y, z, alpha, out, n, head, ws, L, s);
    case LAK_BF16: return axpy_norm2_t<__nv_bfloat16>(x, y, z, alpha, out, n, head, ws, L, s);
    case LAK_F16: return axpy_norm2_t<__half>(x, y, z, alpha, out, n, head, ws, L, s);
    }
    return fail(LAK_EDTYPE, "vec_axpy_norm2: unknown dtype %d", (int)dt);
}

}  // namespace lak
