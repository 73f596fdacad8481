// Vector kernels: copy x <- y, update x <- y + alpha*z, inner product <x, y>
// (Rupp et al., IWOCL'14, Sec. 2).  All three share the two loop skeletons
// of Sec. 2 -- "global increment" (grid-stride) and "local increment" (each
// block walks its own contiguous range) -- and the vector length of Sec. 2,
// realised as V consecutive elements per thread read with the widest aligned
// loads (up to 256-bit on sm_103a).  A scalar prologue/epilogue covers the
// elements before the first aligned address and after the last full group.
#include "lak_internal.cuh"
#include "vec_loop.cuh"

namespace lak {
namespace {

// ---- copy: a bit copy of elements of 2, 4 or 8 bytes ----------------------

template <typename E, int V>
__global__ void __launch_bounds__(512)
copy_kernel(E *__restrict__ x, const E *__restrict__ y, int64_t n, int64_t head,
            int64_t nchunks, int inc) {
    LAK_PDL_ENTRY();
    const E *yb = y + head;
    E *xb = x + head;
    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        Pack<E, V> p;
        load_pack<E, V, STREAM>(p, yb + c * V);
        store_pack<E, V>(xb + c * V, p);
    }
    const int64_t body_end = head + nchunks * V;
    const int64_t nextra = head + (n - body_end);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nextra) {
        const int64_t i = extra_index(t, head, body_end);
        x[i] = y[i];
    }
}

// ---- axpy: x = y + alpha*z, one fused multiply-add per element -------------

template <typename T, int V>
__global__ void __launch_bounds__(512)
axpy_kernel(T *x, const T *y, const T *z, typename Acc<T>::type alpha, int64_t n, int64_t head,
            int64_t nchunks, int inc) {
    LAK_PDL_ENTRY();
    // x may alias y or z, so the loads take the coherent path
    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        const int64_t o = head + c * V;
        Pack<T, V> py, pz, px;
        load_pack<T, V, COHERENT>(py, y + o);
        load_pack<T, V, COHERENT>(pz, z + o);
#pragma unroll
        for (int v = 0; v < V; ++v)
            px.e[v] = narrow<T>(fma_acc(alpha, widen(pz.e[v]), widen(py.e[v])));
        store_pack<T, V>(x + o, px);
    }
    const int64_t body_end = head + nchunks * V;
    const int64_t nextra = head + (n - body_end);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nextra) {
        const int64_t i = extra_index(t, head, body_end);
        x[i] = narrow<T>(fma_acc(alpha, widen(z[i]), widen(y[i])));
    }
}

// ---- dot: single pass, last-arriving block combines -------------------------
//
// Per thread: V independent accumulators in the arithmetic type (FP32 for
// FP32/BF16/FP16 storage).  Per warp: shuffle tree.  Per block: the warp sums
// are added in FP64 and the block partial is stored in the workspace.  The
// block whose arrival ticket is last adds all partials in FP64 in a fixed
// order (strided per thread, then a shuffle tree), so the result does not
// depend on which block happens to arrive last.  The ticket is an
// acquire-release increment with wrap-around at gridDim.x - 1, so a completed
// call leaves the counter at zero for the next call; a one-block grid writes
// its sum directly.

template <typename T, int V>
__global__ void __launch_bounds__(512)
dot_kernel(void *out, const T *__restrict__ x, const T *__restrict__ y, int64_t n,
           int64_t head, int64_t nchunks, int inc, unsigned int *counter,
           double *partials) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    A acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = A(0);

    const Range r = chunk_range(nchunks, inc);
    for (int64_t c = r.begin; c < r.end; c += r.stride) {
        const int64_t o = head + c * V;
        Pack<T, V> px, py;
        load_pack<T, V, STREAM>(px, x + o);
        load_pack<T, V, STREAM>(py, y + o);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma_acc(widen(px.e[v]), widen(py.e[v]), acc[v]);
    }
    {
        const int64_t body_end = head + nchunks * V;
        const int64_t nextra = head + (n - body_end);
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (t < nextra) {
            const int64_t i = extra_index(t, head, body_end);
            acc[0] = fma_acc(widen(x[i]), widen(y[i]), acc[0]);
        }
    }
    // pairwise combine of the thread's accumulators
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

// ---- compensated dot (FP32 arithmetic on FP32 / BF16 / FP16 storage) --------
//
// Per thread, V running sums carried as (s, c): every product is split exactly
// into p + e with one FMA (TwoProduct) and every addition into s' + f with
// Knuth's TwoSum, the errors e and f collecting in c (Ogita, Rump and Oishi's
// Dot2 in FP32: the sum behaves as if accumulated in twice FP32 precision).
// Each (s, c) pair is then added as an exact double, and the warp, block and
// last-block combines run in FP64 as in dot_kernel.  The result is written as
// a double.

template <typename T, int V>
__global__ void __launch_bounds__(512)
dot_comp_kernel(double *out, const T *__restrict__ x, const T *__restrict__ y, int64_t n,
                int64_t head, int64_t nchunks, int inc, unsigned int *counter,
                double *partials) {
    LAK_PDL_ENTRY();
    float sv[V], cv[V];
#pragma unroll
    for (int v = 0; v < V; ++v) sv[v] = cv[v] = 0.0f;

    // Every operation is an explicitly rounded intrinsic: nvcc contracts a plain
    // `s + a * b` into one FMA under its default --fmad=true, which would make
    // t = fma(a, b, s) and f no longer the exact error of s + p.  The _rn
    // intrinsics are never contracted.
    auto add = [](float &s, float &c, float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);      // a*b = p + e exactly
        const float t = __fadd_rn(s, p);          // TwoSum(s, p) = t + f
        const float bv = __fsub_rn(t, s);
        const float f = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
        s = t;
        c = __fadd_rn(c, __fadd_rn(f, e));
    };

    const Range r = chunk_range(nchunks, inc);
    for (int64_t ch = r.begin; ch < r.end; ch += r.stride) {
        const int64_t o = head + ch * V;
        Pack<T, V> px, py;
        load_pack<T, V, STREAM>(px, x + o);
        load_pack<T, V, STREAM>(py, y + o);
#pragma unroll
        for (int v = 0; v < V; ++v) add(sv[v], cv[v], widen(px.e[v]), widen(py.e[v]));
    }
    {
        const int64_t body_end = head + nchunks * V;
        const int64_t nextra = head + (n - body_end);
        const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (t < nextra) {
            const int64_t i = extra_index(t, head, body_end);
            add(sv[0], cv[0], widen(x[i]), widen(y[i]));
        }
    }
    double d = 0.0;
#pragma unroll
    for (int v = 0; v < V; ++v) d += (double)sv[v] + (double)cv[v];
    grid_sum_last_block(d, out, counter, partials);
}

// ---- dispatch ----------------------------------------------------------------

template <typename E>
lak_status copy_vec(int vec, E *x, const E *y, int64_t n, int64_t head, const Launch &L,
                    cudaStream_t s) {
    const int64_t nchunks = (n - head) / vec;
    switch (vec) {
    case 1: launch_k(copy_kernel<E, 1>, L.grid, L.block, 0, s, x, y, n, head, nchunks, L.inc); break;
    case 2: launch_k(copy_kernel<E, 2>, L.grid, L.block, 0, s, x, y, n, head, nchunks, L.inc); break;
    case 4: launch_k(copy_kernel<E, 4>, L.grid, L.block, 0, s, x, y, n, head, nchunks, L.inc); break;
    case 8: launch_k(copy_kernel<E, 8>, L.grid, L.block, 0, s, x, y, n, head, nchunks, L.inc); break;
    case 16: launch_k(copy_kernel<E, 16>, L.grid, L.block, 0, s, x, y, n, head, nchunks, L.inc); break;
    default: return fail(LAK_EINVAL, "vec_copy: unsupported vec %d", vec);
    }
    return check_launch("vec_copy");
}

template <typename T>
lak_status axpy_t(int vec, void *x, const void *y, const void *z, double alpha, int64_t n,
                  int64_t head, const Launch &L, cudaStream_t s) {
    using A = typename Acc<T>::type;
    T *xp = static_cast<T *>(x);
    const T *yp = static_cast<const T *>(y);
    const T *zp = static_cast<const T *>(z);
    const A a = static_cast<A>(alpha);
    const int64_t nchunks = (n - head) / vec;
    switch (vec) {
    case 1: launch_k(axpy_kernel<T, 1>, L.grid, L.block, 0, s, xp, yp, zp, a, n, head, nchunks, L.inc); break;
    case 2: launch_k(axpy_kernel<T, 2>, L.grid, L.block, 0, s, xp, yp, zp, a, n, head, nchunks, L.inc); break;
    case 4: launch_k(axpy_kernel<T, 4>, L.grid, L.block, 0, s, xp, yp, zp, a, n, head, nchunks, L.inc); break;
    case 8: launch_k(axpy_kernel<T, 8>, L.grid, L.block, 0, s, xp, yp, zp, a, n, head, nchunks, L.inc); break;
    case 16: launch_k(axpy_kernel<T, 16>, L.grid, L.block, 0, s, xp, yp, zp, a, n, head, nchunks, L.inc); break;
    default: return fail(LAK_EINVAL, "vec_axpy: unsupported vec %d", vec);
    }
    return check_launch("vec_axpy");
}

template <typename T>
lak_status dot_t(int vec, void *out, const void *x, const void *y, int64_t n, int64_t head,
                 void *ws, const Launch &L, cudaStream_t s) {
    const T *xp = static_cast<const T *>(x);
    const T *yp = static_cast<const T *>(y);
    unsigned int *counter = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
    const int64_t nchunks = (n - head) / vec;
#define LAK_DOT(VV)                                                                     \
    launch_k(dot_kernel<T, VV>, L.grid, L.block, 0, s, out, xp, yp, n, head, nchunks, L.inc, \
                                                 counter, partials)
    switch (vec) {
    case 1: LAK_DOT(1); break;
    case 2: LAK_DOT(2); break;
    case 4: LAK_DOT(4); break;
    case 8: LAK_DOT(8); break;
    case 16: LAK_DOT(16); break;
    default: return fail(LAK_EINVAL, "vec_dot: unsupported vec %d", vec);
    }
#undef LAK_DOT
    return check_launch("vec_dot");
}

template <typename T>
lak_status dot_comp_t(int vec, void *out, const void *x, const void *y, int64_t n, int64_t head,
                      void *ws, const Launch &L, cudaStream_t s) {
    const T *xp = static_cast<const T *>(x);
    const T *yp = static_cast<const T *>(y);
    double *o = static_cast<double *>(out);
    unsigned int *counter = static_cast<unsigned int *>(ws);
    double *partials = reinterpret_cast<double *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
    const int64_t nchunks = (n - head) / vec;
#define LAK_DOTC(VV)                                                                    \
    launch_k(dot_comp_kernel<T, VV>, L.grid, L.block, 0, s, o, xp, yp, n, head, nchunks, L.inc, \
                                                      counter, partials)
    switch (vec) {
    case 1: LAK_DOTC(1); break;
    case 2: LAK_DOTC(2); break;
    case 4: LAK_DOTC(4); break;
    case 8: LAK_DOTC(8); break;
    case 16: LAK_DOTC(16); break;
    default: return fail(LAK_EINVAL, "vec_dot_compensated: unsupported vec %d", vec);
    }
#undef LAK_DOTC
    return check_launch("vec_dot_compensated");
}

}  // namespace

lak_status launch_copy(void *x, const void *y, int64_t n, int es, const Launch &L, int64_t head,
                       cudaStream_t s) {
    switch (es) {
    case 2: return copy_vec<uint16_t>(L.vec, (uint16_t *)x, (const uint16_t *)y, n, head, L, s);
    case 4: return copy_vec<uint32_t>(L.vec, (uint32_t *)x, (const uint32_t *)y, n, head, L, s);
    case 8: return copy_vec<uint64_t>(L.vec, (uint64_t *)x, (const uint64_t *)y, n, head, L, s);
    }
    return fail(LAK_EDTYPE, "vec_copy: element size %d", es);
}

lak_status launch_axpy(lak_dtype dt, void *x, const void *y, const void *z, double alpha,
                       int64_t n, const Launch &L, int64_t head, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return axpy_t<float>(L.vec, x, y, z, alpha, n, head, L, s);
    case LAK_F64: return axpy_t<double>(L.vec, x, y, z, alpha, n, head, L, s);
    case LAK_BF16: return axpy_t<__nv_bfloat16>(L.vec, x, y, z, alpha, n, head, L, s);
    case LAK_F16: return axpy_t<__half>(L.vec, x, y, z, alpha, n, head, L, s);
    }
    return fail(LAK_EDTYPE, "vec_axpy: unknown dtype %d", (int)dt);
}

lak_status launch_dot(lak_dtype dt, void *out, const void *x, const void *y, int64_t n, void *ws,
                      const Launch &L, int64_t head, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return dot_t<float>(L.vec, out, x, y, n, head, ws, L, s);
    case LAK_F64: return dot_t<double>(L.vec, out, x, y, n, head, ws, L, s);
    case LAK_BF16: return dot_t<__nv_bfloat16>(L.vec, out, x, y, n, head, ws, L, s);
    case LAK_F16: return dot_t<__half>(L.vec, out, x, y, n, head, ws, L, s);
    }
    return fail(LAK_EDTYPE, "vec_dot: unknown dtype %d", (int)dt);
}

}  // namespace lak

namespace lak {

lak_status launch_dot_comp(lak_dtype dt, void *out, const void *x, const void *y, int64_t n,
                           void *ws, const Launch &L, int64_t head, cudaStream_t s) {
    switch (dt) {
    case LAK_F32: return dot_comp_t<float>(L.vec, out, x, y, n, head, ws, L, s);
    case LAK_BF16: return dot_comp_t<__nv_bfloat16>(L.vec, out, x, y, n, head, ws, L, s);
    case LAK_F16: return dot_comp_t<__half>(L.vec, out, x, y, n, head, ws, L, s);
    default: break;
    }
    return fail(LAK_EDTYPE, "vec_dot_compensated: FP32, BF16 or FP16 storage only (dtype %d)",
                (int)dt);
}

}  // namespace lak
