// Dot product of one matrix row with x by a group of G lanes, shared by the
// row-major GEMV kernel (k_gemv.cu) and the batched GEMV kernel (k_batch.cu).
//
// The row's first elements up to the next boundary of the access width W are
// taken one per lane (a "head" of fewer than V elements), so the rest of the
// row is read with aligned wide streamed loads whatever the leading dimension.
// x is read with wide cached loads when its matching offset is aligned too,
// else element by element through L1 (it is re-read by every row).
//
// FP32 keeps V partial sums (independent FMA chains); FP64 keeps one chain in
// acc[0]: on GB300 the FP64 pipe, not the FMA latency, bounds the FP64
// product, and V partial sums would cost V - 1 extra FP64 adds per lane and
// row (callers skip the combine when gemv_one_chain<T> holds).
#pragma once

#include "lak_internal.cuh"

namespace lak {

template <typename T>
constexpr bool gemv_one_chain = sizeof(typename Acc<T>::type) == 8;

template <typename T, int V>
__device__ __forceinline__ void row_group_dot(typename Acc<T>::type (&acc)[V],
                                              const T *__restrict__ Ar, const T *__restrict__ x,
                                              int64_t n, int lg, int G) {
    using Ac = typename Acc<T>::type;
    constexpr int ES = (int)sizeof(T);
    constexpr int W = V * ES > 32 ? 32 : V * ES;
    const int64_t mis = (int64_t)(((uintptr_t)Ar % W) / ES);
    int64_t head = mis ? (int64_t)(W / ES) - mis : 0;
    if (head > n) head = n;
    for (int64_t j = lg; j < head; j += G)
        acc[0] = fma_wide(Ar[j], ld_cached(x + j), acc[0]);
    const T *Ab = Ar + head;
    const T *xb = x + head;
    const int64_t nb = n - head;
    const int64_t nch = nb / V;
    if (((uintptr_t)xb % W) == 0) {
#pragma unroll 4
        for (int64_t c = lg; c < nch; c += G) {
            Pack<T, V> pa, px;
            load_pack<T, V, STREAM>(pa, Ab + c * V);
            load_pack<T, V, CACHED>(px, xb + c * V);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                Ac &a = gemv_one_chain<T> ? acc[0] : acc[v];
                a = fma_wide(pa.e[v], px.e[v], a);
            }
        }
    } else {
#pragma unroll 4
        for (int64_t c = lg; c < nch; c += G) {
            Pack<T, V> pa;
            load_pack<T, V, STREAM>(pa, Ab + c * V);
#pragma unroll
            for (int v = 0; v < V; ++v) {
                Ac &a = gemv_one_chain<T> ? acc[0] : acc[v];
                a = fma_wide(pa.e[v], ld_cached(xb + c * V + v), a);
            }
        }
    }
    for (int64_t j = nch * V + lg; j < nb; j += G)
        acc[0] = fma_wide(Ab[j], ld_cached(xb + j), acc[0]);
}

}  // namespace lak
