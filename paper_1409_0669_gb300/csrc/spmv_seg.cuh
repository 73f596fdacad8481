// Body of the warp-segmented CSR product for one block of 32 consecutive rows,
// shared by the single-matrix kernel (k_spmv.cu) and the batched kernel
// (k_batch.cu).
//
// Lane l owns the U consecutive entries [c0 + l*U, c0 + (l+1)*U) of the warp's
// current chunk, reads them with 16-byte vector loads when the arrays allow it,
// and accumulates with one FMA per entry, closing a partial sum whenever it
// crosses a row boundary.  A row that continues across lanes is joined by a
// segmented inclusive scan over the lanes (5 shuffle steps); a row that
// continues across chunks is joined in the warp's shared-memory accumulator.
// Every (row, chunk) partial has exactly one writer, so the result is
// deterministic and needs no atomics.  All 32 lanes of the warp must call it.
#pragma once

#include "lak_internal.cuh"

namespace lak {

template <typename T, int U, bool VLOAD>
__device__ __forceinline__ void seg_rows32(T *__restrict__ y, const int32_t *__restrict__ rp,
                                           const int32_t *__restrict__ ci,
                                           const T *__restrict__ vals, const T *__restrict__ x,
                                           int64_t m, int64_t nnz, int64_t b, int64_t *rs,
                                           typename Acc<T>::type *racc) {
    using Ac = typename Acc<T>::type;
    constexpr int CH = 32 * U;
    const int lane = threadIdx.x & 31;
    const int64_t row = b * 32 + lane;
    const int64_t s_l = row < m ? (int64_t)__ldg(rp + row) : nnz;
    rs[lane] = s_l;
    if (lane == 31) rs[32] = (b * 32 + 32 < m) ? (int64_t)__ldg(rp + b * 32 + 32) : nnz;
    racc[lane] = Ac(0);
    __syncwarp();
    const int64_t S = rs[0];
    const int64_t E = rs[32];
    const int64_t cbeg = VLOAD ? (S & ~(int64_t)3) : S;
    for (int64_t c0 = cbeg; c0 < E; c0 += CH) {  // warp-uniform trip count
        const int64_t k0 = c0 + (int64_t)lane * U;
        int32_t col[U];
        T val[U];
        if constexpr (VLOAD) {
#pragma unroll
            for (int q = 0; q < U; q += 4) {
                const int64_t kq = k0 + q;
                if (kq >= 0 && kq + 4 <= nnz) {
                    ld_raw<16, CACHED>(&col[q], ci + kq);
                    if constexpr (sizeof(T) == 8) {
                        ld_raw<16, CACHED>(&val[q], vals + kq);
                        ld_raw<16, CACHED>(&val[q + 2], vals + kq + 2);
                    } else if constexpr (sizeof(T) == 4) {
                        ld_raw<16, CACHED>(&val[q], vals + kq);
                    } else {
                        ld_raw<8, CACHED>(&val[q], vals + kq);
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int64_t k = kq + t;
                        if (k >= S && k < E) {
                            col[q + t] = __ldg(ci + k);
                            val[q + t] = vals[k];
                        }
                    }
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int64_t k = k0 + j;
                if (k >= S && k < E) {
                    col[j] = __ldg(ci + k);
                    val[j] = vals[k];
                }
            }
        }
        // first valid entry of this lane and the row that holds it
        const int64_t kf = k0 > S ? k0 : S;
        const bool any = kf < E && kf < k0 + U;
        int r = 0;
        if (any) {
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (r + step <= 31 && rs[r + step] <= kf) r += step;
        }
        // walk the lane's entries, one FMA each, splitting at row ends
        Ac part = Ac(0);
        int nseg = 0;                  // segments closed so far in this lane
        Ac head = Ac(0);
        int head_row = r;
        bool head_from_left = any && kf > rs[r];
        int cur = r;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const int64_t k = k0 + j;
            if (k < kf || k >= E) continue;
            if (k >= rs[cur + 1]) {    // the current row ended before k
                if (nseg == 0) {
                    head = part;
                    head_row = cur;
                } else {
                    racc[cur] += part; // a row that started and ended in this lane
                }
                ++nseg;
                part = Ac(0);
                do { ++cur; } while (k >= rs[cur + 1]);
            }
            part = fma_acc(widen(val[j]), widen(ld_cached(x + col[j])), part);
        }
        // segmented scan of the open tails across lanes
        const bool starts_here = any && (nseg > 0 || !head_from_left);
        Ac incl = part;
        bool flag = starts_here || !any;
        // lanes without entries end any carry: treat them as segment heads
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const Ac v_up = __shfl_up_sync(0xffffffffu, incl, d);
            const bool f_up = __shfl_up_sync(0xffffffffu, (int)flag, d) != 0;
            if (lane >= d) {
                if (!flag) incl += v_up;
                flag = flag || f_up;
            }
        }
        Ac carry = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) carry = Ac(0);
        if (any) {
            const int64_t klast = (k0 + U < E ? k0 + U : E) - 1;
            const bool tail_open = klast + 1 < rs[cur + 1];   // the row goes on
            if (nseg > 0) {
                // the first segment ended inside this lane
                racc[head_row] += (head_from_left ? carry : Ac(0)) + head;
                if (!tail_open || lane == 31) racc[cur] += part;
            } else {
                // one segment only: row `cur`
                const Ac total = (head_from_left ? carry : Ac(0)) + part;
                if (!tail_open || lane == 31) racc[cur] += total;
            }
        }
        __syncwarp();
    }
    __syncwarp();
    if (row < m) y[row] = narrow<T>(racc[lane]);
    __syncwarp();
}

}  // namespace lak
