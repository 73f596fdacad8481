// Body of the warp-segmented CSR product for one block of 32 consecutive rows,
// shared by the single-matrix kernel (k_spmv.cu) and the batched kernel
// (k_batch.cu).
//
// Lane l owns the U consecutive entries [c0 + l*U, c0 + (l+1)*U) of the warp's
// current chunk, reads them with 16-byte vector loads when the arrays allow it,
// and accumulates with one FMA per entry, closing a partial sum whenever it
// crosses a row boundary.  A row that continues across lanes is joined by a
// segmented inclusive scan over the lanes, with only as many shuffle steps as
// the chunk's longest run of lanes needs (at most 5); a row that continues
// across chunks leaves its running sum in the warp's shared-memory slot, and
// lane 0 of the next chunk starts its FMA chain from it.  Every slot is only
// ever stored (a row's running total, by the one lane that holds its last entry
// in the chunk), so the result is deterministic and needs no atomics.
//
// Floating-point instructions per chunk: U FMAs per lane, one add per scan step
// and one add to join the carried-in sum; a row that begins and ends inside a
// lane costs no add at all.  This matters for FP64 on GB300, where the FP64
// pipe, not memory, bounds the kernel.  All 32 lanes of the warp must call it.
#pragma once

#include "lak_internal.cuh"

namespace lak {

template <typename T, int U, bool VLOAD>
__device__ __forceinline__ void seg_rows32(T *__restrict__ y, const int32_t *__restrict__ rp,
                                           const int32_t *__restrict__ ci,
                                           const T *__restrict__ vals, const T *__restrict__ x,
                                           int64_t m, int64_t nnz64, int64_t b, uint32_t *rs,
                                           typename Acc<T>::type *racc) {
    using Ac = typename Acc<T>::type;
    constexpr uint32_t CH = 32 * U;
    // Entry positions fit in 32 bits: row_ptr is int32, so nnz < 2^31, and a
    // position never exceeds nnz + CH < 2^32.
    const uint32_t nnz = (uint32_t)nnz64;
    const int lane = threadIdx.x & 31;
    const int64_t row = b * 32 + lane;
    rs[lane] = row < m ? (uint32_t)__ldg(rp + row) : nnz;
    if (lane == 31) rs[32] = (b * 32 + 32 < m) ? (uint32_t)__ldg(rp + b * 32 + 32) : nnz;
    racc[lane] = Ac(0);
    __syncwarp();
    const uint32_t S = rs[0];
    const uint32_t E = rs[32];
    const uint32_t cbeg = VLOAD ? (S & ~3u) : S;
    for (uint32_t c0 = cbeg; c0 < E; c0 += CH) {  // warp-uniform trip count
        const uint32_t k0 = c0 + (uint32_t)lane * U;
        int32_t col[U];
        T val[U];
        if constexpr (VLOAD) {
#pragma unroll
            for (int q = 0; q < U; q += 4) {
                const uint32_t kq = k0 + q;
                if (kq + 4 <= nnz) {
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
                        const uint32_t k = kq + t;
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
                const uint32_t k = k0 + j;
                if (k >= S && k < E) {
                    col[j] = __ldg(ci + k);
                    val[j] = vals[k];
                }
            }
        }
        // first valid entry of this lane and the row that holds it
        const uint32_t kf = k0 > S ? k0 : S;
        const bool any = kf < E && kf < k0 + U;
        int r = 0;
        if (any) {
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (r + step <= 31 && rs[r + step] <= kf) r += step;
        }
        // walk the lane's entries, one FMA each, splitting at row ends; lane 0
        // continues the running sum of a row begun in an earlier chunk
        const bool head_from_left = any && kf > rs[r];
        Ac part = (lane == 0 && head_from_left) ? racc[r] : Ac(0);
        int nseg = 0;                  // segments closed so far in this lane
        Ac head = Ac(0);
        int head_row = r;
        int cur = r;
#pragma unroll
        for (int j = 0; j < U; ++j) {
            const uint32_t k = k0 + j;
            if (k < kf || k >= E) continue;
            if (k >= rs[cur + 1]) {    // the current row ended before k
                if (nseg == 0) {
                    head = part;
                    head_row = cur;
                } else {
                    racc[cur] = part;  // a row that began and ended in this lane
                }
                ++nseg;
                part = Ac(0);
                do { ++cur; } while (k >= rs[cur + 1]);
            }
            part = fma_acc(widen(val[j]), widen(ld_cached(x + col[j])), part);
        }
        // segmented scan of the open tails across lanes; lanes without entries
        // end any carry, so they count as segment heads, and so does lane 0.
        // Each lane knows its distance to its segment's head from one ballot, so
        // at step d it adds the value d lanes up only while d <= that distance
        // (no head flag travels with the values: one shuffle per step)
        const bool starts_here = any && (nseg > 0 || !head_from_left);
        Ac incl = part;
        const bool flag = starts_here || !any;
        const unsigned heads = __ballot_sync(0xffffffffu, flag) | 1u;
        const unsigned at_or_below = heads & (0xffffffffu >> (31 - lane));
        const int dist = lane - (31 - __clz((int)at_or_below));   // lanes back to the head
        const int span = __reduce_max_sync(0xffffffffu, dist);   // warp-uniform
        for (int d = 1; d <= span; d <<= 1) {
            const Ac v_up = __shfl_up_sync(0xffffffffu, incl, d);
            if (d <= dist) incl += v_up;
        }
        Ac carry = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0 || !head_from_left) carry = Ac(0);
        if (any) {
            const uint32_t kend = k0 + U < E ? k0 + U : E;   // one past the lane's last entry
            const bool tail_open = kend < rs[cur + 1];          // the row goes on
            // the lane's first segment, joined to what the lanes before it hold
            const Ac first = carry + (nseg > 0 ? head : part);
            if (nseg > 0) {
                racc[head_row] = first;                        // that row ends here
                if (!tail_open || lane == 31) racc[cur] = part;
            } else if (!tail_open || lane == 31) {
                racc[cur] = first;
            }
        }
        __syncwarp();
    }
    __syncwarp();
    if (row < m) y[row] = narrow<T>(racc[lane]);
    __syncwarp();
}

}  // namespace lak
