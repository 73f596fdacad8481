// Batched operations: many independent instances of uneven sizes in one
// persistent launch.
//
// lak_batch_plan (host, no CUDA call) splits every instance into work units --
// `unit_elems` elements of a vector or a run of rows of a dense matrix with
// about as many entries (about 256 KB of one operand), or one block's rows of a
// CSR matrix -- and writes a table: a header, the exclusive prefix of units per
// instance, and per-instance items (the caller's descriptor plus the launch
// details the plan chose).  lak_batch_run launches one persistent grid over
// all units; a block maps its unit to an instance with a binary search over
// the prefix (a few L1-resident loads) and runs the inner loops of the
// single-instance kernels, except for dense rows: a lane group per row sized
// from the row length takes four rows at a time, and at 16-byte accesses the
// rows reach the lanes through a shared-memory ring of asynchronous copies
// (gemv_group_rows); CSR rows take the warp-segmented body.  Batched dot
// products finish per instance with the last-arriving-unit combine (an arrival
// counter per instance in the workspace counter area), in unit order, so
// results are deterministic.
#include <cstddef>

#include "gemv_row.cuh"
#include "lak_internal.cuh"
#include "spmv_seg.cuh"

namespace lak {
namespace {

struct BatchHead {
    int64_t count;
    int64_t total_units;
    int64_t unit_elems;
    int32_t op;
    int32_t dtype;
    int32_t vec;
    int32_t block;
    int32_t inc;
    int32_t pad;
};

struct AxpyItem {
    lak_axpy_desc d;
    int64_t units;
    int32_t vec_ok;
    int32_t pad;
};
struct DotItem {
    lak_dot_desc d;
    int64_t units;
    int32_t vec_ok;
    int32_t pad;
};
struct GemvItem {
    lak_gemv_desc d;
    int64_t rows_per_unit;
    int32_t vec_ok;
    int32_t group;           // lanes per row (power of two <= 32)
    int32_t period;          // groups of 4+ lanes: rows r and r + period share their alignment
    int32_t pad;
};

// Rows of lane groups of 4+ lanes are taken R at a time by one group: rows
// r, r + P, ..., r + (R-1) P, which share their alignment to the access width,
// so one x pack serves R rows and one reduction closes R sums.  Such groups
// only occur with packs of at most 32 bytes, for which R = 4.
__host__ __device__ constexpr int gemv_rows_per_group(int access_bytes) {
    return access_bytes <= 32 ? 4 : 2;
}
struct CsrItem {
    lak_csr_desc d;
    int64_t rows_per_unit;   // a multiple of the block's rows (32 per warp)
    int32_t vec_ok;
    int32_t pad;
};

constexpr size_t kHeadBytes = 64;
static_assert(sizeof(BatchHead) <= kHeadBytes, "batch header");

size_t offsets_bytes(int64_t count) { return (size_t)(count + 1) * 8; }
size_t items_offset(int64_t count) { return (kHeadBytes + offsets_bytes(count) + 15) / 16 * 16; }

size_t item_size(lak_op op) {
    switch (op) {
    case LAK_OP_AXPY: return sizeof(AxpyItem);
    case LAK_OP_DOT: return sizeof(DotItem);
    case LAK_OP_GEMV_ROW: return sizeof(GemvItem);
    case LAK_OP_SPMV: return sizeof(CsrItem);
    default: return 0;
    }
}

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

bool aligned_to(const void *p, int w) { return (uintptr_t)p % (uintptr_t)w == 0; }

// ---- device helpers ----------------------------------------------------------

// largest i in [0, count) with offs[i] <= u (skips instances without units)
__device__ __forceinline__ int64_t find_instance(const int64_t *offs, int64_t count, int64_t u) {
    int64_t lo = 0, hi = count - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(offs + mid) <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The order in which a block takes units of the vector and GEMV batches follows
// the configuration's increment type (Sec. 2): global = grid-stride (the blocks
// resident on one SM take consecutive units, usually of one instance, and share
// its re-read operands in L1); local = each block walks one contiguous range of
// units.  The CSR batch takes its units dynamically (spmv_batch_kernel).
struct UnitRange {
    int64_t begin, end, step;
};
__device__ __forceinline__ UnitRange unit_range(int64_t total, int inc) {
    if (inc == LAK_INC_GLOBAL) return {(int64_t)blockIdx.x, total, (int64_t)gridDim.x};
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t b = (int64_t)blockIdx.x * per;
    return {b, b + per < total ? b + per : total, 1};
}

template <typename T, int V>
__global__ void __launch_bounds__(512)
axpy_batch_kernel(const BatchHead *__restrict__ head, const int64_t *__restrict__ offs,
                  const AxpyItem *__restrict__ items) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    const int64_t count = head->count, total = head->total_units, ue = head->unit_elems;
    const UnitRange ur = unit_range(total, head->inc);
    for (int64_t u = ur.begin; u < ur.end; u += ur.step) {
        const int64_t i = find_instance(offs, count, u);
        const AxpyItem it = items[i];
        T *x = static_cast<T *>(it.d.x);
        const T *y = static_cast<const T *>(it.d.y);
        const T *z = static_cast<const T *>(it.d.z);
        const A alpha = static_cast<A>(it.d.alpha);
        const int64_t b = (u - __ldg(offs + i)) * ue;
        const int64_t e = b + ue < it.d.n ? b + ue : it.d.n;
        int64_t k = b;
        if (it.vec_ok) {
            const int64_t nfull = (e - b) / V;
            for (int64_t c = threadIdx.x; c < nfull; c += blockDim.x) {
                const int64_t o = b + c * V;
                Pack<T, V> py, pz, px;
                load_pack<T, V, COHERENT>(py, y + o);
                load_pack<T, V, COHERENT>(pz, z + o);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    px.e[v] = narrow<T>(fma_acc(alpha, widen(pz.e[v]), widen(py.e[v])));
                store_pack<T, V>(x + o, px);
            }
            k = b + nfull * V;
        }
        for (int64_t j = k + threadIdx.x; j < e; j += blockDim.x)
            x[j] = narrow<T>(fma_acc(alpha, widen(z[j]), widen(y[j])));
    }
}

template <typename T, int V>
__global__ void __launch_bounds__(512)
dot_batch_kernel(const BatchHead *__restrict__ head, const int64_t *__restrict__ offs,
                 const DotItem *__restrict__ items, unsigned int *tickets, double *partials) {
    LAK_PDL_ENTRY();
    using A = typename Acc<T>::type;
    __shared__ double wsum[32];
    const int64_t count = head->count, total = head->total_units, ue = head->unit_elems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const UnitRange ur = unit_range(total, head->inc);
    for (int64_t u = ur.begin; u < ur.end; u += ur.step) {
        const int64_t i = find_instance(offs, count, u);
        const DotItem it = items[i];
        const T *x = static_cast<const T *>(it.d.x);
        const T *y = static_cast<const T *>(it.d.y);
        const int64_t u0 = __ldg(offs + i);
        const int64_t b = (u - u0) * ue;
        const int64_t e = b + ue < it.d.n ? b + ue : it.d.n;
        A acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = A(0);
        int64_t k = b;
        if (it.vec_ok) {
            const int64_t nfull = (e - b) / V;
            for (int64_t c = threadIdx.x; c < nfull; c += blockDim.x) {
                const int64_t o = b + c * V;
                Pack<T, V> px, py;
                load_pack<T, V, STREAM>(px, x + o);
                load_pack<T, V, STREAM>(py, y + o);
#pragma unroll
                for (int v = 0; v < V; ++v)
                    acc[v] = fma_acc(widen(px.e[v]), widen(py.e[v]), acc[v]);
            }
            k = b + nfull * V;
        }
        for (int64_t j = k + threadIdx.x; j < e; j += blockDim.x)
            acc[0] = fma_acc(widen(x[j]), widen(y[j]), acc[0]);
#pragma unroll
        for (int w = 1; w < V; w <<= 1) {
#pragma unroll
            for (int v = 0; v + w < V; v += 2 * w) acc[v] += acc[v + w];
        }
        const A s = group_sum(acc[0], 32);
        if (lane == 0) wsum[warp] = (double)s;
        __syncthreads();
        if (warp == 0) {
            double bsum = lane < nwarps ? wsum[lane] : 0.0;
            bsum = group_sum(bsum, 32);
            if (lane == 0) {
                partials[u] = bsum;
                __threadfence();
                const unsigned int last = (unsigned int)(it.units - 1);
                if (atomicInc(tickets + i, last) == last) {
                    __threadfence();
                    double f = 0.0;                       // unit order: deterministic
                    for (int64_t q = 0; q < it.units; ++q) f += __ldcg(partials + u0 + q);
                    if constexpr (sizeof(A) == 8)
                        *static_cast<double *>(it.d.out) = f;
                    else
                        *static_cast<float *>(it.d.out) = __double2float_rn(f);
                }
            }
        }
        __syncthreads();                                  // wsum is reused
    }
}

// At most 128 threads per block and 64 registers per thread: eight blocks per
// SM.  The batched GEMV is latency-bound, not arithmetic-bound: twice the
// resident blocks keep twice the loads in flight, which pays for the few values
// the cap spills to L1.
//
// Rows of a lane group of 4 or more lanes (every row when a lane reads at most
// 32 bytes per access, as a group reads at least 128 bytes of a row per step)
// are taken R at a time per group (gemv_group_rows): one x
// pack serves R rows, each lane keeps R loads of A in flight per x load, and one
// reduction (halving exchanges, log2(G) + 1 shuffles for R = 4) closes R
// sums instead of R separate ones.  The R rows are r, r + P, ..., r + (R-1) P,
// with P the smallest row stride for which the rows start at the same offset
// modulo the access width (P = 1 when lda * element size is a multiple of it),
// so all R rows share one scalar head and one aligned body.  Measured on the
// 4096-instance FP32 mix: 2.47 ms (6.05 TB/s) against 3.62 ms for one row per
// lane group; FP64 7.8 against 9.0 ms, BF16 2.34 against 2.98 ms.  At 32-byte
// packs the body is not unrolled: four rows already keep four 32-byte loads in
// flight per lane, and a second copy of them does not fit the 64 registers
// (FP64 7.13 ms against 7.40 for the same four rows unrolled twice and 7.53 for
// two rows unrolled twice; BF16 1.81 against 1.92 and 2.12 ms).  16-byte packs
// keep the unrolled body (FP32 2.40 against 3.93 ms).

// Sum of R per-lane values over each aligned group of G lanes (G a power of two,
// 4..32) by halving exchanges: afterwards lane lg of a group holds the total of
// value lg / (G / R), the same in each of its G / R consecutive lanes.
template <typename A, int R>
__device__ __forceinline__ A group_sum_rows(const A (&v)[R], int lg, int G) {
    const int h1 = G >> 1;
    const bool hi = lg & h1;
    if constexpr (R == 4) {
        const int h2 = G >> 2;
        const A r0 = __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[2], h1);
        const A r1 = __shfl_xor_sync(0xffffffffu, hi ? v[1] : v[3], h1);
        const A k0 = (hi ? v[2] : v[0]) + r0;      // rows 0/2
        const A k1 = (hi ? v[3] : v[1]) + r1;      // rows 1/3
        const bool h8 = lg & h2;
        A k = (h8 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, h2);
        for (int o = h2 >> 1; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        return k;                                  // row (hi ? 2 : 0) + (h8 ? 1 : 0)
    } else {
        A k = (hi ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, hi ? v[0] : v[1], h1);
        for (int o = h1 >> 1; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        return k;                                  // row (hi ? 1 : 0)
    }
}

// Asynchronous 16-byte copies from global to shared memory (bypassing L1), and
// the per-thread group bookkeeping that orders them: a thread waits only for its
// own copies, so no barrier is involved.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows of A at 16-byte accesses reach the lanes through a two-stage ring in
// shared memory filled by asynchronous copies (per warp: stages x R rows x 32
// lanes x 16 bytes = 4 KB), so the loads a lane keeps in flight no longer cost
// registers.  Measured on the 4096-instance mixes: BF16 at 8 elements per access
// 2.49 -> 1.33 ms (5.6 TB/s, against 1.69 ms for the best register-staged shape,
// 16 elements per access), FP16 the same; FP32 and FP64 unchanged (2.40 / 7.12 ms
// at their best shapes).  Three stages: BF16 1.38 ms, four: 2.0 ms (the ring
// takes the L1 capacity that serves x).  At 32-byte accesses the ring measured
// slower (FP64 7.12 -> 7.51 ms), so those keep the register path.
constexpr int kGemvRingStages = 2;
constexpr int kGemvRingBytes = 16;

inline size_t gemv_ring_smem(int block, int vec, int es) {
    return vec * es == kGemvRingBytes
               ? (size_t)(block / 32) * kGemvRingStages * gemv_rows_per_group(kGemvRingBytes) * 32 *
                     kGemvRingBytes
               : 0;
}

template <typename T, int V>
__device__ __forceinline__ void gemv_group_rows(const GemvItem &it, int64_t r0, int64_t r1,
                                               int lane, int warp, int nwarps) {
    using Ac = typename Acc<T>::type;
    constexpr int ES = (int)sizeof(T);
    constexpr int W = V * ES > 32 ? 32 : V * ES;
    constexpr int R = gemv_rows_per_group(W);
    const T *Am = static_cast<const T *>(it.d.A);
    const T *x = static_cast<const T *>(it.d.x);
    T *y = static_cast<T *>(it.d.y);
    const int64_t n = it.d.n, lda = it.d.lda;
    const int G = it.group;                       // lanes per row group: 4 .. 32
    const int ng = 32 / G;                        // row groups per warp
    const int lg = lane % G, gi = lane / G;
    const int P = it.period;
    const int64_t span = (int64_t)R * P;
    const int64_t ngroups = (r1 - r0 + span - 1) / span * P;
    for (int64_t gb = (int64_t)warp * ng; gb < ngroups; gb += (int64_t)nwarps * ng) {  // warp-uniform
        const int64_t g = gb + gi;
        const int64_t row0 = r0 + (g / P) * span + (g % P);
        const T *a[R];
        bool ok[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            ok[j] = g < ngroups && row0 + (int64_t)j * P < r1;
            a[j] = Am + (ok[j] ? row0 + (int64_t)j * P : r0) * lda;
        }
        const int64_t mis = (int64_t)(((uintptr_t)a[0] % W) / ES);
        int64_t h = mis ? (int64_t)(W / ES) - mis : 0;
        if (h > n) h = n;
        Ac acc[R];
#pragma unroll
        for (int j = 0; j < R; ++j) acc[j] = Ac(0);
        for (int64_t k = lg; k < h; k += G) {
            const T xv = ld_cached(x + k);
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (ok[j]) acc[j] = fma_wide(a[j][k], xv, acc[j]);
        }
        const int64_t nb = n - h;
        const int64_t nch = nb / V;
        const T *xb = x + h;
        const bool xal = ((uintptr_t)xb % W) == 0;
        constexpr bool kRing = V * ES == kGemvRingBytes;
        if constexpr (kRing) {
            // the lane's steps t = 0, 1, ... (packs c = lg + t G) through its
            // ring slots: step t + NS - 1 is issued before step t is waited for;
            // a lane reads back only the slots it filled itself
            constexpr int NS = kGemvRingStages;
            extern __shared__ __align__(16) unsigned char gemv_ring[];
            unsigned char *ring = gemv_ring + (size_t)warp * NS * R * 32 * W;
            const int64_t steps = lg < nch ? (nch - lg + G - 1) / G : 0;
            auto issue = [&](int64_t t) {
                if (t < steps) {
                    const int64_t c = lg + t * G;
                    unsigned char *slot = ring + (size_t)(t % NS) * R * 32 * W;
#pragma unroll
                    for (int j = 0; j < R; ++j)
                        if (ok[j]) cp_async16(slot + ((size_t)j * 32 + lane) * W, a[j] + h + c * V);
                }
                cp_async_commit();                    // an empty group past the last step
            };
#pragma unroll
            for (int t = 0; t < NS - 1; ++t) issue(t);
            for (int64_t t = 0; t < steps; ++t) {
                issue(t + NS - 1);
                cp_async_wait<NS - 1>();              // step t has landed
                const int64_t c = lg + t * G;
                Pack<T, V> px;
                if (xal) {
                    load_pack<T, V, CACHED>(px, xb + c * V);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) px.e[v] = ld_cached(xb + c * V + v);
                }
                const unsigned char *slot = ring + (size_t)(t % NS) * R * 32 * W;
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    if (!ok[j]) continue;
                    Pack<T, V> pa;
                    memcpy(&pa, slot + ((size_t)j * 32 + lane) * W, W);
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[j] = fma_wide(pa.e[v], px.e[v], acc[j]);
                }
            }
            cp_async_wait<0>();
        }
        constexpr int kUnroll = W <= 16 ? 2 : 1;
#pragma unroll kUnroll
        for (int64_t c = lg; c < (kRing ? 0 : nch); c += G) {
            Pack<T, V> px;
            if (xal) {
                load_pack<T, V, CACHED>(px, xb + c * V);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) px.e[v] = ld_cached(xb + c * V + v);
            }
#pragma unroll
            for (int j = 0; j < R; ++j) {
                if (!ok[j]) continue;
                Pack<T, V> pa;
                load_pack<T, V, STREAM>(pa, a[j] + h + c * V);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[j] = fma_wide(pa.e[v], px.e[v], acc[j]);
            }
        }
        for (int64_t k = h + nch * V + lg; k < n; k += G) {
            const T xv = ld_cached(x + k);
#pragma unroll
            for (int j = 0; j < R; ++j)
                if (ok[j]) acc[j] = fma_wide(a[j][k], xv, acc[j]);
        }
        const Ac s = group_sum_rows<Ac, R>(acc, lg, G);
        const int per = G / R;                                  // lanes holding one row's sum
        if (lg % per == 0) {
            const int j = lg / per;
            const int64_t row = row0 + (int64_t)j * P;
            if (g < ngroups && row < r1) y[row] = narrow<T>(s);
        }
    }
}

// The batched GEMV waits for the kernel before it like every kernel, but lets
// the next one launch only when it has finished (no early
// griddepcontrol.launch_dependents): blocks of a dependent grid started early
// would land on SMs configured for this kernel's shared-memory ring, with less
// L1, and a persistent dependent keeps that configuration to its end -- the
// batched CSR product right after it in one graph ran 1.4 ms (7 %) slower.
template <typename T, int V>
__global__ void __launch_bounds__(kGemvBatchMaxBlock, 8)
gemv_batch_kernel(const BatchHead *__restrict__ head, const int64_t *__restrict__ offs,
                  const GemvItem *__restrict__ items) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    using A = typename Acc<T>::type;
    const int64_t count = head->count, total = head->total_units;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const UnitRange ur = unit_range(total, head->inc);
    for (int64_t u = ur.begin; u < ur.end; u += ur.step) {
        const int64_t i = find_instance(offs, count, u);
        const GemvItem it = items[i];
        const T *Am = static_cast<const T *>(it.d.A);
        const T *x = static_cast<const T *>(it.d.x);
        T *y = static_cast<T *>(it.d.y);
        const int64_t n = it.d.n, lda = it.d.lda;
        const int G = it.group;                     // lanes per row
        const int rpw = 32 / G;                     // rows per warp at a time
        const int lg = lane % G;
        const int64_t r0 = (u - __ldg(offs + i)) * it.rows_per_unit;
        const int64_t r1 = r0 + it.rows_per_unit < it.d.m ? r0 + it.rows_per_unit : it.d.m;
        if (G >= 4) {
            gemv_group_rows<T, V>(it, r0, r1, lane, warp, nwarps);
            continue;
        }
        for (int64_t rb = r0 + (int64_t)warp * rpw; rb < r1; rb += (int64_t)nwarps * rpw) {
            const int64_t row = rb + lane / G;       // warp-uniform trip count
            A acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = A(0);
            if (row < r1) row_group_dot<T, V>(acc, Am + row * lda, x, n, lg, G);
            if constexpr (!gemv_one_chain<T>) {
#pragma unroll
                for (int w = 1; w < V; w <<= 1) {
#pragma unroll
                    for (int v = 0; v + w < V; v += 2 * w) acc[v] += acc[v + w];
                }
            }
            const A s = group_sum(acc[0], G);
            if (lg == 0 && row < r1) y[row] = narrow<T>(s);
        }
    }
}

// CSR instances are scheduled dynamically, one 32-row block per warp: lane 0
// takes tickets from a counter in the workspace (ticket t = unit t / wpb, the
// warp slot t % wpb within it), so the warps work through the units in order
// and the rows in flight at any time stay within a few instances, whose x
// vectors L2 then holds.  A static order (grid-stride or ranges) lets the
// blocks drift apart over a long launch until their x vectors no longer fit in
// L2: 4096 instances took 37.0 ms as one launch and 23.4 ms as sixteen launches
// of 256.  The next ticket is fetched while the current rows run.  The result
// does not depend on which warp takes a ticket.  The last warp to leave resets
// the counters for the next run (workspace: 8-byte ticket counter, then a
// 4-byte count of warps that have left).
template <typename T, int U>
__global__ void __launch_bounds__(512)
spmv_batch_kernel(const BatchHead *__restrict__ head, const int64_t *__restrict__ offs,
                  const CsrItem *__restrict__ items, unsigned long long *sched) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    __shared__ uint32_t rs_all[16][33];
    __shared__ Ac racc_all[16][32];
    const int64_t count = head->count, total = head->total_units;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    unsigned int *left = reinterpret_cast<unsigned int *>(sched + 1);
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(sched, 1ull);
    for (;;) {
        const unsigned long long t = __shfl_sync(0xffffffffu, next, 0);
        const int64_t u = (int64_t)(t / (unsigned long long)wpb);
        if (u >= total) break;                                        // warp-uniform
        if (lane == 0) next = atomicAdd(sched, 1ull);                 // in flight meanwhile
        const int64_t i = find_instance(offs, count, u);
        const CsrItem it = items[i];
        const int64_t nb = (it.d.m + 31) / 32;                        // 32-row blocks
        const int64_t b = (u - __ldg(offs + i)) * (it.rows_per_unit / 32) +
                          (int64_t)(t % (unsigned long long)wpb);
        if (b >= nb) continue;                                        // past the last rows
        const int64_t nnz = __ldg(it.d.row_ptr + it.d.m);
        if (it.vec_ok)
            seg_rows32<T, U, true>(static_cast<T *>(it.d.y), it.d.row_ptr, it.d.col_idx,
                                   static_cast<const T *>(it.d.vals),
                                   static_cast<const T *>(it.d.x), it.d.m, nnz, b,
                                   rs_all[warp], racc_all[warp]);
        else
            seg_rows32<T, U, false>(static_cast<T *>(it.d.y), it.d.row_ptr, it.d.col_idx,
                                    static_cast<const T *>(it.d.vals),
                                    static_cast<const T *>(it.d.x), it.d.m, nnz, b,
                                    rs_all[warp], racc_all[warp]);
    }
    if (lane == 0) {
        // every warp's last ticket was taken before it counts itself out, so
        // the last warp out may reset both counters
        __threadfence();
        if (atomicAdd(left, 1u) == gridDim.x * (unsigned int)wpb - 1u) {
            atomicExch(sched, 0ull);
            atomicExch(left, 0u);
        }
    }
}

// ---- host side ---------------------------------------------------------------

template <typename T>
lak_status run_typed(const lak_batch_info &info, const char *table, void *ws, dim3 grid,
                     int block, cudaStream_t s) {
    const BatchHead *head = reinterpret_cast<const BatchHead *>(table);
    const int64_t *offs = reinterpret_cast<const int64_t *>(table + kHeadBytes);
    const char *items = table + items_offset(info.count);
    const int vec = info.cfg.vec;
#define LAK_VECSW(KERNEL, ...)                                                              \
    switch (vec) {                                                                          \
    case 1: launch_k(KERNEL<T, 1>, grid, block, 0, s, __VA_ARGS__); break;                        \
    case 2: launch_k(KERNEL<T, 2>, grid, block, 0, s, __VA_ARGS__); break;                        \
    case 4: launch_k(KERNEL<T, 4>, grid, block, 0, s, __VA_ARGS__); break;                        \
    case 8: launch_k(KERNEL<T, 8>, grid, block, 0, s, __VA_ARGS__); break;                        \
    case 16: launch_k(KERNEL<T, 16>, grid, block, 0, s, __VA_ARGS__); break;                      \
    default: return fail(LAK_EINVAL, "lak_batch_run: unsupported vec %d", vec);             \
    }
    switch ((lak_op)info.op) {
    case LAK_OP_AXPY:
        LAK_VECSW(axpy_batch_kernel, head, offs, reinterpret_cast<const AxpyItem *>(items));
        break;
    case LAK_OP_DOT: {
        unsigned int *tickets = static_cast<unsigned int *>(ws);
        double *partials =
            reinterpret_cast<double *>(static_cast<char *>(ws) + LAK_WS_COUNTER_BYTES);
        LAK_VECSW(dot_batch_kernel, head, offs, reinterpret_cast<const DotItem *>(items), tickets,
                  partials);
        break;
    }
    case LAK_OP_GEMV_ROW: {
        const size_t ring = gemv_ring_smem(block, vec, (int)sizeof(T));
        switch (vec) {
        case 1: launch_k(gemv_batch_kernel<T, 1>, grid, block, ring, s, head, offs, reinterpret_cast<const GemvItem *>(items)); break;
        case 2: launch_k(gemv_batch_kernel<T, 2>, grid, block, ring, s, head, offs, reinterpret_cast<const GemvItem *>(items)); break;
        case 4: launch_k(gemv_batch_kernel<T, 4>, grid, block, ring, s, head, offs, reinterpret_cast<const GemvItem *>(items)); break;
        case 8: launch_k(gemv_batch_kernel<T, 8>, grid, block, ring, s, head, offs, reinterpret_cast<const GemvItem *>(items)); break;
        case 16: launch_k(gemv_batch_kernel<T, 16>, grid, block, ring, s, head, offs, reinterpret_cast<const GemvItem *>(items)); break;
        default: return fail(LAK_EINVAL, "lak_batch_run: unsupported vec %d", vec);
        }
        break;
    }
    case LAK_OP_SPMV:
        LAK_VECSW(spmv_batch_kernel, head, offs, reinterpret_cast<const CsrItem *>(items),
                  static_cast<unsigned long long *>(ws));
        break;
    default: return fail(LAK_EINVAL, "lak_batch_run: unsupported op %d", info.op);
    }
#undef LAK_VECSW
    return check_launch("lak_batch_run");
}

}  // namespace
}  // namespace lak

using namespace lak;

extern "C" {

LAK_API lak_status lak_batch_plan(lak_op op, lak_dtype dtype, const void *host_descs, int64_t count,
                                  const lak_cfg *cfg, void *host_table, size_t table_bytes,
                                  lak_batch_info *info) {
    if (!info) return fail(LAK_EINVAL, "lak_batch_plan: NULL info");
    if (op != LAK_OP_AXPY && op != LAK_OP_DOT && op != LAK_OP_GEMV_ROW && op != LAK_OP_SPMV)
        return fail(LAK_EINVAL, "lak_batch_plan: op %d has no batched form", (int)op);
    if (dtype != LAK_F32 && dtype != LAK_F64 && dtype != LAK_BF16 && dtype != LAK_F16)
        return fail(LAK_EDTYPE, "lak_batch_plan: unknown dtype %d", (int)dtype);
    if (count < 0 || (count > 0 && !host_descs))
        return fail(LAK_EINVAL, "lak_batch_plan: bad count or NULL descriptors");
    if (op == LAK_OP_DOT && count > LAK_WS_COUNTER_BYTES / 4)
        return fail(LAK_EINVAL, "lak_batch_plan: at most %d dot instances per batch",
                    LAK_WS_COUNTER_BYTES / 4);
    if (cfg && cfg->block != 0 &&
        (cfg->block < 32 || cfg->block > 512 || cfg->block % 32 || cfg->grid < 0 ||
         (cfg->vec != 0 && cfg->vec != 1 && cfg->vec != 2 && cfg->vec != 4 && cfg->vec != 8 &&
          cfg->vec != 16)))
        return fail(LAK_EINVAL, "lak_batch_plan: invalid cfg");
    const lak_cfg c = batch_config(op, dtype, cfg);
    if (op == LAK_OP_GEMV_ROW && c.block > kGemvBatchMaxBlock)
        return fail(LAK_EINVAL, "lak_batch_plan: batched GEMV takes at most %d threads per block",
                    kGemvBatchMaxBlock);
    int vec = c.vec;
    if (op == LAK_OP_SPMV) vec = vec < 4 ? 4 : (vec > 8 ? 8 : vec);   // seg rows: 4..8 entries
    const int es = esize(dtype);
    const int w = access_bytes(vec, es);
    // work units of about 256 KB of one operand: vectors and GEMV entries in
    // multiples of one pass of the block; CSR rows in multiples of the block's
    // rows (32 per warp), sized from the instance's mean row length
    const int64_t pass = (int64_t)c.block * vec;
    const int64_t ue = cdiv((int64_t)262144 / es, pass) * pass;
    // CSR: one block's rows per unit (32 per warp); co-resident blocks take
    // consecutive units of the same instance and share its x in L1
    auto csr_rows_per_unit = [&](const lak_csr_desc &) { return (int64_t)c.block; };
    auto gemv_item = [&](const lak_gemv_desc &d) {
        GemvItem it{};
        it.d = d;
        const int64_t rpu = d.n > 0 ? (cdiv(ue, d.n) < d.m ? cdiv(ue, d.n) : d.m) : d.m;
        it.rows_per_unit = rpu > 0 ? rpu : 1;
        it.vec_ok = aligned_to(d.A, w) && aligned_to(d.x, w) && (d.lda * es) % w == 0;
        // lanes per row: at least one 128-byte line of the row per warp
        // instruction (DRAM fetches whole lines), more while every lane
        // still sees about 4 vector groups
        int G = 1;
        while (G < 32 && (int64_t)G * vec * es < 128) G *= 2;
        while (G < 32 && (int64_t)G * 2 * vec * 4 <= d.n) G *= 2;
        it.group = G;
        it.period = 1;
        if (G >= 4) {
            // rows r and r + P start at the same offset modulo the access width
            const int64_t rb = (d.lda * es) % w;
            int P = 1;
            while ((rb * P) % w) ++P;
            it.period = P;
            const int64_t span = (int64_t)gemv_rows_per_group(w) * P;
            it.rows_per_unit = (it.rows_per_unit + span - 1) / span * span;
        }
        return it;
    };
    const size_t isz = item_size(op);
    const size_t need = items_offset(count) + isz * (size_t)count;

    // units per instance
    int64_t total = 0;
    for (int64_t i = 0; i < count; ++i) {
        int64_t units = 0;
        switch (op) {
        case LAK_OP_AXPY: {
            const lak_axpy_desc &d = static_cast<const lak_axpy_desc *>(host_descs)[i];
            if (d.n < 0) return fail(LAK_EINVAL, "lak_batch_plan: instance %lld: n < 0", (long long)i);
            units = cdiv(d.n, ue);
            break;
        }
        case LAK_OP_DOT: {
            const lak_dot_desc &d = static_cast<const lak_dot_desc *>(host_descs)[i];
            if (d.n < 0) return fail(LAK_EINVAL, "lak_batch_plan: instance %lld: n < 0", (long long)i);
            units = d.n > 0 ? cdiv(d.n, ue) : 1;        // an empty dot still writes 0
            break;
        }
        case LAK_OP_GEMV_ROW: {
            const lak_gemv_desc &d = static_cast<const lak_gemv_desc *>(host_descs)[i];
            if (d.m < 0 || d.n < 0 || d.lda < (d.n > 1 ? d.n : 1))
                return fail(LAK_EINVAL, "lak_batch_plan: instance %lld: bad m, n or lda", (long long)i);
            units = d.m > 0 ? cdiv(d.m, gemv_item(d).rows_per_unit) : 0;
            break;
        }
        case LAK_OP_SPMV: {
            const lak_csr_desc &d = static_cast<const lak_csr_desc *>(host_descs)[i];
            if (d.m < 0 || d.n < 0 || d.nnz < 0 || d.nnz > 0x7fffffffLL)
                return fail(LAK_EINVAL, "lak_batch_plan: instance %lld: bad sizes", (long long)i);
            units = cdiv(d.m, csr_rows_per_unit(d));
            break;
        }
        default: break;
        }
        total += units;
    }
    info->count = count;
    info->total_units = total;
    info->unit_elems = ue;
    info->table_bytes = need;
    info->workspace_bytes =
        op == LAK_OP_DOT    ? (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)total
        : op == LAK_OP_SPMV ? (size_t)LAK_WS_COUNTER_BYTES     // ticket counters
                            : 0;
    info->cfg = lak_cfg{c.block, c.grid, vec, c.increment};
    info->op = (int32_t)op;
    info->dtype = (int32_t)dtype;
    if (!host_table) return LAK_OK;
    if (table_bytes < need)
        return fail(LAK_EINVAL, "lak_batch_plan: table of %zu bytes needed, %zu given", need,
                    table_bytes);
    char *t = static_cast<char *>(host_table);
    memset(t, 0, need);
    BatchHead *h = reinterpret_cast<BatchHead *>(t);
    h->count = count;
    h->total_units = total;
    h->unit_elems = ue;
    h->op = (int32_t)op;
    h->dtype = (int32_t)dtype;
    h->vec = vec;
    h->block = c.block;
    h->inc = c.increment;
    int64_t *offs = reinterpret_cast<int64_t *>(t + kHeadBytes);
    char *items = t + items_offset(count);
    int64_t acc = 0;
    for (int64_t i = 0; i < count; ++i) {
        offs[i] = acc;
        switch (op) {
        case LAK_OP_AXPY: {
            const lak_axpy_desc &d = static_cast<const lak_axpy_desc *>(host_descs)[i];
            AxpyItem it{};
            it.d = d;
            it.units = cdiv(d.n, ue);
            it.vec_ok = aligned_to(d.x, w) && aligned_to(d.y, w) && aligned_to(d.z, w);
            memcpy(items + isz * i, &it, sizeof it);
            acc += it.units;
            break;
        }
        case LAK_OP_DOT: {
            const lak_dot_desc &d = static_cast<const lak_dot_desc *>(host_descs)[i];
            DotItem it{};
            it.d = d;
            it.units = d.n > 0 ? cdiv(d.n, ue) : 1;
            it.vec_ok = aligned_to(d.x, w) && aligned_to(d.y, w);
            memcpy(items + isz * i, &it, sizeof it);
            acc += it.units;
            break;
        }
        case LAK_OP_GEMV_ROW: {
            const lak_gemv_desc &d = static_cast<const lak_gemv_desc *>(host_descs)[i];
            GemvItem it = gemv_item(d);
            memcpy(items + isz * i, &it, sizeof it);
            acc += d.m > 0 ? cdiv(d.m, it.rows_per_unit) : 0;
            break;
        }
        case LAK_OP_SPMV: {
            const lak_csr_desc &d = static_cast<const lak_csr_desc *>(host_descs)[i];
            CsrItem it{};
            it.d = d;
            it.rows_per_unit = csr_rows_per_unit(d);
            it.vec_ok = aligned_to(d.col_idx, 16) && aligned_to(d.vals, 16);
            memcpy(items + isz * i, &it, sizeof it);
            acc += cdiv(d.m, it.rows_per_unit);
            break;
        }
        default: break;
        }
    }
    offs[count] = acc;
    return LAK_OK;
}

LAK_API lak_status lak_batch_run(const lak_batch_info *info, const void *dev_table, void *workspace,
                                 size_t ws_bytes, void *stream) {
    if (!info) return fail(LAK_EINVAL, "lak_batch_run: NULL info");
    if (info->count < 0 || info->total_units < 0)
        return fail(LAK_EINVAL, "lak_batch_run: bad info");
    if (info->total_units == 0) return LAK_OK;
    if (!dev_table || (uintptr_t)dev_table % 16)
        return fail(LAK_EINVAL, "lak_batch_run: table must be a 16-byte aligned device buffer");
    if (info->workspace_bytes > 0) {
        if (!workspace || ws_bytes < info->workspace_bytes)
            return fail(LAK_EWORKSPACE, "lak_batch_run: workspace of %zu bytes needed, %zu given",
                        info->workspace_bytes, workspace ? ws_bytes : (size_t)0);
        if ((uintptr_t)workspace % 256)
            return fail(LAK_EWORKSPACE, "lak_batch_run: workspace not 256-byte aligned");
    }
    const int block = info->cfg.block;
    if (block < 32 || block > 512 || block % 32 ||
        (info->op == LAK_OP_GEMV_ROW && block > kGemvBatchMaxBlock))
        return fail(LAK_EINVAL, "lak_batch_run: bad block %d", block);
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    int64_t grid = info->cfg.grid;
    if (grid <= 0) grid = (int64_t)di->sms * (di->max_threads_per_sm / block);
    if (grid > info->total_units) grid = info->total_units;
    const char *table = static_cast<const char *>(dev_table);
    cudaStream_t s = (cudaStream_t)stream;
    switch ((lak_dtype)info->dtype) {
    case LAK_F32: return run_typed<float>(*info, table, workspace, dim3((unsigned)grid), block, s);
    case LAK_F64: return run_typed<double>(*info, table, workspace, dim3((unsigned)grid), block, s);
    case LAK_BF16:
        return run_typed<__nv_bfloat16>(*info, table, workspace, dim3((unsigned)grid), block, s);
    case LAK_F16: return run_typed<__half>(*info, table, workspace, dim3((unsigned)grid), block, s);
    }
    return fail(LAK_EDTYPE, "lak_batch_run: unknown dtype %d", info->dtype);
}

}  // extern "C"
