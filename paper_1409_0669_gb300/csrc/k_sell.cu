// Sliced ELLPACK (SELL-C-sigma, C = 32): an SpMV format variant of the CSR
// product for matrices whose rows a warp can process in lockstep.
//
// Layout (the same as the oracle's): rows are ordered by decreasing length
// within windows of `sigma` rows (sigma = 1: no reordering), ties by row index;
// position p of that order holds original row perm[p] (-1 for padding past the
// last row).  Slice s = positions 32s .. 32s+31, padded to its longest row
// (slice_len[s] entries per row), stored column-major from slice_ptr[s]: entry
// j of the row at position 32s + r is slot slice_ptr[s] + 32j + r.  cols holds
// the column or -1 (padding); map holds the CSR position or -1.
//
// Product: one warp per slice, lane r owns the row at position 32s + r; every
// load of cols / vals is 32 consecutive slots (128 coalesced bytes for 4-byte
// data), there are no per-row row-pointer loads, and each row's entries are
// added in stored order (the CSR order).
#include "lak_internal.cuh"

namespace lak {
namespace {

constexpr int kC = 32;
constexpr int kMaxSigma = 4096;

__global__ void identity_perm_kernel(int32_t *perm, int64_t m, int64_t mp) {
    LAK_PDL_ENTRY();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < mp;
         p += (int64_t)gridDim.x * blockDim.x)
        perm[p] = p < m ? (int32_t)p : -1;
}

// One block per window: rank each row by (length desc, index asc).
__global__ void window_sort_kernel(int32_t *perm, const int32_t *__restrict__ rp, int64_t m,
                                   int64_t mp, int sigma) {
    LAK_PDL_ENTRY();
    extern __shared__ int32_t lens[];
    const int64_t w0 = (int64_t)blockIdx.x * sigma;
    const int wn = (int)(mp - w0 < sigma ? mp - w0 : sigma);
    for (int t = threadIdx.x; t < wn; t += blockDim.x) {
        const int64_t p = w0 + t;
        lens[t] = p < m ? (int32_t)(rp[p + 1] - rp[p]) : -1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < wn; t += blockDim.x) {
        const int32_t l = lens[t];
        int rank = 0;
        for (int u = 0; u < wn; ++u) {
            const int32_t lu = lens[u];
            rank += (lu > l) || (lu == l && u < t);
        }
        const int64_t p = w0 + t;
        perm[w0 + rank] = p < m ? (int32_t)p : -1;
    }
}

// One warp per slice: the longest row of the slice.
__global__ void slice_len_kernel(int32_t *slen, const int32_t *__restrict__ perm,
                                 const int32_t *__restrict__ rp, int64_t ns) {
    LAK_PDL_ENTRY();
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = gw; s < ns; s += nw) {
        const int32_t i = perm[s * kC + lane];
        int32_t l = i >= 0 ? rp[i + 1] - rp[i] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int32_t u = __shfl_xor_sync(0xffffffffu, l, o);
            l = u > l ? u : l;
        }
        if (lane == 0) slen[s] = l;
    }
}

// Single block: slice_ptr = exclusive prefix of 32 * slice_len; slice_ptr[ns] = total.
__global__ void __launch_bounds__(1024)
slice_ptr_kernel(int64_t *sptr, const int32_t *__restrict__ slen, int64_t ns) {
    LAK_PDL_ENTRY();
    __shared__ int64_t part[1024];
    const int T = blockDim.x;
    const int64_t per = (ns + T - 1) / T;
    const int64_t b = threadIdx.x * per;
    const int64_t e = b + per < ns ? b + per : ns;
    int64_t sum = 0;
    for (int64_t s = b; s < e; ++s) sum += (int64_t)kC * slen[s];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {              // inclusive Hillis-Steele scan
        const int64_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = part[threadIdx.x] - sum;
    for (int64_t s = b; s < e; ++s) {
        sptr[s] = run;
        run += (int64_t)kC * slen[s];
    }
    if (threadIdx.x == T - 1) sptr[ns] = part[T - 1];
}

__global__ void fill_kernel(int32_t *cols, int32_t *map, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ slen, const int64_t *__restrict__ sptr,
                            int64_t mp) {
    LAK_PDL_ENTRY();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < mp;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = p / kC;
        const int r = (int)(p % kC);
        const int32_t i = perm[p];
        const int64_t k0 = i >= 0 ? rp[i] : 0;
        const int64_t li = i >= 0 ? rp[i + 1] - k0 : 0;
        const int32_t L = slen[s];
        const int64_t base = sptr[s] + r;
        for (int32_t j = 0; j < L; ++j) {
            const int64_t slot = base + (int64_t)j * kC;
            if (j < li) {
                cols[slot] = ci[k0 + j];
                map[slot] = (int32_t)(k0 + j);
            } else {
                cols[slot] = -1;
                map[slot] = -1;
            }
        }
    }
}

template <typename E>
__global__ void pack_kernel(E *__restrict__ dst, const E *__restrict__ src,
                            const int32_t *__restrict__ map, int64_t total) {
    LAK_PDL_ENTRY();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = map[q];
        dst[q] = k >= 0 ? src[k] : E(0);
    }
}

template <typename T, int U>
__global__ void __launch_bounds__(512)
sell_spmv_kernel(T *__restrict__ y, const int64_t *__restrict__ sptr,
                 const int32_t *__restrict__ slen, const int32_t *__restrict__ perm,
                 const int32_t *__restrict__ cols, const T *__restrict__ vals,
                 const T *__restrict__ x, int64_t ns, int inc) {
    LAK_PDL_ENTRY();
    using Ac = typename Acc<T>::type;
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * wpb;
    int64_t s0, s1, step;
    if (inc == LAK_INC_GLOBAL) {
        s0 = gw;
        s1 = ns;
        step = nw;
    } else {
        const int64_t per = (ns + nw - 1) / nw;
        s0 = gw * per;
        s1 = s0 + per < ns ? s0 + per : ns;
        step = 1;
    }
    for (int64_t s = s0; s < s1; s += step) {
        const int64_t base = __ldg(sptr + s) + lane;
        const int32_t L = __ldg(slen + s);
        const int32_t i = __ldg(perm + s * kC + lane);
        Ac acc = Ac(0);
        for (int32_t j0 = 0; j0 < L; j0 += U) {
            int32_t c[U];
            T v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j0 + u < L) {
                    const int64_t slot = base + (int64_t)(j0 + u) * kC;
                    ld_raw<4, STREAM>(&c[u], cols + slot);
                    ld_raw<(int)sizeof(T), STREAM>(&v[u], vals + slot);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j0 + u < L && c[u] >= 0)
                    acc = fma_acc(widen(v[u]), widen(ld_cached(x + c[u])), acc);
        }
        if (i >= 0) y[i] = narrow<T>(acc);
    }
}

int grid_cap(int block) {
    const DeviceInfo *di = device_info();
    return di ? di->sms * (di->max_threads_per_sm / block) : 1024;
}

int grid_for(int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    const int64_t cap = grid_cap(block);
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <typename T>
lak_status sell_spmv_t(void *y, const int64_t *sptr, const int32_t *slen, const int32_t *perm,
                       const int32_t *cols, const void *vals, const void *x, int64_t ns,
                       const lak_cfg &c, cudaStream_t s) {
    T *yp = static_cast<T *>(y);
    const T *vp = static_cast<const T *>(vals);
    const T *xp = static_cast<const T *>(x);
    const int64_t wpb = c.block / 32;
    int64_t grid = c.grid > 0 ? c.grid : (ns + wpb - 1) / wpb;
    if (grid > 0x7fffffff) grid = 0x7fffffff;
#define LAK_SELL(UU) \
    launch_k(sell_spmv_kernel<T, UU>, (unsigned)grid, c.block, 0, s, yp, sptr, slen, perm, cols, vp, xp, \
                                                                ns, c.increment)
    switch (c.vec) {
    case 1: LAK_SELL(1); break;
    case 2: LAK_SELL(2); break;
    case 4: LAK_SELL(4); break;
    case 8: LAK_SELL(8); break;
    case 16: LAK_SELL(16); break;
    default: return fail(LAK_EINVAL, "sell_spmv: unsupported vec %d", c.vec);
    }
#undef LAK_SELL
    return check_launch("sell_spmv");
}

bool valid_dt(lak_dtype dt) { return dt == LAK_F32 || dt == LAK_F64 || dt == LAK_BF16 || dt == LAK_F16; }

}  // namespace
}  // namespace lak

using namespace lak;

extern "C" {

LAK_API lak_status csr_to_sell_count(const int32_t *row_ptr, int64_t m, int32_t sigma,
                                     int32_t *perm, int32_t *slice_len, int64_t *slice_ptr,
                                     void *stream) {
    if (m < 0) return fail(LAK_EINVAL, "csr_to_sell_count: m < 0");
    if (!(sigma == 1 || (sigma >= kC && sigma % kC == 0 && sigma <= kMaxSigma)))
        return fail(LAK_EINVAL,
                    "csr_to_sell_count: sigma=%d must be 1 or a multiple of 32 up to %d", sigma,
                    kMaxSigma);
    if (!slice_ptr) return fail(LAK_EINVAL, "csr_to_sell_count: NULL slice_ptr");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t mp = (m + kC - 1) / kC * kC;
    const int64_t ns = mp / kC;
    if (ns == 0) {
        const cudaError_t e = cudaMemsetAsync(slice_ptr, 0, 8, s);
        if (e != cudaSuccess) return fail(LAK_ECUDA, "csr_to_sell_count: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    if (!row_ptr || !perm || !slice_len) return fail(LAK_EINVAL, "csr_to_sell_count: NULL pointer");
    const int block = 256;
    if (sigma == 1)
        launch_k(identity_perm_kernel, grid_for(mp, block), block, 0, s, perm, m, mp);
    else
        launch_k(window_sort_kernel, (unsigned)((mp + sigma - 1) / sigma), 256, sigma * 4, s, 
            perm, row_ptr, m, mp, sigma);
    launch_k(slice_len_kernel, grid_for(ns * 32, block), block, 0, s, slice_len, perm, row_ptr, ns);
    launch_k(slice_ptr_kernel, 1, 1024, 0, s, slice_ptr, slice_len, ns);
    return check_launch("csr_to_sell_count");
}

LAK_API lak_status csr_to_sell_fill(const int32_t *row_ptr, const int32_t *col_idx, int64_t m,
                                    const int32_t *perm, const int32_t *slice_len,
                                    const int64_t *slice_ptr, int32_t *cols, int32_t *map,
                                    void *stream) {
    if (m < 0) return fail(LAK_EINVAL, "csr_to_sell_fill: m < 0");
    if (m == 0) return LAK_OK;
    if (!row_ptr || !perm || !slice_len || !slice_ptr || !cols || !map)
        return fail(LAK_EINVAL, "csr_to_sell_fill: NULL pointer");
    const int64_t mp = (m + kC - 1) / kC * kC;
    const int block = 256;
    launch_k(fill_kernel, grid_for(mp, block), block, 0, (cudaStream_t)stream, 
        cols, map, row_ptr, col_idx, perm, slice_len, slice_ptr, mp);
    return check_launch("csr_to_sell_fill");
}

LAK_API lak_status sell_pack_values(void *sell_vals, const void *csr_vals, const int32_t *map,
                                    int64_t total, lak_dtype dtype, void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "sell_pack_values: unknown dtype %d", (int)dtype);
    if (total < 0) return fail(LAK_EINVAL, "sell_pack_values: total < 0");
    if (total == 0) return LAK_OK;
    if (!sell_vals || !map) return fail(LAK_EINVAL, "sell_pack_values: NULL pointer");
    const int block = 256;
    const int grid = grid_for(total, block);
    cudaStream_t s = (cudaStream_t)stream;
    switch (esize(dtype)) {
    case 2: launch_k(pack_kernel<uint16_t>, grid, block, 0, s, (uint16_t *)sell_vals, (const uint16_t *)csr_vals, map, total); break;
    case 4: launch_k(pack_kernel<uint32_t>, grid, block, 0, s, (uint32_t *)sell_vals, (const uint32_t *)csr_vals, map, total); break;
    case 8: launch_k(pack_kernel<uint64_t>, grid, block, 0, s, (uint64_t *)sell_vals, (const uint64_t *)csr_vals, map, total); break;
    }
    return check_launch("sell_pack_values");
}

LAK_API lak_status sell_spmv(void *y, const int64_t *slice_ptr, const int32_t *slice_len,
                             const int32_t *perm, const int32_t *cols, const void *vals,
                             const void *x, int64_t m, lak_dtype dtype, const lak_cfg *cfg,
                             void *stream) {
    if (!valid_dt(dtype)) return fail(LAK_EDTYPE, "sell_spmv: unknown dtype %d", (int)dtype);
    if (m < 0) return fail(LAK_EINVAL, "sell_spmv: m < 0");
    if (m == 0) return LAK_OK;
    if (!y || !slice_ptr || !slice_len || !perm)
        return fail(LAK_EINVAL, "sell_spmv: NULL pointer");
    lak_cfg c{256, 0, 4, LAK_INC_GLOBAL};
    if (cfg && cfg->block != 0) {
        c = *cfg;
        if (c.block < 32 || c.block > 512 || c.block % 32 || c.grid < 0 ||
            (c.increment != LAK_INC_GLOBAL && c.increment != LAK_INC_LOCAL))
            return fail(LAK_EINVAL, "sell_spmv: invalid cfg");
        if (c.vec == 0) c.vec = 4;
    }
    const int64_t ns = (m + kC - 1) / kC;
    cudaStream_t s = (cudaStream_t)stream;
    switch (dtype) {
    case LAK_F32: return sell_spmv_t<float>(y, slice_ptr, slice_len, perm, cols, vals, x, ns, c, s);
    case LAK_F64: return sell_spmv_t<double>(y, slice_ptr, slice_len, perm, cols, vals, x, ns, c, s);
    case LAK_BF16: return sell_spmv_t<__nv_bfloat16>(y, slice_ptr, slice_len, perm, cols, vals, x, ns, c, s);
    case LAK_F16: return sell_spmv_t<__half>(y, slice_ptr, slice_len, perm, cols, vals, x, ns, c, s);
    }
    return LAK_EDTYPE;
}

}  // extern "C"
