// Internal declarations shared by the library's translation units: storage
// type traits, wide load/store primitives (inline PTX, up to 256-bit), warp
// reductions, the resolved launch description and host-side error helpers.
// Nothing here is part of the C ABI (include/lak.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "lak.h"

namespace lak {

// ---------------------------------------------------------------------------
// Host side: errors, device facts, resolved launch shape
// ---------------------------------------------------------------------------

// Records a printf-style message for lak_last_error() and returns `st`.
lak_status fail(lak_status st, const char *fmt, ...);

// Maps a pending launch error to LAK_ECUDA (message names `what`), else LAK_OK.
lak_status check_launch(const char *what);

struct DeviceInfo {
    int device;
    int sms;                 // streaming multiprocessors (152 on GB300)
    int max_threads_per_sm;  // 2048 on sm_103a
};

// Facts about the current device, cached per device ordinal; nullptr (with
// the message set) if the runtime cannot answer.
const DeviceInfo *device_info();

// A launch after defaults and automatic fields are filled in.
struct Launch {
    int block;   // threads per block
    int grid;    // blocks (for column-major GEMV: total over both grid axes)
    int vec;     // elements per access group (see lak_cfg)
    int inc;     // LAK_INC_GLOBAL / LAK_INC_LOCAL
};

inline int esize(lak_dtype dt) {
    switch (dt) {
    case LAK_F32: return 4;
    case LAK_F64: return 8;
    case LAK_BF16: return 2;
    case LAK_F16: return 2;
    }
    return 0;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Widest single access (bytes) used for a group of `vec` elements.
inline int access_bytes(int vec, int es) {
    int b = vec * es;
    return b > 32 ? 32 : b;
}

// Programmatic dependent launch (sm_90 and later).  Every kernel of the library
// begins with LAK_PDL_ENTRY(): it waits until the kernel before it in the stream
// has completed and its writes are visible (griddepcontrol.wait; a no-op when
// the launch did not ask for programmatic serialization), then lets the next
// kernel in the stream start launching (griddepcontrol.launch_dependents: the
// next grid is scheduled once every block of this one has started, so its
// launch and block set-up overlap this grid's tail instead of following it).
// No kernel touches global memory before the wait, so the stream's ordering is
// unchanged; launch_k launches with the attribute unless LAK_PDL=0.  (The
// batched GEMV only waits; it lets its dependents launch when it completes.)
#define LAK_PDL_ENTRY()                                              \
    do {                                                             \
        asm volatile("griddepcontrol.wait;" ::: "memory");           \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
    } while (0)

// Host: whether launches ask for programmatic serialization (LAK_PDL, read once).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                            cudaStream_t s, Args &&...args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// Largest block of the batched GEMV kernel (its register budget is set for it).
constexpr int kGemvBatchMaxBlock = 128;

// The configuration a batched launch starts from (explicit cfg, else the
// batched kernels' own defaults), with vec filled in; host only, no CUDA
// call; grid left as given.
lak_cfg batch_config(lak_op op, lak_dtype dt, const lak_cfg *cfg);

// Largest vec <= want (power of two) whose access width divides the byte
// offsets of every pointer in `ptrs` modulo the access width identically, so
// that one scalar prologue aligns all of them at once.  Also returns the
// prologue length (elements) in *head.
int pick_vec(int want, int es, const void *const *ptrs, int nptrs, int64_t n, int64_t *head);

// The launch vec_dot makes for these operands (configuration, the vector
// width both pointers' alignment allows, the grid for that width) and its
// scalar prologue length; other entry points that run the dot kernel take it
// from here so that they sum in the same block order.
lak_status plan_dot(const char *who, lak_dtype dt, int64_t n, const lak_cfg *cfg, const void *x,
                    const void *y, Launch *L, int64_t *head);

// Launchers (one per kernel family), called after validation.
lak_status launch_copy(void *x, const void *y, int64_t n, int es, const Launch &L,
                       int64_t head, cudaStream_t s);
lak_status launch_axpy(lak_dtype dt, void *x, const void *y, const void *z, double alpha,
                       int64_t n, const Launch &L, int64_t head, cudaStream_t s);
lak_status launch_dot(lak_dtype dt, void *out, const void *x, const void *y, int64_t n,
                      void *ws, const Launch &L, int64_t head, cudaStream_t s);
lak_status launch_dot_comp(lak_dtype dt, void *out, const void *x, const void *y, int64_t n,
                           void *ws, const Launch &L, int64_t head, cudaStream_t s);
lak_status launch_axpby(lak_dtype dt, void *x, double alpha, const void *y, double beta,
                        const void *z, int64_t n, const Launch &L, int64_t head, cudaStream_t s);
lak_status launch_axpby_strided(lak_dtype dt, void *x, int64_t incx, double alpha, const void *y,
                                int64_t incy, double beta, const void *z, int64_t incz, int64_t n,
                                int grid, int block, cudaStream_t s);
lak_status launch_dot_sparse(lak_dtype dt, void *out, const void *vals, const int32_t *idx,
                             const void *y, int64_t nnz, void *ws, const Launch &L, int64_t head,
                             cudaStream_t s);
lak_status launch_axpy_norm2(lak_dtype dt, void *x, const void *y, const void *z, double alpha,
                             void *out, int64_t n, void *ws, const Launch &L, int64_t head,
                             cudaStream_t s);
// GEMV launchers compute y = alpha*A*x + beta*y (y is not read when beta == 0).
lak_status launch_gemv_row(lak_dtype dt, void *y, const void *A, const void *x, int64_t m,
                           int64_t n, int64_t lda, const Launch &L, int group, double alpha,
                           double beta, cudaStream_t s);
lak_status launch_gemv_col(lak_dtype dt, void *y, const void *A, const void *x, int64_t m,
                           int64_t n, int64_t lda, const Launch &L, int splits, void *ws,
                           double alpha, double beta, cudaStream_t s);
lak_status launch_spmv(lak_dtype dt, void *y, const int32_t *rp, const int32_t *ci,
                       const void *vals, const void *x, int64_t m, const Launch &L, int group,
                       cudaStream_t s);

// ---------------------------------------------------------------------------
// Device side: storage traits and conversions
// ---------------------------------------------------------------------------

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float widen(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T narrow(typename Acc<T>::type v);
template <> __device__ __forceinline__ float narrow<float>(float v) { return v; }
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 narrow<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half narrow<__half>(float v) { return __float2half_rn(v); }

// fused multiply-add in the arithmetic type: one rounding
__device__ __forceinline__ float fma_acc(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_acc(double a, double b, double c) { return __fma_rn(a, b, c); }

// a * b + c for two stored values and the accumulator, rounded once.  FP32 and
// FP64 storage: one FMA.  16-bit storage: one mixed-precision FMA (16-bit
// factors, FP32 addend and result) -- widening a 16-bit value to FP32 is exact,
// so this is the same FMA on the same values as widening both factors first
// (one PTX instruction instead of two conversions and an FMA; the results are
// bit-identical).  The dense products use it: BF16 / FP16 GEMV 2-4 % faster
// (row-major, column-major, batched).  The streaming inner products keep the
// widened form, which measured 11 % faster there.
__device__ __forceinline__ float fma_wide(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_wide(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_wide(__nv_bfloat16 a, __nv_bfloat16 b, float c) {
    float d;
    asm("fma.rn.f32.bf16 %0, %1, %2, %3;"
        : "=f"(d) : "h"(__bfloat16_as_ushort(a)), "h"(__bfloat16_as_ushort(b)), "f"(c));
    return d;
}
__device__ __forceinline__ float fma_wide(__half a, __half b, float c) {
    float d;
    asm("fma.rn.f32.f16 %0, %1, %2, %3;"
        : "=f"(d) : "h"(__half_as_ushort(a)), "h"(__half_as_ushort(b)), "f"(c));
    return d;
}

// ---------------------------------------------------------------------------
// Device side: wide loads and stores
// ---------------------------------------------------------------------------

template <typename T, int V> struct Pack { T e[V]; };

// Load policies.  STREAM: read-only path, no L1 allocation (data read once and
// not written by the kernel).  COHERENT: ordinary coherent load, no L1
// allocation (an output may alias this input).  CACHED: read-only path with
// L1 allocation (operands many threads re-read, e.g. the GEMV right-hand side).
enum { STREAM = 0, COHERENT = 1, CACHED = 2 };

template <int B, int P> __device__ __forceinline__ void ld_raw(void *dst, const void *p);

template <> __device__ __forceinline__ void ld_raw<2, STREAM>(void *dst, const void *p) {
    unsigned short h;
    asm("ld.global.nc.L1::no_allocate.b16 %0, [%1];" : "=h"(h) : "l"(p));
    memcpy(dst, &h, 2);
}
template <> __device__ __forceinline__ void ld_raw<2, COHERENT>(void *dst, const void *p) {
    unsigned short h;
    asm("ld.global.L1::no_allocate.b16 %0, [%1];" : "=h"(h) : "l"(p));
    memcpy(dst, &h, 2);
}
template <> __device__ __forceinline__ void ld_raw<4, STREAM>(void *dst, const void *p) {
    uint32_t w;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(w) : "l"(p));
    memcpy(dst, &w, 4);
}
template <> __device__ __forceinline__ void ld_raw<4, COHERENT>(void *dst, const void *p) {
    uint32_t w;
    asm("ld.global.L1::no_allocate.b32 %0, [%1];" : "=r"(w) : "l"(p));
    memcpy(dst, &w, 4);
}
template <> __device__ __forceinline__ void ld_raw<8, STREAM>(void *dst, const void *p) {
    uint32_t w[2];
    asm("ld.global.nc.L1::no_allocate.v2.b32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    memcpy(dst, w, 8);
}
template <> __device__ __forceinline__ void ld_raw<8, COHERENT>(void *dst, const void *p) {
    uint32_t w[2];
    asm("ld.global.L1::no_allocate.v2.b32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    memcpy(dst, w, 8);
}
template <> __device__ __forceinline__ void ld_raw<16, STREAM>(void *dst, const void *p) {
    uint32_t w[4];
    asm("ld.global.nc.L1::no_allocate.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    memcpy(dst, w, 16);
}
template <> __device__ __forceinline__ void ld_raw<16, COHERENT>(void *dst, const void *p) {
    uint32_t w[4];
    asm("ld.global.L1::no_allocate.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    memcpy(dst, w, 16);
}
// 256-bit loads (sm_100 and later).
template <> __device__ __forceinline__ void ld_raw<32, STREAM>(void *dst, const void *p) {
    uint32_t w[8];
    asm("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
    memcpy(dst, w, 32);
}
template <> __device__ __forceinline__ void ld_raw<32, COHERENT>(void *dst, const void *p) {
    uint32_t w[8];
    asm("ld.global.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
    memcpy(dst, w, 32);
}

template <> __device__ __forceinline__ void ld_raw<2, CACHED>(void *dst, const void *p) {
    unsigned short h;
    asm("ld.global.nc.b16 %0, [%1];" : "=h"(h) : "l"(p));
    memcpy(dst, &h, 2);
}
template <> __device__ __forceinline__ void ld_raw<4, CACHED>(void *dst, const void *p) {
    uint32_t w;
    asm("ld.global.nc.b32 %0, [%1];" : "=r"(w) : "l"(p));
    memcpy(dst, &w, 4);
}
template <> __device__ __forceinline__ void ld_raw<8, CACHED>(void *dst, const void *p) {
    uint32_t w[2];
    asm("ld.global.nc.v2.b32 {%0,%1}, [%2];" : "=r"(w[0]), "=r"(w[1]) : "l"(p));
    memcpy(dst, w, 8);
}
template <> __device__ __forceinline__ void ld_raw<16, CACHED>(void *dst, const void *p) {
    uint32_t w[4];
    asm("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]) : "l"(p));
    memcpy(dst, w, 16);
}
template <> __device__ __forceinline__ void ld_raw<32, CACHED>(void *dst, const void *p) {
    uint32_t w[8];
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7])
        : "l"(p));
    memcpy(dst, w, 32);
}

template <int B> __device__ __forceinline__ void st_raw(void *p, const void *src);
template <> __device__ __forceinline__ void st_raw<2>(void *p, const void *src) {
    unsigned short h;
    memcpy(&h, src, 2);
    asm volatile("st.global.b16 [%0], %1;" ::"l"(p), "h"(h));
}
template <> __device__ __forceinline__ void st_raw<4>(void *p, const void *src) {
    uint32_t w;
    memcpy(&w, src, 4);
    asm volatile("st.global.b32 [%0], %1;" ::"l"(p), "r"(w));
}
template <> __device__ __forceinline__ void st_raw<8>(void *p, const void *src) {
    uint32_t w[2];
    memcpy(w, src, 8);
    asm volatile("st.global.v2.b32 [%0], {%1,%2};" ::"l"(p), "r"(w[0]), "r"(w[1]));
}
template <> __device__ __forceinline__ void st_raw<16>(void *p, const void *src) {
    uint32_t w[4];
    memcpy(w, src, 16);
    asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]));
}
template <> __device__ __forceinline__ void st_raw<32>(void *p, const void *src) {
    uint32_t w[8];
    memcpy(w, src, 32);
    asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7]));
}

// Load V consecutive elements starting at p (aligned to min(V*sizeof(T), 32)).
template <typename T, int V, int P>
__device__ __forceinline__ void load_pack(Pack<T, V> &pk, const T *p) {
    constexpr int B = V * (int)sizeof(T);
    if constexpr (B <= 32) {
        ld_raw<B, P>(&pk, p);
    } else {
        static_assert(B % 32 == 0, "pack size");
#pragma unroll
        for (int c = 0; c < B / 32; ++c)
            ld_raw<32, P>(reinterpret_cast<char *>(&pk) + 32 * c,
                           reinterpret_cast<const char *>(p) + 32 * c);
    }
}

template <typename T, int V>
__device__ __forceinline__ void store_pack(T *p, const Pack<T, V> &pk) {
    constexpr int B = V * (int)sizeof(T);
    if constexpr (B <= 32) {
        st_raw<B>(p, &pk);
    } else {
#pragma unroll
        for (int c = 0; c < B / 32; ++c)
            st_raw<32>(reinterpret_cast<char *>(p) + 32 * c,
                       reinterpret_cast<const char *>(&pk) + 32 * c);
    }
}

// Cached (L1-allocating) read-only scalar load, for operands that many
// threads re-read (the right-hand side x of GEMV / SpMV).
template <typename T> __device__ __forceinline__ T ld_cached(const T *p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// Device side: reductions
// ---------------------------------------------------------------------------

// Sum over aligned groups of `width` lanes (width a power of two <= 32); every
// lane of the warp must call it.  All lanes of a group end with the sum.
template <typename A> __device__ __forceinline__ A group_sum(A v, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Arrival ticket at GPU scope, one instruction: the increment wraps back to 0
// after `last`, release orders the caller's earlier stores (its block partial)
// before it, and acquire orders the caller's later loads after every earlier
// arrival's release.
__device__ __forceinline__ unsigned int ticket_acq_rel(unsigned int *counter, unsigned int last) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.inc.u32 %0, [%1], %2;"
                 : "=r"(old) : "l"(counter), "r"(last) : "memory");
    return old;
}

// Deterministic sum over the whole grid of one value per thread, written to
// *out: a warp reduction in A, FP64 across the block's warps into one partial
// per block, and the last block to arrive (ticket on *counter, which wraps
// back to 0 for the next launch) adds the partials in block order; a grid of
// one block writes its sum directly (the same value: the last-block pass adds
// only zeros to it).  Every thread of every block must call it, as the
// kernel's last action.
template <typename A, typename OutT>
__device__ __forceinline__ void grid_sum_last_block(A v, OutT *out, unsigned int *counter,
                                                    double *partials) {
    __shared__ double wsum[32];
    __shared__ int am_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    const A s = group_sum(v, 32);
    if (lane == 0) wsum[warp] = (double)s;
    __syncthreads();
    if (warp == 0) {
        double b = lane < nwarps ? wsum[lane] : 0.0;
        b = group_sum(b, 32);
        if (lane == 0) {
            if (gridDim.x == 1) {
                *out = static_cast<OutT>(b);
                am_last = 0;
            } else {
                partials[blockIdx.x] = b;
                am_last = ticket_acq_rel(counter, gridDim.x - 1) == gridDim.x - 1;
            }
        }
    }
    __syncthreads();
    if (!am_last) return;
    // thread 0's acquire saw every block's partial; the barrier above orders
    // this block's reads of them after it
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partials + b);
    t = group_sum(t, 32);
    if (lane == 0) wsum[warp] = t;
    __syncthreads();
    if (warp == 0) {
        double f = lane < nwarps ? wsum[lane] : 0.0;
        f = group_sum(f, 32);
        if (lane == 0) *out = static_cast<OutT>(f);
    }
}

}  // namespace lak
