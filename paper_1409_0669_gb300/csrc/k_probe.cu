// Throughput probe: the device's FP64 FMA rate, measured.  On GB300 the FP64
// GEMV and CSR products are bound by the FP64 pipe rather than by HBM, so this
// rate -- not a unit count from a data sheet -- is the roof they are held
// against.  Every thread runs kChains independent FMA chains (enough
// independent work per warp to cover the pipe's latency), then the chains are
// summed and reduced across the warp so that no chain can be discarded as dead
// code; lane 0 of each warp writes one double.
#include "lak_internal.cuh"

namespace lak {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(1024)
fma_f64_probe_kernel(double *out, int64_t iters, double b, double c) {
    LAK_PDL_ENTRY();
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 0.125 * k + 1e-3 * (threadIdx.x & 31);
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0)
        out[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32] = s;
}

}  // namespace
}  // namespace lak

using namespace lak;

extern "C" LAK_API lak_status lak_probe_fma_f64(double *out, int64_t iters, int32_t grid,
                                               int32_t block, void *stream) {
    if (!out || (uintptr_t)out % 8) return fail(LAK_EINVAL, "lak_probe_fma_f64: bad out");
    if (iters < 1) return fail(LAK_EINVAL, "lak_probe_fma_f64: iters=%lld < 1", (long long)iters);
    if (grid < 1 || block < 32 || block > 1024 || block % 32)
        return fail(LAK_EINVAL, "lak_probe_fma_f64: grid %d, block %d (block: 32..1024, multiple "
                    "of 32)", grid, block);
    // b < 1 and c > 0: every chain converges towards c / (1 - b) = 1 and stays
    // a normal number, so no operand is ever subnormal
    launch_k(fma_f64_probe_kernel, dim3((unsigned)grid), dim3((unsigned)block), 0,
             (cudaStream_t)stream, out, iters, 0.9999999, 1e-7);
    return check_launch("lak_probe_fma_f64");
}

extern "C" LAK_API int64_t lak_probe_fma_f64_flops(int64_t iters, int32_t grid, int32_t block) {
    return 2 * (int64_t)kChains * iters * (int64_t)grid * (int64_t)block;
}
