// vec_dot_noalloc: the inner product of vec_dot for callers that cannot hand
// the library any scratch memory -- for example a host application whose
// memory manager owns every device buffer and gives out only the operands, or
// a foreign-language binding that has no way to allocate device memory.  Its
// scratch (the per-block partial sums and the arrival counter) lives in a
// fixed array compiled into the library, so this call allocates nothing and
// takes no workspace argument.
//
// The array below is a device-side object.  On the host its name is only a
// stand-in for the symbol, not a device address: the device address is looked
// up once per device with cudaGetSymbolAddress and cached.  The first call on
// a device does that look-up (which can also load this library's GPU code onto
// the device), so make the first call on each device before any stream
// capture begins.  Every call on a device uses the same array: calls that
// overlap on the GPU (for example on two streams) race and give wrong results,
// and a call starts by clearing the arrival counter that must begin at zero.
#include <mutex>

#include "lak_internal.cuh"

namespace {

// Counter area (as in any workspace) followed by one FP64 partial per block.
constexpr size_t kScratchBytes =
    (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)LAK_DOT_NOALLOC_MAX_BLOCKS;

static __device__ __align__(256) unsigned char g_dot_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];

// Device address of g_dot_scratch on the current device (looked up once).
lak_status scratch_on_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return lak::fail(LAK_ECUDA, "vec_dot_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return lak::fail(LAK_ECUDA, "vec_dot_noalloc: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dot_scratch);
        if (e != cudaSuccess || !p)
            return lak::fail(LAK_ECUDA, "vec_dot_noalloc: cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LAK_OK;
}

}  // namespace

extern "C" LAK_API lak_status vec_dot_noalloc(void *out, const void *x, const void *y, int64_t n,
                                             lak_dtype dtype, const lak_cfg *cfg, void *stream) {
    using lak::fail;
    if (dtype != LAK_F32 && dtype != LAK_F64 && dtype != LAK_BF16 && dtype != LAK_F16)
        return fail(LAK_EDTYPE, "vec_dot_noalloc: unknown dtype %d", (int)dtype);
    if (n < 0) return fail(LAK_EINVAL, "vec_dot_noalloc: n=%lld < 0", (long long)n);
    if (!out) return fail(LAK_EINVAL, "vec_dot_noalloc: NULL out");
    const int out_bytes = dtype == LAK_F64 ? 8 : 4;
    if ((uintptr_t)out % out_bytes) return fail(LAK_EINVAL, "vec_dot_noalloc: out misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, out_bytes, s);
        if (e != cudaSuccess)
            return fail(LAK_ECUDA, "vec_dot_noalloc: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    const int es = lak::esize(dtype);
    if (!x || !y) return fail(LAK_EINVAL, "vec_dot_noalloc: NULL pointer");
    if ((uintptr_t)x % es || (uintptr_t)y % es)
        return fail(LAK_EINVAL, "vec_dot_noalloc: pointers not aligned to the element size");

    // exactly the launch vec_dot makes for these operands, so both sum in the
    // same block order and give the same bits
    lak::Launch L{};
    int64_t head = 0;
    lak_status st = lak::plan_dot("vec_dot_noalloc", dtype, n, cfg, x, y, &L, &head);
    if (st != LAK_OK) return st;
    if (L.grid > LAK_DOT_NOALLOC_MAX_BLOCKS)
        return fail(LAK_EINVAL,
                    "vec_dot_noalloc: %d blocks exceed the built-in scratch, which holds %d "
                    "block partials; pass a cfg with grid <= %d or use vec_dot with a workspace",
                    L.grid, LAK_DOT_NOALLOC_MAX_BLOCKS, LAK_DOT_NOALLOC_MAX_BLOCKS);

    void *scratch = nullptr;
    st = scratch_on_current_device(&scratch);
    if (st != LAK_OK) return st;
    // the arrival counter must start at zero; an interrupted earlier call could
    // have left it otherwise
    const cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess)
        return fail(LAK_ECUDA, "vec_dot_noalloc: clearing the counter: %s", cudaGetErrorString(e));
    return lak::launch_dot(dtype, out, x, y, n, scratch, L, head, s);
}
