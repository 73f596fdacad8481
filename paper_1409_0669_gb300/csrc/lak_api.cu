// The C ABI (include/lak.h): argument checks, launch-configuration resolution
// (defaults, automatic grid / vector width / group size), workspace sizing and
// dispatch to the kernel launchers.  Host code only.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "lak_internal.cuh"

namespace lak {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------

static thread_local char g_msg[512] = "";

lak_status fail(lak_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    return st;
}

lak_status check_launch(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(LAK_ECUDA, "%s: launch failed: %s", what, cudaGetErrorString(e));
    return LAK_OK;
}

// ---------------------------------------------------------------------------
// device facts
// ---------------------------------------------------------------------------

namespace {
constexpr int kMaxDevices = 64;
DeviceInfo g_dev[kMaxDevices];
bool g_dev_ok[kMaxDevices];
std::mutex g_dev_mu;
}  // namespace

bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("LAK_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

const DeviceInfo *device_info() {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) {
        fail(LAK_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
        return nullptr;
    }
    if (d < 0 || d >= kMaxDevices) {
        fail(LAK_ECUDA, "device ordinal %d out of range", d);
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_dev_ok[d]) {
        DeviceInfo di{};
        di.device = d;
        e = cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, d);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&di.max_threads_per_sm,
                                       cudaDevAttrMaxThreadsPerMultiProcessor, d);
        if (e != cudaSuccess) {
            fail(LAK_ECUDA, "device attributes: %s", cudaGetErrorString(e));
            return nullptr;
        }
        g_dev[d] = di;
        g_dev_ok[d] = true;
    }
    return &g_dev[d];
}

// ---------------------------------------------------------------------------
// configuration
// ---------------------------------------------------------------------------

namespace {

// Size buckets: a call's algorithmic bytes (operands read + results written)
// select one of LAK_SIZE_BUCKETS default configurations.  Below ~8 MB a call
// is launch-latency bound, up to ~64 MB (the paper's own problem sizes on a
// 7 TB/s part) the DRAM latency and the ramp of the first wave still show, and
// from ~512 MB on the launch streams at the bandwidth ceiling.
constexpr int64_t kBucketBound[LAK_SIZE_BUCKETS - 1] = {8LL << 20, 64LL << 20, 512LL << 20};

int64_t op_bytes(lak_op op, lak_dtype dt, int64_t m, int64_t n, int64_t nnz) {
    const int64_t es = esize(dt);
    switch (op) {
    case LAK_OP_COPY:
    case LAK_OP_DOT: return 2 * n * es;
    case LAK_OP_AXPY: return 3 * n * es;
    case LAK_OP_GEMV_ROW:
    case LAK_OP_GEMV_COL: return (m * n + m + n) * es;
    case LAK_OP_SPMV: return nnz * (es + 4) + (m + 1) * 4 + (m + n) * es;
    default: return 0;
    }
}

int bucket_of(int64_t bytes) {
    int b = 0;
    while (b < LAK_SIZE_BUCKETS - 1 && bytes >= kBucketBound[b]) ++b;
    return b;
}

// Built-in defaults per op, storage type and size bucket, measured on GB300
// with the autotuner (every combination of block 64..512, grid 1..32 blocks
// per SM or automatic, vec 1..16 and both increments, at the sweep sizes that
// fall in each bucket; the entry kept has the best worst-case ratio to each
// size's own optimum).  Like the paper's GPU guideline (Sec. 4) the entries
// for large calls favour many work-groups and the global increment; unlike
// it, wide per-thread accesses pay off there (32-64 bytes per thread per
// step), while calls of a few MB prefer narrow accesses and fewer blocks.
//   block        threads per block
//   grid_per_sm  vector ops: cap of the automatic grid, in blocks per SM;
//                dense_gemv / csr_spmv: the grid itself in blocks per SM
//                (0 = the op's automatic grid)
//   vec          elements per access of the row's storage type (csr_spmv:
//                loads per lane)
//   inc          LAK_INC_GLOBAL / LAK_INC_LOCAL
struct DefaultCfg {
    int block, grid_per_sm, vec, inc;
};

constexpr int G_ = LAK_INC_GLOBAL, L_ = LAK_INC_LOCAL;
// [op][0 = FP32, 1 = FP64, 2 = 16-bit storage (BF16 / FP16)][bucket].  Each
// 16-bit entry is the better of two candidates timed side by side on BF16 at the
// bucket's sweep sizes (best worst-case ratio): the FP32 entry at the same bytes
// per access, and the autotuner's own BF16 choice.  Copy, the CSR kernel and
// the smallest column-major GEMV bucket keep the FP32 entries; the update, the
// inner product and the GEMVs gain up to 1.2-1.4x at some sizes from the
// BF16-tuned ones.
constexpr DefaultCfg kDefaults[LAK_OP_COUNT][3][LAK_SIZE_BUCKETS] = {
    // copy
    {{{128, 32, 8, G_}, {128, 8, 16, L_}, {256, 32, 8, G_}, {512, 32, 16, G_}},
     {{512, 4, 4, G_}, {64, 32, 8, G_}, {256, 32, 4, G_}, {512, 32, 8, G_}},
     {{128, 32, 16, G_}, {128, 8, 16, L_}, {256, 32, 16, G_}, {512, 32, 16, G_}}},
    // axpy (and axpby, the fused update + norm)
    {{{256, 32, 8, G_}, {128, 32, 4, G_}, {128, 32, 8, G_}, {512, 32, 16, G_}},
     {{256, 16, 2, G_}, {256, 8, 2, G_}, {128, 32, 4, G_}, {512, 32, 8, G_}},
     {{256, 4, 4, G_}, {256, 0, 8, G_}, {128, 32, 16, G_}, {512, 32, 16, G_}}},
    // dot
    {{{256, 8, 8, G_}, {512, 4, 4, G_}, {512, 1, 16, G_}, {512, 2, 8, G_}},
     {{256, 1, 2, G_}, {512, 1, 4, G_}, {512, 2, 1, G_}, {256, 4, 4, G_}},
     {{256, 0, 16, G_}, {256, 4, 8, G_}, {512, 2, 8, G_}, {512, 2, 16, G_}}},
    // row-major GEMV
    {{{256, 0, 2, G_}, {128, 8, 8, G_}, {32, 32, 8, G_}, {64, 0, 8, G_}},
     {{128, 8, 4, G_}, {32, 16, 8, G_}, {32, 0, 2, G_}, {32, 0, 8, G_}},
     {{128, 0, 2, G_}, {128, 8, 8, G_}, {32, 32, 8, G_}, {64, 0, 8, G_}}},
    // column-major GEMV
    {{{512, 1, 4, L_}, {512, 0, 8, G_}, {512, 2, 8, L_}, {128, 0, 4, G_}},
     {{512, 4, 2, G_}, {512, 2, 4, G_}, {128, 8, 2, L_}, {512, 16, 2, L_}},
     {{512, 1, 8, L_}, {512, 4, 8, G_}, {512, 4, 8, L_}, {256, 8, 8, L_}}},
    // CSR SpMV, group-per-row kernel (short and long rows)
    {{{512, 2, 4, G_}, {128, 16, 4, G_}, {128, 16, 4, G_}, {128, 16, 4, G_}},
     {{256, 0, 4, G_}, {64, 16, 8, G_}, {64, 16, 8, G_}, {64, 16, 8, G_}},
     {{512, 2, 4, G_}, {128, 16, 4, G_}, {128, 16, 4, G_}, {128, 16, 4, G_}}},
};

// CSR SpMV, warp-segmented kernel (mean row length 13..64): tuned on the
// power-law matrix (2M rows), where the group-per-row entries above lose 6 %
// (FP32) and 4 % (FP64).  FP64 takes 4 entries per lane: at 48-50 registers a
// thread that leaves more warps resident than 8 entries (60 registers), and
// the gathers, not the FP64 pipe, bound this kernel now (186 vs 195 us).  The
// large buckets follow the re-ranking tuner's sweep on the current kernel
// (FP32 64 threads: 139.3 against 140.5 us at 128; 16-bit 64 threads and 8
// entries per lane: 129.4 against 132.9 us).  [0 = FP32, 1 = FP64, 2 = 16-bit]
constexpr DefaultCfg kSpmvSegDefaults[3][LAK_SIZE_BUCKETS] = {
    {{128, 0, 4, G_}, {128, 0, 4, G_}, {64, 0, 4, G_}, {64, 0, 4, G_}},
    {{64, 0, 4, G_}, {64, 0, 4, G_}, {64, 0, 4, G_}, {64, 0, 4, G_}},
    {{128, 0, 4, G_}, {128, 0, 4, G_}, {64, 0, 8, G_}, {64, 0, 8, G_}},
};

bool is_vector_op(lak_op op) { return op == LAK_OP_COPY || op == LAK_OP_AXPY || op == LAK_OP_DOT; }

int storage_row(lak_dtype dt) { return dt == LAK_F64 ? 1 : (dt == LAK_BF16 || dt == LAK_F16) ? 2 : 0; }

DefaultCfg default_row(lak_op op, lak_dtype dt, int bucket) { return kDefaults[op][storage_row(dt)][bucket]; }

// Fallback launch shapes of the batched persistent kernels (lak_batch_run), used
// only where no autotuned entry is installed (lak_set_batch_default_cfg; the
// package ships the entries it measured on GB300).
struct BatchCfg {
    int block, bytes, inc;
};

BatchCfg batch_row(lak_op op, lak_dtype dt) {
    const bool f64 = dt == LAK_F64;
    switch (op) {
    case LAK_OP_AXPY: return {512, 64, LAK_INC_GLOBAL};
    case LAK_OP_DOT: return {512, f64 ? 32 : 16, LAK_INC_GLOBAL};
    case LAK_OP_GEMV_ROW: return {128, 16, LAK_INC_GLOBAL};  // row groups take 4 rows each
    default: return {64, 16, LAK_INC_GLOBAL};      // CSR: 4 loads per lane (see batch_config)
    }
}

int vec_for_bytes(int bytes, int es) {
    int v = bytes / es;
    if (v < 1) v = 1;
    if (v > 16) v = 16;
    return v;
}

// The built-in default as a cfg: dense_gemv / csr_spmv entries with a grid
// carry it (blocks per SM x SMs); the vector ops keep grid 0 (automatic,
// capped by default_grid_per_sm).
lak_cfg builtin_default(lak_op op, lak_dtype dt, int bucket) {
    const DefaultCfg d = default_row(op, dt, bucket);
    lak_cfg c{d.block, 0, d.vec, d.inc};
    if (!is_vector_op(op) && d.grid_per_sm > 0) {
        const DeviceInfo *di = device_info();
        if (di) c.grid = d.grid_per_sm * di->sms;
    }
    return c;
}

// Automatic grid cap (blocks per SM) for the grid-stride vector kernels.
int default_grid_per_sm(lak_op op, lak_dtype dt, int bucket) {
    const int g = default_row(op, dt, bucket).grid_per_sm;
    return g > 0 ? g : 0;
}

lak_cfg g_override[LAK_OP_COUNT][4][LAK_SIZE_BUCKETS];
bool g_has_override[LAK_OP_COUNT][4][LAK_SIZE_BUCKETS];
std::mutex g_cfg_mu;

// Batched defaults installed with lak_set_batch_default_cfg (axpy, dot,
// row-major GEMV, CSR), per storage type.
lak_cfg g_batch_override[4][4];
bool g_has_batch_override[4][4];

int batch_op_index(lak_op op) {
    switch (op) {
    case LAK_OP_AXPY: return 0;
    case LAK_OP_DOT: return 1;
    case LAK_OP_GEMV_ROW: return 2;
    case LAK_OP_SPMV: return 3;
    default: return -1;
    }
}

bool valid_dtype(lak_dtype dt) { return dt == LAK_F32 || dt == LAK_F64 || dt == LAK_BF16 || dt == LAK_F16; }
bool valid_op(lak_op op) { return op >= 0 && op < LAK_OP_COUNT; }
bool pow2_vec(int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16; }

lak_status check_cfg(const lak_cfg *c, const char *who) {
    if (!c || c->block == 0) return LAK_OK;
    if (c->block < 32 || c->block > 512 || c->block % 32)
        return fail(LAK_EINVAL, "%s: cfg.block=%d must be a multiple of 32 in [32, 512]", who, c->block);
    if (c->grid < 0) return fail(LAK_EINVAL, "%s: cfg.grid=%d must be >= 0", who, c->grid);
    if (c->vec != 0 && !pow2_vec(c->vec))
        return fail(LAK_EINVAL, "%s: cfg.vec=%d must be 0, 1, 2, 4, 8 or 16", who, c->vec);
    if (c->increment != LAK_INC_GLOBAL && c->increment != LAK_INC_LOCAL)
        return fail(LAK_EINVAL, "%s: cfg.increment=%d must be 0 (global) or 1 (local)", who,
                    c->increment);
    return LAK_OK;
}

// Explicit cfg, else the override table, else the built-in default; zero
// grid / vec fields stay zero here (filled per op below).
lak_cfg base_cfg(lak_op op, lak_dtype dt, int bucket, const lak_cfg *cfg) {
    if (cfg && cfg->block != 0) return *cfg;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    if (g_has_override[op][dt][bucket]) return g_override[op][dt][bucket];
    return builtin_default(op, dt, bucket);
}

int pow2_floor(int64_t v) {
    int p = 1;
    while ((int64_t)p * 2 <= v && p < (1 << 30)) p *= 2;
    return p;
}

// largest power of two dividing the block size (groups must tile the block)
int block_pow2(int block) { return block & -block; }

int waves_grid(const DeviceInfo *di, int block) {
    int per_sm = di->max_threads_per_sm / block;
    if (per_sm < 1) per_sm = 1;
    return di->sms * per_sm;
}

struct VecPlan {
    Launch L;
    int64_t head;
};

lak_status plan_vector(lak_op op, lak_dtype dt, int64_t n, const lak_cfg *cfg,
                       const void *const *ptrs, int nptrs, VecPlan *out) {
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int bucket = bucket_of(op_bytes(op, dt, n, n, 0));
    lak_cfg c = base_cfg(op, dt, bucket, cfg);
    const int es = esize(dt);
    int want = c.vec ? c.vec : builtin_default(op, dt, bucket).vec;
    int64_t head = 0;
    int vec = ptrs ? pick_vec(want, es, ptrs, nptrs, n, &head) : want;
    const int64_t nchunks = vec > 0 ? (n - head) / vec : n;
    int64_t grid = c.grid;
    if (grid == 0) {
        const int64_t need = ceil_div(nchunks > 0 ? nchunks : 1, c.block);
        const int per_sm = default_grid_per_sm(op, dt, bucket);
        const int64_t cap = per_sm > 0 ? (int64_t)per_sm * di->sms : waves_grid(di, c.block);
        grid = need < cap ? need : cap;
        // an inner product one block covers in two passes skips the grid-wide
        // combine (a ticket and a second block pass, ~2 us; a pass is less)
        if (op == LAK_OP_DOT && need <= 2) grid = 1;
    }
    if (grid < 1) grid = 1;
    if (grid > 0x7fffffff) grid = 0x7fffffff;
    out->L = Launch{c.block, (int)grid, vec, c.increment};
    out->head = head;
    return LAK_OK;
}

struct RowPlan {
    Launch L;
    int group;
};

// Row-major GEMV: group size G grows with the row length (each lane should
// see at least 4 V-groups), limited by the block.
lak_status plan_gemv_row(lak_dtype dt, int64_t m, int64_t n, int64_t lda, const lak_cfg *cfg,
                         const void *A, const void *x, RowPlan *out) {
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int bucket = bucket_of(op_bytes(LAK_OP_GEMV_ROW, dt, m, n, 0));
    lak_cfg c = base_cfg(LAK_OP_GEMV_ROW, dt, bucket, cfg);
    const int es = esize(dt);
    const int vec = c.vec ? c.vec : builtin_default(LAK_OP_GEMV_ROW, dt, bucket).vec;
    (void)A;   // rows are brought to the access width in the kernel (per-row head)
    (void)x;
    (void)lda;
    const int64_t nch = n / vec;
    int G = pow2_floor(nch / 4 > 0 ? nch / 4 : 1);
    // at least one 128-byte line of a row per group access: DRAM fetches whole
    // lines, so narrower groups would waste part of every fetch
    while (G < 32 && (int64_t)G * vec * es < 128) G *= 2;
    const int bp = block_pow2(c.block);
    if (G > bp) G = bp;
    const int R = c.block / G;
    int64_t grid = c.grid;
    if (grid == 0) grid = ceil_div(m > 0 ? m : 1, R);
    if (grid > 0x7fffffff) grid = 0x7fffffff;
    out->L = Launch{c.block, (int)grid, vec, c.increment};
    out->group = G;
    return LAK_OK;
}

struct ColPlan {
    Launch L;
    int splits;
    int64_t tiles;
    size_t ws_bytes;
};

lak_status plan_gemv_col(lak_dtype dt, int64_t m, int64_t n, int64_t lda, const lak_cfg *cfg,
                         const void *A, ColPlan *out) {
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int bucket = bucket_of(op_bytes(LAK_OP_GEMV_COL, dt, m, n, 0));
    lak_cfg c = base_cfg(LAK_OP_GEMV_COL, dt, bucket, cfg);
    const int es = esize(dt);
    int vec = c.vec ? c.vec : builtin_default(LAK_OP_GEMV_COL, dt, bucket).vec;
    while (vec > 1) {
        const int w = access_bytes(vec, es);
        if ((!A || (uintptr_t)A % w == 0) && ((lda * es) % w == 0)) break;
        vec >>= 1;
    }
    const int64_t tiles = ceil_div(m > 0 ? m : 1, 32LL * vec);
    const int nwarps = c.block / 32;
    int64_t target = c.grid ? c.grid : 2LL * waves_grid(di, c.block);
    int64_t splits = ceil_div(target, tiles);
    const int64_t max_splits = n / (4LL * nwarps);      // >= 4 columns per warp per split
    if (splits > max_splits) splits = max_splits;
    if (splits > 65535) splits = 65535;
    // one arrival counter per row tile, all inside the workspace counter area
    if (tiles > LAK_WS_COUNTER_BYTES / 4) splits = 1;
    if (splits < 1) splits = 1;
    const int acc_bytes = dt == LAK_F64 ? 8 : 4;
    size_t ws = 0;
    if (splits > 1) ws = (size_t)LAK_WS_COUNTER_BYTES + (size_t)splits * (size_t)m * acc_bytes;
    out->L = Launch{c.block, (int)(tiles * splits > 0x7fffffff ? 0x7fffffff : tiles * splits), vec,
                    c.increment};
    out->splits = (int)splits;
    out->tiles = tiles;
    out->ws_bytes = ws;
    return LAK_OK;
}

struct SpmvPlan {
    Launch L;
    int group;     // lanes per row (long-row variant); 0 = warp-stream variant
};

// Mean row lengths between which the warp-segmented variant is used; below
// the range one lane (or two) per row, above it a group of lanes per row.
int64_t env_int(const char *name, int64_t dflt) {
    const char *e = getenv(name);
    if (e && *e) {
        char *end = nullptr;
        const long long x = strtoll(e, &end, 10);
        if (end && *end == 0 && x >= 0) return (int64_t)x;
    }
    return dflt;
}

int64_t spmv_seg_min_mean() {
    static const int64_t v = env_int("LAK_SPMV_SEG_MIN_MEAN", 13);
    return v;
}

int64_t spmv_seg_max_mean() {
    static const int64_t v = env_int("LAK_SPMV_SEG_MAX_MEAN", 64);
    return v;
}

// The built-in default for the warp-segmented SpMV kernel (an override set for
// LAK_OP_SPMV applies to both SpMV kernels).
lak_cfg seg_default(lak_dtype dt, int bucket) {
    const DefaultCfg d = kSpmvSegDefaults[storage_row(dt)][bucket];
    lak_cfg c{d.block, 0, d.vec, d.inc};
    if (d.grid_per_sm > 0) {
        const DeviceInfo *di = device_info();
        if (di) c.grid = d.grid_per_sm * di->sms;
    }
    return c;
}

lak_status plan_spmv(lak_dtype dt, int64_t m, int64_t n, int64_t nnz, const lak_cfg *cfg,
                     SpmvPlan *out) {
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int bucket = bucket_of(op_bytes(LAK_OP_SPMV, dt, m, n, nnz));
    const int64_t mean = m > 0 ? ceil_div(nnz, m) : 1;
    const bool seg = mean >= spmv_seg_min_mean() && mean <= spmv_seg_max_mean();
    lak_cfg c = base_cfg(LAK_OP_SPMV, dt, bucket, cfg);
    bool overridden = cfg && cfg->block != 0;
    if (!overridden) {
        std::lock_guard<std::mutex> lk(g_cfg_mu);
        overridden = g_has_override[LAK_OP_SPMV][dt][bucket];
    }
    if (seg && !overridden) c = seg_default(dt, bucket);
    int vec = c.vec ? c.vec : (seg ? seg_default(dt, bucket) : builtin_default(LAK_OP_SPMV, dt, bucket)).vec;
    int G = 0;
    int64_t rows_per_block;
    if (seg) {
        rows_per_block = c.block;                // a warp per 32 rows
    } else {
        // lanes per row: the power of two covering the mean row length in
        // `vec` loads per lane, up to a warp
        G = 1;
        while (G < 32 && (int64_t)G * vec < mean) G *= 2;
        const int bp = block_pow2(c.block);
        if (G > bp) G = bp;
        rows_per_block = c.block / G;
    }
    int64_t grid = c.grid;
    if (grid == 0) grid = ceil_div(m > 0 ? m : 1, rows_per_block);
    if (grid > 0x7fffffff) grid = 0x7fffffff;
    out->L = Launch{c.block, (int)grid, vec, c.increment};
    out->group = G;
    return LAK_OK;
}

}  // namespace

lak_cfg batch_config(lak_op op, lak_dtype dt, const lak_cfg *cfg) {
    const BatchCfg b = batch_row(op, dt);
    lak_cfg c{b.block, 0, 0, b.inc};
    if (cfg && cfg->block != 0) {
        c = *cfg;
    } else {
        std::lock_guard<std::mutex> lk(g_cfg_mu);
        const int bi = batch_op_index(op);
        if (bi >= 0 && g_has_batch_override[bi][dt]) c = g_batch_override[bi][dt];
    }
    if (c.vec == 0) c.vec = op == LAK_OP_SPMV ? 4 : vec_for_bytes(b.bytes, esize(dt));
    return c;
}

lak_status plan_dot(const char *who, lak_dtype dt, int64_t n, const lak_cfg *cfg, const void *x,
                    const void *y, Launch *L, int64_t *head) {
    lak_status st = check_cfg(cfg, who);
    if (st != LAK_OK) return st;
    const void *ptrs[2] = {x, y};
    VecPlan p;
    st = plan_vector(LAK_OP_DOT, dt, n, cfg, ptrs, 2, &p);
    if (st != LAK_OK) return st;
    *L = p.L;
    *head = p.head;
    return LAK_OK;
}

int pick_vec(int want, int es, const void *const *ptrs, int nptrs, int64_t n, int64_t *head) {
    for (int vec = want; vec > 1; vec >>= 1) {
        const int w = access_bytes(vec, es);
        const uintptr_t off = (uintptr_t)ptrs[0] % w;
        bool same = true;
        for (int i = 1; i < nptrs; ++i)
            if ((uintptr_t)ptrs[i] % w != off) same = false;
        if (!same || off % es) continue;
        int64_t h = (int64_t)((w - off) % w) / es;
        if (h > n) h = n;
        *head = h;
        return vec;
    }
    *head = 0;
    return 1;
}

}  // namespace lak

using namespace lak;

// ---------------------------------------------------------------------------
// exported entry points
// ---------------------------------------------------------------------------

namespace {

bool aligned_elem(const void *p, int es) { return (uintptr_t)p % (uintptr_t)es == 0; }

lak_status common_checks(const char *who, lak_dtype dt, const lak_cfg *cfg) {
    if (!valid_dtype(dt)) return fail(LAK_EDTYPE, "%s: unknown dtype %d", who, (int)dt);
    return check_cfg(cfg, who);
}

}  // namespace

extern "C" {

LAK_API const char *lak_last_error(void) { return g_msg; }

LAK_API int32_t lak_abi_version(void) { return 1; }

LAK_API lak_status lak_set_default_cfg_bucket(lak_op op, lak_dtype dtype, int32_t bucket,
                                              const lak_cfg *cfg) {
    const char *who = "lak_set_default_cfg";
    if (!valid_op(op)) return fail(LAK_EINVAL, "%s: unknown op %d", who, (int)op);
    if (!valid_dtype(dtype)) return fail(LAK_EDTYPE, "%s: unknown dtype %d", who, (int)dtype);
    if (bucket < -1 || bucket >= LAK_SIZE_BUCKETS)
        return fail(LAK_EINVAL, "%s: bucket %d not in [-1, %d)", who, (int)bucket, LAK_SIZE_BUCKETS);
    if (cfg && cfg->block == 0)
        return fail(LAK_EINVAL, "%s: cfg.block must be set (or pass NULL)", who);
    lak_status st = check_cfg(cfg, who);
    if (st != LAK_OK) return st;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    for (int b = 0; b < LAK_SIZE_BUCKETS; ++b) {
        if (bucket >= 0 && b != bucket) continue;
        if (cfg) g_override[op][dtype][b] = *cfg;
        g_has_override[op][dtype][b] = cfg != nullptr;
    }
    return LAK_OK;
}

LAK_API lak_status lak_set_default_cfg(lak_op op, lak_dtype dtype, const lak_cfg *cfg) {
    return lak_set_default_cfg_bucket(op, dtype, -1, cfg);
}

LAK_API lak_status lak_set_batch_default_cfg(lak_op op, lak_dtype dtype, const lak_cfg *cfg) {
    const int bi = batch_op_index(op);
    if (bi < 0) return fail(LAK_EINVAL, "lak_set_batch_default_cfg: op %d has no batched form", (int)op);
    if (!valid_dtype(dtype))
        return fail(LAK_EDTYPE, "lak_set_batch_default_cfg: unknown dtype %d", (int)dtype);
    if (cfg && cfg->block != 0) {
        const int max_block = op == LAK_OP_GEMV_ROW ? kGemvBatchMaxBlock : 512;
        if (cfg->block < 32 || cfg->block > max_block || cfg->block % 32 || cfg->grid < 0 ||
            (cfg->vec != 0 && !pow2_vec(cfg->vec)) ||
            (cfg->increment != LAK_INC_GLOBAL && cfg->increment != LAK_INC_LOCAL))
            return fail(LAK_EINVAL, "lak_set_batch_default_cfg: invalid cfg (%d, %d, %d, %d)",
                        cfg->block, cfg->grid, cfg->vec, cfg->increment);
    }
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    g_has_batch_override[bi][dtype] = cfg && cfg->block != 0;
    if (g_has_batch_override[bi][dtype]) g_batch_override[bi][dtype] = *cfg;
    return LAK_OK;
}

LAK_API int32_t lak_size_bucket(lak_op op, lak_dtype dtype, int64_t m, int64_t n, int64_t nnz) {
    if (!valid_op(op)) return fail(LAK_EINVAL, "lak_size_bucket: unknown op %d", (int)op);
    if (!valid_dtype(dtype)) return fail(LAK_EDTYPE, "lak_size_bucket: unknown dtype %d", (int)dtype);
    if (m < 0 || n < 0 || nnz < 0) return fail(LAK_EINVAL, "lak_size_bucket: negative size");
    return bucket_of(op_bytes(op, dtype, m, n, nnz));
}

LAK_API lak_status lak_resolve_cfg(lak_op op, lak_dtype dtype, int64_t m, int64_t n, int64_t nnz,
                                   const lak_cfg *cfg, lak_cfg *out) {
    if (!valid_op(op)) return fail(LAK_EINVAL, "lak_resolve_cfg: unknown op %d", (int)op);
    lak_status st = common_checks("lak_resolve_cfg", dtype, cfg);
    if (st != LAK_OK) return st;
    if (!out || m < 0 || n < 0 || nnz < 0)
        return fail(LAK_EINVAL, "lak_resolve_cfg: bad sizes or NULL out");
    Launch L{};
    switch (op) {
    case LAK_OP_COPY:
    case LAK_OP_AXPY:
    case LAK_OP_DOT: {
        VecPlan p;
        st = plan_vector(op, dtype, m, cfg, nullptr, 0, &p);
        L = p.L;
        break;
    }
    case LAK_OP_GEMV_ROW: {
        RowPlan p;
        st = plan_gemv_row(dtype, m, n, n, cfg, nullptr, nullptr, &p);
        L = p.L;
        break;
    }
    case LAK_OP_GEMV_COL: {
        ColPlan p;
        st = plan_gemv_col(dtype, m, n, m, cfg, nullptr, &p);
        L = p.L;
        break;
    }
    case LAK_OP_SPMV: {
        SpmvPlan p;
        st = plan_spmv(dtype, m, n, nnz, cfg, &p);
        L = p.L;
        break;
    }
    default: return fail(LAK_EINVAL, "lak_resolve_cfg: unknown op");
    }
    if (st != LAK_OK) return st;
    *out = lak_cfg{L.block, L.grid, L.vec, L.inc};
    return LAK_OK;
}

LAK_API lak_status vec_copy(void *x, const void *y, int64_t n, lak_dtype dtype, const lak_cfg *cfg,
                            void *stream) {
    lak_status st = common_checks("vec_copy", dtype, cfg);
    if (st != LAK_OK) return st;
    if (n < 0) return fail(LAK_EINVAL, "vec_copy: n=%lld < 0", (long long)n);
    if (n == 0) return LAK_OK;
    const int es = esize(dtype);
    if (!x || !y) return fail(LAK_EINVAL, "vec_copy: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es))
        return fail(LAK_EINVAL, "vec_copy: pointers not aligned to the element size");
    const void *ptrs[2] = {x, y};
    VecPlan p;
    st = plan_vector(LAK_OP_COPY, dtype, n, cfg, ptrs, 2, &p);
    if (st != LAK_OK) return st;
    return launch_copy(x, y, n, es, p.L, p.head, (cudaStream_t)stream);
}

LAK_API lak_status vec_axpy(void *x, const void *y, const void *z, double alpha, int64_t n,
                            lak_dtype dtype, const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_axpy", dtype, cfg);
    if (st != LAK_OK) return st;
    if (n < 0) return fail(LAK_EINVAL, "vec_axpy: n=%lld < 0", (long long)n);
    if (n == 0) return LAK_OK;
    const int es = esize(dtype);
    if (!x || !y || !z) return fail(LAK_EINVAL, "vec_axpy: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es) || !aligned_elem(z, es))
        return fail(LAK_EINVAL, "vec_axpy: pointers not aligned to the element size");
    const void *ptrs[3] = {x, y, z};
    VecPlan p;
    st = plan_vector(LAK_OP_AXPY, dtype, n, cfg, ptrs, 3, &p);
    if (st != LAK_OK) return st;
    return launch_axpy(dtype, x, y, z, alpha, n, p.L, p.head, (cudaStream_t)stream);
}

LAK_API size_t vec_dot_workspace(int64_t n, lak_dtype dtype, const lak_cfg *cfg) {
    if (!valid_dtype(dtype) || n < 0 || check_cfg(cfg, "vec_dot_workspace") != LAK_OK) return 0;
    VecPlan p;
    if (plan_vector(LAK_OP_DOT, dtype, n, cfg, nullptr, 0, &p) != LAK_OK) return 0;
    // The grid never grows when alignment forces a narrower vec (fewer chunks
    // per thread would need more blocks only without the cap): size for the
    // widest grid any alignment of these n elements can produce.
    VecPlan p1;
    lak_cfg c = base_cfg(LAK_OP_DOT, dtype, bucket_of(op_bytes(LAK_OP_DOT, dtype, n, n, 0)), cfg);
    c.vec = 1;
    if (plan_vector(LAK_OP_DOT, dtype, n, &c, nullptr, 0, &p1) != LAK_OK) return 0;
    const int grid = p1.L.grid > p.L.grid ? p1.L.grid : p.L.grid;
    return (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)grid;
}

LAK_API lak_status vec_dot(void *out, const void *x, const void *y, int64_t n, lak_dtype dtype,
                           void *workspace, size_t ws_bytes, const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_dot", dtype, cfg);
    if (st != LAK_OK) return st;
    if (n < 0) return fail(LAK_EINVAL, "vec_dot: n=%lld < 0", (long long)n);
    if (!out) return fail(LAK_EINVAL, "vec_dot: NULL out");
    const int out_bytes = dtype == LAK_F64 ? 8 : 4;
    if ((uintptr_t)out % out_bytes) return fail(LAK_EINVAL, "vec_dot: out misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, out_bytes, s);
        if (e != cudaSuccess) return fail(LAK_ECUDA, "vec_dot: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    const int es = esize(dtype);
    if (!x || !y) return fail(LAK_EINVAL, "vec_dot: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es))
        return fail(LAK_EINVAL, "vec_dot: pointers not aligned to the element size");
    const void *ptrs[2] = {x, y};
    VecPlan p;
    st = plan_vector(LAK_OP_DOT, dtype, n, cfg, ptrs, 2, &p);
    if (st != LAK_OK) return st;
    const size_t need = (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)p.L.grid;
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "vec_dot: workspace of %zu bytes needed, %zu given", need,
                    workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "vec_dot: workspace not 256-byte aligned");
    return launch_dot(dtype, out, x, y, n, workspace, p.L, p.head, s);
}

LAK_API size_t vec_dot_sparse_workspace(int64_t nnz, lak_dtype dtype, const lak_cfg *cfg) {
    return vec_dot_workspace(nnz, dtype, cfg);
}

LAK_API lak_status vec_dot_sparse(void *out, const void *vals, const int32_t *idx, const void *y,
                                  int64_t nnz, int64_t n, lak_dtype dtype, void *workspace,
                                  size_t ws_bytes, const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_dot_sparse", dtype, cfg);
    if (st != LAK_OK) return st;
    if (nnz < 0 || n < 0) return fail(LAK_EINVAL, "vec_dot_sparse: negative size");
    if (!out) return fail(LAK_EINVAL, "vec_dot_sparse: NULL out");
    const int out_bytes = dtype == LAK_F64 ? 8 : 4;
    if ((uintptr_t)out % out_bytes) return fail(LAK_EINVAL, "vec_dot_sparse: out misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (nnz == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, out_bytes, s);
        if (e != cudaSuccess)
            return fail(LAK_ECUDA, "vec_dot_sparse: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    const int es = esize(dtype);
    if (!vals || !idx || !y || n == 0) return fail(LAK_EINVAL, "vec_dot_sparse: NULL pointer or n = 0");
    if (!aligned_elem(vals, es) || !aligned_elem(y, es) || (uintptr_t)idx % 4)
        return fail(LAK_EINVAL, "vec_dot_sparse: pointers not aligned to the element size");
    // the dot's configuration; the widest vec (<= 8) for which one prologue
    // aligns both the values and the indices
    VecPlan p;
    st = plan_vector(LAK_OP_DOT, dtype, nnz, cfg, nullptr, 0, &p);
    if (st != LAK_OK) return st;
    int vec = p.L.vec > 8 ? 8 : p.L.vec;
    int64_t head = 0;
    for (; vec > 1; vec >>= 1) {
        const int wv = access_bytes(vec, es), wi = access_bytes(vec, 4);
        const int64_t h = (int64_t)((wv - (uintptr_t)vals % wv) % wv) / es;
        if (((uintptr_t)idx + 4 * h) % wi == 0) {
            head = h < nnz ? h : nnz;
            break;
        }
    }
    if (vec == 1) head = 0;
    if (vec != p.L.vec) {
        lak_cfg c{p.L.block, cfg && cfg->block ? cfg->grid : 0, vec, p.L.inc};
        st = plan_vector(LAK_OP_DOT, dtype, nnz, &c, nullptr, 0, &p);
        if (st != LAK_OK) return st;
    }
    const size_t need = (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)p.L.grid;
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "vec_dot_sparse: workspace of %zu bytes needed, %zu given", need,
                    workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "vec_dot_sparse: workspace not 256-byte aligned");
    return launch_dot_sparse(dtype, out, vals, idx, y, nnz, workspace, p.L, head, s);
}

LAK_API lak_status vec_dot_compensated(double *out, const void *x, const void *y, int64_t n,
                                       lak_dtype dtype, void *workspace, size_t ws_bytes,
                                       const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_dot_compensated", dtype, cfg);
    if (st != LAK_OK) return st;
    if (dtype == LAK_F64)
        return fail(LAK_EDTYPE, "vec_dot_compensated: FP32, BF16 or FP16 storage only");
    if (n < 0) return fail(LAK_EINVAL, "vec_dot_compensated: n=%lld < 0", (long long)n);
    if (!out || (uintptr_t)out % 8) return fail(LAK_EINVAL, "vec_dot_compensated: bad out");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, 8, s);
        if (e != cudaSuccess)
            return fail(LAK_ECUDA, "vec_dot_compensated: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    const int es = esize(dtype);
    if (!x || !y) return fail(LAK_EINVAL, "vec_dot_compensated: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es))
        return fail(LAK_EINVAL, "vec_dot_compensated: pointers not aligned to the element size");
    const void *ptrs[2] = {x, y};
    VecPlan p;
    st = plan_vector(LAK_OP_DOT, dtype, n, cfg, ptrs, 2, &p);
    if (st != LAK_OK) return st;
    const size_t need = (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)p.L.grid;
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "vec_dot_compensated: workspace of %zu bytes needed, %zu given",
                    need, workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "vec_dot_compensated: workspace not 256-byte aligned");
    return launch_dot_comp(dtype, out, x, y, n, workspace, p.L, p.head, s);
}

LAK_API size_t dense_gemv_workspace(int64_t m, int64_t n, lak_layout layout, lak_dtype dtype,
                                    const lak_cfg *cfg) {
    if (!valid_dtype(dtype) || m < 0 || n < 0 || check_cfg(cfg, "dense_gemv_workspace") != LAK_OK)
        return 0;
    if (layout != LAK_COL_MAJOR) return 0;
    // the widest vec the call could pick gives the fewest tiles; narrower vecs
    // (forced by alignment) only add tiles, so size for vec = 1 as well
    size_t best = 0;
    const int bucket = bucket_of(op_bytes(LAK_OP_GEMV_COL, dtype, m, n, 0));
    lak_cfg c = base_cfg(LAK_OP_GEMV_COL, dtype, bucket, cfg);
    const int want = c.vec ? c.vec : builtin_default(LAK_OP_GEMV_COL, dtype, bucket).vec;
    for (int v = want; v >= 1; v >>= 1) {
        lak_cfg cv = c;
        cv.vec = v;
        ColPlan p;
        if (plan_gemv_col(dtype, m, n, m, &cv, nullptr, &p) != LAK_OK) return 0;
        if (p.ws_bytes > best) best = p.ws_bytes;
    }
    return best;
}

}  // extern "C"

namespace {

lak_status gemv_impl(const char *who, void *y, const void *A, const void *x, int64_t m, int64_t n,
                     int64_t lda, lak_layout layout, lak_dtype dtype, void *workspace,
                     size_t ws_bytes, const lak_cfg *cfg, double alpha, double beta,
                     void *stream) {
    lak_status st = common_checks(who, dtype, cfg);
    if (st != LAK_OK) return st;
    if (layout != LAK_ROW_MAJOR && layout != LAK_COL_MAJOR)
        return fail(LAK_ELAYOUT, "%s: unknown layout %d", who, (int)layout);
    if (m < 0 || n < 0) return fail(LAK_EINVAL, "%s: negative size", who);
    const int64_t ld_min = layout == LAK_ROW_MAJOR ? (n > 1 ? n : 1) : (m > 1 ? m : 1);
    if (lda < ld_min)
        return fail(LAK_EINVAL, "%s: lda=%lld < %lld", who, (long long)lda, (long long)ld_min);
    if (m == 0) return LAK_OK;
    const int es = esize(dtype);
    if (!y || (n > 0 && (!A || !x))) return fail(LAK_EINVAL, "%s: NULL pointer", who);
    if (!aligned_elem(y, es) || !aligned_elem(A, es) || !aligned_elem(x, es))
        return fail(LAK_EINVAL, "%s: pointers not aligned to the element size", who);
    cudaStream_t s = (cudaStream_t)stream;
    if (layout == LAK_ROW_MAJOR) {
        RowPlan p;
        st = plan_gemv_row(dtype, m, n, lda, cfg, A, x, &p);
        if (st != LAK_OK) return st;
        return launch_gemv_row(dtype, y, A, x, m, n, lda, p.L, p.group, alpha, beta, s);
    }
    ColPlan p;
    st = plan_gemv_col(dtype, m, n, lda, cfg, A, &p);
    if (st != LAK_OK) return st;
    if (p.ws_bytes > 0) {
        if (!workspace || ws_bytes < p.ws_bytes)
            return fail(LAK_EWORKSPACE, "%s: workspace of %zu bytes needed, %zu given", who,
                        p.ws_bytes, workspace ? ws_bytes : (size_t)0);
        if ((uintptr_t)workspace % 256)
            return fail(LAK_EWORKSPACE, "%s: workspace not 256-byte aligned", who);
    }
    return launch_gemv_col(dtype, y, A, x, m, n, lda, p.L, p.splits, workspace, alpha, beta, s);
}

}  // namespace

extern "C" {

LAK_API lak_status dense_gemv(void *y, const void *A, const void *x, int64_t m, int64_t n,
                              int64_t lda, lak_layout layout, lak_dtype dtype, void *workspace,
                              size_t ws_bytes, const lak_cfg *cfg, void *stream) {
    return gemv_impl("dense_gemv", y, A, x, m, n, lda, layout, dtype, workspace, ws_bytes, cfg,
                     1.0, 0.0, stream);
}

LAK_API lak_status dense_gemv_axpby(void *y, double alpha, const void *A, const void *x,
                                    double beta, int64_t m, int64_t n, int64_t lda,
                                    lak_layout layout, lak_dtype dtype, void *workspace,
                                    size_t ws_bytes, const lak_cfg *cfg, void *stream) {
    return gemv_impl("dense_gemv_axpby", y, A, x, m, n, lda, layout, dtype, workspace, ws_bytes,
                     cfg, alpha, beta, stream);
}

LAK_API lak_status dense_gemv_trans(void *y, const void *A, const void *x, int64_t m, int64_t n,
                                    int64_t lda, lak_layout layout, lak_dtype dtype,
                                    void *workspace, size_t ws_bytes, const lak_cfg *cfg,
                                    void *stream) {
    if (layout != LAK_ROW_MAJOR && layout != LAK_COL_MAJOR)
        return fail(LAK_ELAYOUT, "dense_gemv_trans: unknown layout %d", (int)layout);
    // A^T of an m-by-n matrix in one layout is an n-by-m matrix in the other
    const lak_layout other = layout == LAK_ROW_MAJOR ? LAK_COL_MAJOR : LAK_ROW_MAJOR;
    return gemv_impl("dense_gemv_trans", y, A, x, n, m, lda, other, dtype, workspace, ws_bytes,
                     cfg, 1.0, 0.0, stream);
}

LAK_API size_t vec_axpy_norm2_workspace(int64_t n, lak_dtype dtype, const lak_cfg *cfg) {
    if (!valid_dtype(dtype) || n < 0 || check_cfg(cfg, "vec_axpy_norm2_workspace") != LAK_OK)
        return 0;
    VecPlan p, p1;
    if (plan_vector(LAK_OP_AXPY, dtype, n, cfg, nullptr, 0, &p) != LAK_OK) return 0;
    lak_cfg c = base_cfg(LAK_OP_AXPY, dtype, bucket_of(op_bytes(LAK_OP_AXPY, dtype, n, n, 0)), cfg);
    c.vec = 1;
    if (plan_vector(LAK_OP_AXPY, dtype, n, &c, nullptr, 0, &p1) != LAK_OK) return 0;
    const int grid = p1.L.grid > p.L.grid ? p1.L.grid : p.L.grid;
    return (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)grid;
}

LAK_API lak_status vec_axpy_norm2(void *x, const void *y, const void *z, double alpha, void *out,
                                  int64_t n, lak_dtype dtype, void *workspace, size_t ws_bytes,
                                  const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_axpy_norm2", dtype, cfg);
    if (st != LAK_OK) return st;
    if (n < 0) return fail(LAK_EINVAL, "vec_axpy_norm2: n=%lld < 0", (long long)n);
    if (!out) return fail(LAK_EINVAL, "vec_axpy_norm2: NULL out");
    const int out_bytes = dtype == LAK_F64 ? 8 : 4;
    if ((uintptr_t)out % out_bytes) return fail(LAK_EINVAL, "vec_axpy_norm2: out misaligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(out, 0, out_bytes, s);
        if (e != cudaSuccess)
            return fail(LAK_ECUDA, "vec_axpy_norm2: memset: %s", cudaGetErrorString(e));
        return LAK_OK;
    }
    const int es = esize(dtype);
    if (!x || !y || !z) return fail(LAK_EINVAL, "vec_axpy_norm2: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es) || !aligned_elem(z, es))
        return fail(LAK_EINVAL, "vec_axpy_norm2: pointers not aligned to the element size");
    const void *ptrs[3] = {x, y, z};
    VecPlan p;
    st = plan_vector(LAK_OP_AXPY, dtype, n, cfg, ptrs, 3, &p);
    if (st != LAK_OK) return st;
    const size_t need = (size_t)LAK_WS_COUNTER_BYTES + 8 * (size_t)p.L.grid;
    if (!workspace || ws_bytes < need)
        return fail(LAK_EWORKSPACE, "vec_axpy_norm2: workspace of %zu bytes needed, %zu given",
                    need, workspace ? ws_bytes : (size_t)0);
    if ((uintptr_t)workspace % 256)
        return fail(LAK_EWORKSPACE, "vec_axpy_norm2: workspace not 256-byte aligned");
    return launch_axpy_norm2(dtype, x, y, z, alpha, out, n, workspace, p.L, p.head, s);
}

LAK_API lak_status vec_axpby(void *x, double alpha, const void *y, double beta, const void *z,
                             int64_t n, lak_dtype dtype, const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("vec_axpby", dtype, cfg);
    if (st != LAK_OK) return st;
    if (n < 0) return fail(LAK_EINVAL, "vec_axpby: n=%lld < 0", (long long)n);
    if (n == 0) return LAK_OK;
    const int es = esize(dtype);
    if (!x || !y || !z) return fail(LAK_EINVAL, "vec_axpby: NULL pointer");
    if (!aligned_elem(x, es) || !aligned_elem(y, es) || !aligned_elem(z, es))
        return fail(LAK_EINVAL, "vec_axpby: pointers not aligned to the element size");
    const void *ptrs[3] = {x, y, z};
    VecPlan p;
    st = plan_vector(LAK_OP_AXPY, dtype, n, cfg, ptrs, 3, &p);
    if (st != LAK_OK) return st;
    return launch_axpby(dtype, x, alpha, y, beta, z, n, p.L, p.head, (cudaStream_t)stream);
}

LAK_API lak_status vec_axpby_strided(void *x, int64_t incx, double alpha, const void *y,
                                     int64_t incy, double beta, const void *z, int64_t incz,
                                     int64_t n, lak_dtype dtype, void *stream) {
    if (!valid_dtype(dtype)) return fail(LAK_EDTYPE, "vec_axpby_strided: unknown dtype %d", (int)dtype);
    if (n < 0) return fail(LAK_EINVAL, "vec_axpby_strided: n=%lld < 0", (long long)n);
    if (n == 0) return LAK_OK;
    if (!x || !y || !z) return fail(LAK_EINVAL, "vec_axpby_strided: NULL pointer");
    if (incx == 0) return fail(LAK_EINVAL, "vec_axpby_strided: incx must not be 0");
    const int es = esize(dtype);
    if (!aligned_elem(x, es) || !aligned_elem(y, es) || !aligned_elem(z, es))
        return fail(LAK_EINVAL, "vec_axpby_strided: pointers not aligned to the element size");
    const DeviceInfo *di = device_info();
    if (!di) return LAK_ECUDA;
    const int block = 256;
    int64_t grid = ceil_div(n, block);
    const int64_t cap = (int64_t)di->sms * (di->max_threads_per_sm / block);
    if (grid > cap) grid = cap;
    return launch_axpby_strided(dtype, x, incx, alpha, y, incy, beta, z, incz, n, (int)grid, block,
                                (cudaStream_t)stream);
}

LAK_API lak_status csr_spmv(void *y, const int32_t *row_ptr, const int32_t *col_idx,
                            const void *vals, const void *x, int64_t m, int64_t n, int64_t nnz,
                            lak_dtype dtype, const lak_cfg *cfg, void *stream) {
    lak_status st = common_checks("csr_spmv", dtype, cfg);
    if (st != LAK_OK) return st;
    if (m < 0 || n < 0 || nnz < 0) return fail(LAK_EINVAL, "csr_spmv: negative size");
    if (nnz > 0x7fffffffLL) return fail(LAK_EINVAL, "csr_spmv: nnz exceeds int32 indices");
    if (m == 0) return LAK_OK;
    const int es = esize(dtype);
    if (!y || !row_ptr) return fail(LAK_EINVAL, "csr_spmv: NULL y or row_ptr");
    if (nnz > 0 && (!col_idx || !vals || !x))
        return fail(LAK_EINVAL, "csr_spmv: NULL col_idx, vals or x with nnz > 0");
    if (!aligned_elem(y, es) || !aligned_elem(vals, es) || !aligned_elem(x, es) ||
        !aligned_elem(row_ptr, 4) || !aligned_elem(col_idx, 4))
        return fail(LAK_EINVAL, "csr_spmv: pointers not aligned to their element size");
    SpmvPlan p;
    st = plan_spmv(dtype, m, n, nnz, cfg, &p);
    if (st != LAK_OK) return st;
    return launch_spmv(dtype, y, row_ptr, col_idx, vals, x, m, p.L, p.group, (cudaStream_t)stream);
}

}  // extern "C"
