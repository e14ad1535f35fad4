// api.cpp -- the C ABI of include/sel.h: contexts, argument checks, the
// exact count (§3.1), the push-down with its maxSize contract (Algorithm 1,
// Execute), and batched probe plans with autotuned launch shapes replayed
// from CUDA graphs.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "bucket.h"
#include "internal.h"

namespace sel {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

// Allocation failure injection: the n-th allocation from the arming call on
// (process-wide, every context and thread) fails; 0 = disarmed.
static std::atomic<int64_t> g_fail_alloc{0};

static bool injected_failure() {
    int64_t v = g_fail_alloc.load();
    while (v > 0) {
        if (g_fail_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
    }
    return false;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t host_alloc(void** p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

static sel_status cuda_fail(const char* where, cudaError_t e) {
    set_error("%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SEL_ERR_OOM : SEL_ERR_CUDA;
}

#define SEL_CUDA(where, call)                          \
    do {                                               \
        cudaError_t e__ = (call);                      \
        if (e__ != cudaSuccess) return cuda_fail(where, e__); \
    } while (0)

// A device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    sel_status ensure(size_t bytes, const char* what) {
        if (bytes <= cap) return SEL_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = dev_alloc(&p, std::max<size_t>(bytes, 256));
        if (e != cudaSuccess) return cuda_fail(what, e);
        cap = std::max<size_t>(bytes, 256);
        return SEL_OK;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

struct Shape {
    int tile_rows = 0, stages = 0, ctas_per_sm = 0;
    int warps = 0, group = 0;   // count-scan variant: consumer warps, chunks per instruction pass
    bool auto_tile = false;     // tile_rows is the library's choice: run_scan may shrink it for small tables
};

}  // namespace sel

using namespace sel;

struct sel_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sm = 0;
    int max_smem = 0;         // opt-in shared memory per block
    int max_smem_scan = 0;    // dynamic shared memory available to the scan kernel
    int max_smem_pdp = 0;     // dynamic shared memory available to the persistent push-down
    int max_smem_bucket = 0;  // dynamic shared memory available to the bucket count kernel
    int batch_kernel = 0;     // batch plans: 0 autotuned choice, 1 interpreter only, 2 bucket kernel only
    DevBuf counts;            // sel_count / batch staging
    DevBuf err;               // 4 bytes: error flag of the last launches
    DevBuf pd_scratch;        // push-down: tile status | tile counter | total
    DevBuf pd_mask;           // two-pass push-down: row masks | chunk counts | segment counts | group offsets
    DevBuf distinct_vals;     // sel_count_distinct: the selected values
    DevBuf distinct_table;    // sel_count_distinct: hash set | new-key counter | flags
    DevBuf join_vals;         // sel_join_count: the second side's selected keys
    unsigned long long* h_pinned = nullptr;   // pinned host results (count, total)
    unsigned int* h_err = nullptr;
    size_t h_cap = 0;
    Shape shape;              // overrides for single-predicate scans
    uint64_t launches = 0;
    std::map<std::string, sel_batch_plan*> plans;   // sel_count_batch cache
    long long debug_skip_tile = -1;
    unsigned long long debug_wait_ns = kWaitNs;
    uint32_t pd_super_rows = 0;   // push-down super-tile target (0: chosen from the table size)
    int pd_method = SEL_PD_AUTO;  // push-down method
    cudaEvent_t pd_split_event = nullptr;   // recorded between the two passes of a push-down (timing)
};

struct sel_batch_plan {
    sel_ctx* ctx = nullptr;
    int n = 0;
    void* d_blob = nullptr;
    void* d_counts = nullptr;
    uint32_t blob_bytes = 0, instr_off = 0, pool_off = 0;
    std::vector<TableArg> tables;      // slot pointers, programs per table
    uint32_t n_progs = 0;
    Shape shape;
    float ms = 0.f;
    cudaGraphExec_t graph = nullptr;
    int launches_per_run = 0;
    // the column-bucket form of the same probes (bucket.h), when they fit it
    int kernel = 0;                    // the kernel the plan runs: 0 interpreter, 1 bucket
    void* d_bk_blob = nullptr;
    uint32_t bk_blob_bytes = 0, bk_gb_slots = 0, bk_gb_quad = 0, bk_n_out = 0;
    // graphs that write the counts to a caller's device buffer, by buffer
    std::vector<std::pair<void*, cudaGraphExec_t>> out_graphs;
    // a plan with more than kPlanPartProbes probes on one table runs as parts of
    // at most that many per table, one launch each, into the same counts
    std::vector<sel_batch_plan*> parts;
    ~sel_batch_plan() {
        for (sel_batch_plan* q : parts) delete q;
        if (graph) cudaGraphExecDestroy(graph);
        for (auto& kv : out_graphs) cudaGraphExecDestroy(kv.second);
        if (d_bk_blob) cudaFree(d_bk_blob);
        if (d_blob) cudaFree(d_blob);
        if (d_counts) cudaFree(d_counts);
    }
};

namespace sel {

static sel_status ensure_host(sel_ctx* c, size_t n) {
    if (n <= c->h_cap) return SEL_OK;
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    c->h_pinned = nullptr;
    c->h_cap = 0;
    SEL_CUDA("cudaMallocHost", host_alloc(reinterpret_cast<void**>(&c->h_pinned), n * 8 + 64));
    c->h_cap = n;
    return SEL_OK;
}

static sel_status check_table(const sel_table* t, const char* who) {
    if (!t || (t->n_cols > 0 && !t->cols) || t->n_cols < 0 || t->n_rows < 0) {
        set_error("%s: bad table descriptor", who);
        return SEL_ERR_INVALID_ARG;
    }
    return SEL_OK;
}

// The columns a program reads must exist with the compiled types, be non-null
// and element-aligned.
static sel_status check_pred_on_table(const sel_pred* p, const sel_table* t, const char* who) {
    sel_status s = check_table(t, who);
    if (s != SEL_OK) return s;
    if (!p) {
        set_error("%s: predicate is NULL", who);
        return SEL_ERR_INVALID_ARG;
    }
    for (size_t j = 0; j < p->prog.slot_col.size(); ++j) {
        const int c = p->prog.slot_col[j];
        if (c >= t->n_cols) {
            set_error("%s: predicate reads column %d, table has %d", who, c, t->n_cols);
            return SEL_ERR_INVALID_ARG;
        }
        if (t->cols[c].type != p->col_types[c]) {
            set_error("%s: column %d has type %d, predicate was compiled for %d", who, c, t->cols[c].type,
                      p->col_types[c]);
            return SEL_ERR_TYPE;
        }
        if (t->n_rows > 0) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(t->cols[c].data);
            if (!a || a % p->prog.slot_width[j]) {
                set_error("%s: column %d data pointer is null or not element-aligned", who, c);
                return SEL_ERR_INVALID_ARG;
            }
        }
    }
    return SEL_OK;
}

static void fill_table_arg(TableArg& ta, const std::vector<int32_t>& slot_col, const sel_table* t) {
    std::memset(&ta, 0, sizeof(ta));
    ta.n_rows = t->n_rows;
    ta.n_slots = (uint32_t)slot_col.size();
    ta.tma = 1;
    uint32_t rb = 0;
    for (size_t j = 0; j < slot_col.size(); ++j) {
        const sel_column& c = t->cols[slot_col[j]];
        ta.col[j] = static_cast<const uint8_t*>(c.data);
        ta.width[j] = c.type == SEL_I64 ? 8u : 4u;
        rb += ta.width[j];
        if (reinterpret_cast<uintptr_t>(c.data) % 16) ta.tma = 0;
    }
    ta.row_bytes = rb;
}

static int default_tile_rows(uint32_t row_bytes, int stage_target) {
    if (row_bytes == 0) return 2048;
    int r = (int)(stage_target / row_bytes) / kChunkRows * kChunkRows;
    return std::max(kChunkRows, std::min(kMaxTileRows, r));
}

// The launch shape actually used for a scan: the largest tile (multiple of
// 256 rows, at most the requested one) whose stages fit in shared memory next
// to the counters and the programs, and, when the tile is the library's
// choice, small enough for about 4 tiles per CTA on small tables.
static sel_status resolve_shape(sel_ctx* ctx, uint32_t blob_bytes, uint32_t n_progs,
                                const std::vector<TableArg>& tables, const Shape& sh_in, Shape* out) {
    Shape sh = sh_in;
    uint32_t max_rb = 0;
    for (auto& t : tables) max_rb = std::max(max_rb, t.row_bytes);
    ScanArgs probe;
    std::memset(&probe, 0, sizeof(probe));
    probe.n_progs = n_progs;
    probe.stages = (uint32_t)sh.stages;
    probe.blob_bytes = blob_bytes;
    probe.prog_in_smem = blob_bytes <= 48u * 1024u ? 1u : 0u;
    const size_t fixed = scan_layout(probe);
    if (fixed + 128 * (size_t)sh.stages > (size_t)ctx->max_smem_scan || sh.stages < 1) {
        set_error("scan: %u programs and %d stages do not fit in shared memory", n_progs, sh.stages);
        return SEL_ERR_UNSUPPORTED;
    }
    if (max_rb > 0) {
        const size_t per_stage = ((size_t)ctx->max_smem_scan - fixed) / (size_t)sh.stages;
        const int fit = (int)(per_stage / max_rb) / kChunkRows * kChunkRows;
        if (fit < kChunkRows) {
            set_error("scan: %d stages of 256 rows x %u bytes do not fit in shared memory", sh.stages, max_rb);
            return SEL_ERR_UNSUPPORTED;
        }
        sh.tile_rows = std::min(sh.tile_rows, fit);
    }
    if (sh.auto_tile) {
        int64_t rows = 0;
        for (auto& t : tables) rows += t.n_rows;
        const int64_t want = 4ll * ctx->n_sm * std::max(1, sh.ctas_per_sm);
        const int64_t cap = rows / want / kChunkRows * kChunkRows;
        if (cap < sh.tile_rows) sh.tile_rows = (int)std::max<int64_t>(kChunkRows, cap);
        sh.auto_tile = false;
    }
    *out = sh;
    return SEL_OK;
}

// Fills shape-dependent fields and launches (several launches when the
// tables do not fit in one).
// mask / ccnt: the two-pass push-down's first pass (one program on one
// table: the row masks and chunk counts of ScanArgs), else null.
static sel_status run_scan(sel_ctx* ctx, const uint8_t* d_blob, uint32_t blob_bytes, uint32_t instr_off,
                           uint32_t pool_off, uint32_t n_progs, std::vector<TableArg> tables,
                           unsigned long long* d_counts, const Shape& sh_in, int* n_launches,
                           uint8_t* mask = nullptr, uint16_t* ccnt = nullptr) {
    int launches = 0;
    Shape sh;
    {
        const sel_status rs = resolve_shape(ctx, blob_bytes, n_progs, tables, sh_in, &sh);
        if (rs != SEL_OK) return rs;
    }
    for (size_t t0 = 0; t0 < tables.size(); t0 += kMaxTables) {
        ScanArgs a;
        std::memset(&a, 0, sizeof(a));
        a.blob = d_blob;
        a.n_progs = n_progs;
        a.instr_off = instr_off;
        a.pool_off = pool_off;
        a.blob_bytes = blob_bytes;
        a.tile_rows = (uint32_t)sh.tile_rows;
        a.stages = (uint32_t)sh.stages;
        a.counts = d_counts;
        a.err = static_cast<unsigned int*>(ctx->err.p);
        a.mask = mask;
        a.ccnt = ccnt;
        const size_t t1 = std::min(tables.size(), t0 + kMaxTables);
        a.n_tables = (uint32_t)(t1 - t0);
        uint32_t max_rb = 0;
        int64_t tiles = 0;
        for (size_t i = t0; i < t1; ++i) {
            TableArg ta = tables[i];
            ta.n_tiles = (ta.n_rows + sh.tile_rows - 1) / sh.tile_rows;
            ta.tile_begin = tiles;
            tiles += ta.n_tiles;
            uint32_t off = 0;
            for (uint32_t j = 0; j < ta.n_slots; ++j) {
                ta.slot_off[j] = off;
                off += (uint32_t)sh.tile_rows * ta.width[j];
            }
            max_rb = std::max(max_rb, ta.row_bytes);
            a.t[i - t0] = ta;
        }
        a.total_tiles = tiles;
        a.stage_bytes = ((uint32_t)sh.tile_rows * max_rb + 127u) / 128u * 128u;
        a.prog_in_smem = blob_bytes <= 48u * 1024u ? 1u : 0u;
        size_t smem = scan_layout(a);
        if (smem > (size_t)ctx->max_smem_scan) {
            set_error("scan: %zu bytes of shared memory needed (tile_rows %d, stages %d)", smem, sh.tile_rows,
                      sh.stages);
            return SEL_ERR_UNSUPPORTED;
        }
        if (tiles == 0) continue;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->n_sm * sh.ctas_per_sm));
        cudaError_t e = launch_scan_count(a, (int)grid, smem, ctx->stream, sh.warps, sh.group);
        if (e != cudaSuccess) return cuda_fail("scan launch", e);
        ++launches;
        ctx->launches++;
    }
    if (n_launches) *n_launches = launches;
    return SEL_OK;
}

// The bucket kernel's launch arguments for a plan's tables (one launch: at
// most kMaxTables tables): the largest tile (multiple of 256 rows, at most the
// requested one) whose stages fit next to the counters, the bucket blob and
// the per-warp bucket-index buffers; the library's choice also keeps about 4
// tiles per CTA on small tables.  *smem: the dynamic shared memory needed.
static sel_status resolve_bucket(sel_ctx* ctx, const sel_batch_plan* p, const std::vector<TableArg>& tables,
                                 const Shape& sh_in, ScanArgs* args, size_t* smem, Shape* used) {
    Shape sh = sh_in;
    if (!bucket_variant_ok(sh.warps, sh.group) || sh.stages < 1 || tables.size() > (size_t)kMaxTables) {
        set_error("bucket scan: unsupported launch shape");
        return SEL_ERR_UNSUPPORTED;
    }
    ScanArgs& a = *args;
    std::memset(&a, 0, sizeof(a));
    a.blob = static_cast<const uint8_t*>(p->d_bk_blob);
    a.blob_bytes = p->bk_blob_bytes;
    a.n_progs = p->bk_n_out;
    a.stages = (uint32_t)sh.stages;
    a.err = static_cast<unsigned int*>(ctx->err.p);
    a.n_tables = (uint32_t)tables.size();
    uint32_t max_rb = 0;
    int64_t rows = 0;
    for (auto& t : tables) {
        max_rb = std::max(max_rb, t.row_bytes);
        rows += t.n_rows;
    }
    // bucket indices of a warp's chunk group (the kernel computes the same stride)
    const uint32_t gb_bytes = bk_gb_bytes_per_warp(p->bk_gb_slots, p->bk_gb_quad, (uint32_t)sh.group);
    const size_t fixed = bucket_layout(a, sh.warps, gb_bytes);
    if (fixed + 128 * (size_t)sh.stages > (size_t)ctx->max_smem_bucket) {
        set_error("bucket scan: %zu bytes of tables and counters leave no room for %d stages", fixed, sh.stages);
        return SEL_ERR_UNSUPPORTED;
    }
    if (max_rb > 0) {
        const size_t per_stage = ((size_t)ctx->max_smem_bucket - fixed) / (size_t)sh.stages;
        const int fit = (int)(per_stage / max_rb) / kChunkRows * kChunkRows;
        if (fit < kChunkRows) {
            set_error("bucket scan: %d stages of 256 rows x %u bytes do not fit in shared memory", sh.stages, max_rb);
            return SEL_ERR_UNSUPPORTED;
        }
        sh.tile_rows = std::min(sh.tile_rows, fit);
    }
    if (sh.auto_tile) {
        const int64_t want = 4ll * ctx->n_sm * std::max(1, sh.ctas_per_sm);
        const int64_t cap = rows / want / kChunkRows * kChunkRows;
        if (cap < sh.tile_rows) sh.tile_rows = (int)std::max<int64_t>(kChunkRows, cap);
        sh.auto_tile = false;
    }
    a.tile_rows = (uint32_t)sh.tile_rows;
    int64_t tiles = 0;
    for (size_t i = 0; i < tables.size(); ++i) {
        TableArg ta = tables[i];
        ta.n_tiles = (ta.n_rows + sh.tile_rows - 1) / sh.tile_rows;
        ta.tile_begin = tiles;
        tiles += ta.n_tiles;
        uint32_t off = 0;
        for (uint32_t j = 0; j < ta.n_slots; ++j) {
            ta.slot_off[j] = off;
            off += (uint32_t)sh.tile_rows * ta.width[j];
        }
        a.t[i] = ta;
    }
    a.total_tiles = tiles;
    {   // the kernel's per-CTA counts are 32-bit: a CTA (one of at least n_sm) must scan fewer than 2^32 rows
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)ctx->n_sm * sh.ctas_per_sm));
        if ((tiles + grid - 1) / grid * (int64_t)sh.tile_rows >= (int64_t(1) << 32)) {
            set_error("bucket scan: more than 2^32 rows a CTA");
            return SEL_ERR_UNSUPPORTED;
        }
    }
    a.stage_bytes = ((uint32_t)sh.tile_rows * max_rb + 127u) / 128u * 128u;
    *smem = bucket_layout(a, sh.warps, gb_bytes);
    if (*smem > (size_t)ctx->max_smem_bucket) {
        set_error("bucket scan: %zu bytes of shared memory needed", *smem);
        return SEL_ERR_UNSUPPORTED;
    }
    if (used) *used = sh;
    return SEL_OK;
}

static sel_status run_bucket(sel_ctx* ctx, const sel_batch_plan* p, const Shape& sh_in, unsigned long long* d_counts,
                             int* n_launches) {
    ScanArgs a;
    size_t smem = 0;
    Shape sh;
    sel_status s = resolve_bucket(ctx, p, p->tables, sh_in, &a, &smem, &sh);
    if (s != SEL_OK) return s;
    a.counts = d_counts;
    int launches = 0;
    if (a.total_tiles > 0) {
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(a.total_tiles, (int64_t)ctx->n_sm * sh.ctas_per_sm));
        cudaError_t e = launch_bucket_count(a, (int)grid, smem, ctx->stream, sh.warps, sh.group);
        if (e != cudaSuccess) return cuda_fail("bucket scan launch", e);
        ++launches;
        ctx->launches++;
    }
    if (n_launches) *n_launches = launches;
    return SEL_OK;
}

static Shape single_shape(sel_ctx* ctx, uint32_t row_bytes) {
    Shape s;
    // 3 stages that fill shared memory (the tile is shrunk to fit by
    // run_scan), one CTA per SM of 15 consumer warps (128 registers a thread)
    // with 3 chunks per instruction pass: over the 203 push-downs of a
    // 1.2B-row table their count passes took 527 ms, against 550 ms with 16
    // warps of 96 registers and 2 chunks
    (void)row_bytes;
    s.stages = ctx->shape.stages > 0 ? ctx->shape.stages : 3;
    s.ctas_per_sm = ctx->shape.ctas_per_sm > 0 ? ctx->shape.ctas_per_sm : 1;
    s.tile_rows = ctx->shape.tile_rows > 0 ? ctx->shape.tile_rows : kMaxTileRows;
    s.auto_tile = ctx->shape.tile_rows <= 0;
    s.warps = kScanDefaultWarps;
    s.group = kScanDefaultGroup;
    if (ctx->shape.warps > 0 && scan_variant_ok(ctx->shape.warps, ctx->shape.group)) {   // not a bucket-only variant
        s.warps = ctx->shape.warps;
        s.group = ctx->shape.group;
    }
    return s;
}

static sel_status sync_and_check(sel_ctx* ctx, const char* who) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(who, e);
    return SEL_OK;
}

}  // namespace sel

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" const char* sel_last_error(void) { return sel::g_err.c_str(); }

extern "C" const char* sel_status_str(sel_status s) {
    switch (s) {
    case SEL_OK: return "SEL_OK";
    case SEL_ERR_INVALID_ARG: return "SEL_ERR_INVALID_ARG";
    case SEL_ERR_TYPE: return "SEL_ERR_TYPE";
    case SEL_ERR_UNSUPPORTED: return "SEL_ERR_UNSUPPORTED";
    case SEL_ERR_OOM: return "SEL_ERR_OOM";
    case SEL_ERR_CUDA: return "SEL_ERR_CUDA";
    case SEL_ERR_TOO_LARGE: return "SEL_ERR_TOO_LARGE";
    case SEL_ERR_TIMEOUT: return "SEL_ERR_TIMEOUT";
    }
    return "SEL_ERR_UNKNOWN";
}

extern "C" sel_status sel_ctx_create(void* cuda_stream, sel_ctx** out) {
    if (!out) {
        set_error("sel_ctx_create: out is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int dev = 0;
    SEL_CUDA("cudaGetDevice", cudaGetDevice(&dev));
    std::unique_ptr<sel_ctx> c(new sel_ctx());
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->device = dev;
    SEL_CUDA("cudaDeviceGetAttribute", cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev));
    SEL_CUDA("cudaDeviceGetAttribute",
             cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    SEL_CUDA("scan smem attribute", scan_kernel_max_smem(c->max_smem, &c->max_smem_scan));
    SEL_CUDA("push-down smem attribute", pushdown_persistent_max_smem(c->max_smem, &c->max_smem_pdp));
    SEL_CUDA("bucket smem attribute", bucket_kernel_max_smem(c->max_smem, &c->max_smem_bucket));
    // The push-down's gathers read one 4- or 8-byte value per selected row:
    // with the L2 fetching 32 bytes per miss instead of a whole line they move
    // a quarter of the DRAM bytes (the scans and their bulk copies read whole
    // lines either way).  A hint of this process's context on the device.
    SEL_CUDA("cudaDeviceSetLimit", cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32));
    sel_status s = c->err.ensure(256, "error flag");
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemset", cudaMemset(c->err.p, 0, 256));
    s = ensure_host(c.get(), 64);
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMallocHost", host_alloc(reinterpret_cast<void**>(&c->h_err), 64));
    *out = c.release();
    return SEL_OK;
}

extern "C" void sel_ctx_destroy(sel_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->plans) sel_batch_plan_free(kv.second);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->h_err) cudaFreeHost(c->h_err);
    delete c;
}

extern "C" sel_status sel_ctx_set_scan_shape(sel_ctx* c, int32_t tile_rows, int32_t stages, int32_t ctas_per_sm) {
    if (!c || tile_rows < 0 || tile_rows % kChunkRows || tile_rows > kMaxTileRows || stages < 0 || stages > 16 ||
        ctas_per_sm < 0 || ctas_per_sm > 8) {
        set_error("sel_ctx_set_scan_shape: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    c->shape.tile_rows = tile_rows;
    c->shape.stages = stages;
    c->shape.ctas_per_sm = ctas_per_sm;
    return SEL_OK;
}

extern "C" sel_status sel_ctx_set_scan_variant(sel_ctx* c, int32_t consumer_warps, int32_t chunks_per_pass) {
    if (!c || !((consumer_warps == 0 && chunks_per_pass == 0) || scan_variant_ok(consumer_warps, chunks_per_pass) ||
                bucket_variant_ok(consumer_warps, chunks_per_pass) ||
                pushdown_persistent_ok(consumer_warps, chunks_per_pass))) {
        set_error("sel_ctx_set_scan_variant: bad arguments (0,0; warps 8|16 with chunks 1|2; warps 8 with chunks 4; warps 15 with chunks 2|3; "
                  "bucket kernel only: warps 11|15 with chunks 1|2; push-down only: warps 12 with chunks 1|2|3)");
        return SEL_ERR_INVALID_ARG;
    }
    c->shape.warps = consumer_warps;
    c->shape.group = chunks_per_pass;
    return SEL_OK;
}

extern "C" uint64_t sel_ctx_launch_count(const sel_ctx* c) { return c ? c->launches : 0; }

extern "C" sel_status sel_debug_fail_allocation(int64_t nth) {
    if (nth < 0) {
        set_error("sel_debug_fail_allocation: nth must be >= 0");
        return SEL_ERR_INVALID_ARG;
    }
    g_fail_alloc.store(nth);
    return SEL_OK;
}

namespace sel {
cudaStream_t ctx_stream(sel_ctx* c) { return c->stream; }
uint64_t& thread_launches() {
    thread_local uint64_t n = 0;
    return n;
}
int& thread_tally_depth() {
    thread_local int d = 0;
    return d;
}
void ctx_add_launches(sel_ctx* c, uint64_t n) { c->launches += n; }
}

extern "C" sel_status sel_ctx_set_pushdown_super_rows(sel_ctx* c, int32_t rows) {
    if (!c || rows < 0 || (rows > 0 && (rows % kChunkRows || rows > kPdpMaxChunks * kChunkRows))) {
        set_error("sel_ctx_set_pushdown_super_rows: rows must be 0 or a multiple of 256 up to %d",
                  kPdpMaxChunks * kChunkRows);
        return SEL_ERR_INVALID_ARG;
    }
    c->pd_super_rows = (uint32_t)rows;
    return SEL_OK;
}

extern "C" sel_status sel_ctx_set_pushdown_method(sel_ctx* c, int32_t method) {
    if (!c || method < SEL_PD_AUTO || method > SEL_PD_ONE_PASS) {
        set_error("sel_ctx_set_pushdown_method: method must be SEL_PD_AUTO, SEL_PD_TWO_PASS or SEL_PD_ONE_PASS");
        return SEL_ERR_INVALID_ARG;
    }
    c->pd_method = method;
    return SEL_OK;
}

extern "C" sel_status sel_ctx_set_pushdown_split_event(sel_ctx* c, void* cuda_event) {
    if (!c) {
        set_error("sel_ctx_set_pushdown_split_event: ctx is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    c->pd_split_event = static_cast<cudaEvent_t>(cuda_event);
    return SEL_OK;
}

extern "C" sel_status sel_ctx_debug_pushdown_fault(sel_ctx* c, int64_t skip_tile, uint64_t wait_ns) {
    if (!c) {
        set_error("sel_ctx_debug_pushdown_fault: ctx is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    c->debug_skip_tile = skip_tile;
    c->debug_wait_ns = wait_ns ? wait_ns : kWaitNs;
    return SEL_OK;
}

static sel_status count_enqueue(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                unsigned long long* d_out, const char* who) {
    sel_status s = check_pred_on_table(pred, table, who);
    if (s != SEL_OK) return s;
    s = pred_upload(pred);
    if (s != SEL_OK) return s;
    TableArg ta;
    fill_table_arg(ta, pred->prog.slot_col, table);
    ta.prog_begin = 0;
    ta.prog_end = 1;
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(d_out, 0, 8, ctx->stream));
    const Shape sh = single_shape(ctx, ta.row_bytes);
    return run_scan(ctx, static_cast<const uint8_t*>(pred->d_blob), pred->blob_bytes, pred->instr_off,
                    pred->pool_off, 1, {ta}, d_out, sh, nullptr);
}

extern "C" sel_status sel_count_async(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                      uint64_t* dev_out_count) {
    if (!ctx || !dev_out_count) {
        set_error("sel_count_async: null context or output");
        return SEL_ERR_INVALID_ARG;
    }
    return count_enqueue(ctx, pred, table, reinterpret_cast<unsigned long long*>(dev_out_count), "sel_count_async");
}

extern "C" sel_status sel_count(sel_ctx* ctx, const sel_pred* pred, const sel_table* table, uint64_t* out_count) {
    if (!ctx || !out_count) {
        set_error("sel_count: null context or output");
        return SEL_ERR_INVALID_ARG;
    }
    sel_status s = ctx->counts.ensure(64, "count buffer");
    if (s != SEL_OK) return s;
    unsigned long long* d = static_cast<unsigned long long*>(ctx->counts.p);
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(ctx->err.p, 0, 4, ctx->stream));
    s = count_enqueue(ctx, pred, table, d, "sel_count");
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_pinned, d, 8, cudaMemcpyDeviceToHost, ctx->stream));
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, ctx->err.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_and_check(ctx, "sel_count");
    if (s != SEL_OK) return s;
    if (*ctx->h_err) {
        set_error("sel_count: a device wait timed out");
        return SEL_ERR_TIMEOUT;
    }
    *out_count = ctx->h_pinned[0];
    return SEL_OK;
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// The two-pass push-down: the count scan with the mask output (chunk masks
// and counts), the segment counts, the group offsets and the exact count
// (d_total), and the scatter of the selected rows (skipped when nothing is to
// be written).  `a` holds the projection.
static sel_status pushdown_two_pass(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                    const PushdownArgs& a, int64_t* dev_out_rowids, uint64_t max_rows,
                                    unsigned long long* d_total) {
    const int64_t n = table->n_rows;
    if (n == 0) {
        SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(d_total, 0, 8, ctx->stream));
        return SEL_OK;
    }
    const int64_t n_chunks = (n + kChunkRows - 1) / kChunkRows;
    const int64_t n_seg = (n_chunks + kSegChunks - 1) / kSegChunks;
    const int64_t n_grp = (n_seg + kGrpSegs - 1) / kGrpSegs;
    // scratch: segment counts | group offsets | chunk counts | row masks (every entry written before it is read)
    const size_t seg_bytes = align256((size_t)n_grp * kGrpSegs * 4);
    const size_t off_bytes = align256((size_t)n_grp * 8);
    const size_t ccnt_bytes = align256((size_t)n_chunks * 2);
    const size_t mask_bytes = align256((size_t)n_chunks * 32);
    sel_status s = ctx->pd_mask.ensure(seg_bytes + off_bytes + ccnt_bytes + mask_bytes, "push-down masks");
    if (s != SEL_OK) return s;
    uint8_t* base = static_cast<uint8_t*>(ctx->pd_mask.p);
    uint32_t* seg_cnt = reinterpret_cast<uint32_t*>(base);
    unsigned long long* grp_off = reinterpret_cast<unsigned long long*>(base + seg_bytes);
    uint16_t* ccnt = reinterpret_cast<uint16_t*>(base + seg_bytes + off_bytes);
    uint8_t* mask = base + seg_bytes + off_bytes + ccnt_bytes;
    TableArg ta;
    fill_table_arg(ta, pred->prog.slot_col, table);
    ta.prog_begin = 0;
    ta.prog_end = 1;
    const Shape sh = single_shape(ctx, ta.row_bytes);
    s = run_scan(ctx, static_cast<const uint8_t*>(pred->d_blob), pred->blob_bytes, pred->instr_off, pred->pool_off,
                 1, {ta}, d_total, sh, nullptr, mask, ccnt);
    if (s != SEL_OK) return s;
    if (ctx->pd_split_event) SEL_CUDA("cudaEventRecord", cudaEventRecord(ctx->pd_split_event, ctx->stream));
    cudaError_t e = launch_seg_sum(ccnt, n_chunks, seg_cnt, n_grp, ctx->stream);
    if (e == cudaSuccess) e = launch_seg_scan(seg_cnt, grp_off, n_grp, d_total, ctx->stream);
    if (e != cudaSuccess) return cuda_fail("push-down offsets launch", e);
    ctx->launches += 2;
    if (max_rows == 0 || (a.n_proj == 0 && !dev_out_rowids)) return SEL_OK;
    ScatterArgs sa;
    std::memset(&sa, 0, sizeof(sa));
    sa.mask = mask;
    sa.ccnt = ccnt;
    sa.seg_cnt = seg_cnt;
    sa.grp_off = grp_off;
    sa.n_rows = n;
    sa.n_seg = n_seg;
    sa.n_proj = a.n_proj;
    for (uint32_t j = 0; j < a.n_proj; ++j) {
        sa.src[j] = a.proj_src[j];
        sa.dst[j] = a.proj_dst[j];
        sa.width[j] = a.proj_width[j];
    }
    sa.rowids = reinterpret_cast<long long*>(dev_out_rowids);
    sa.max_rows = max_rows;
    e = launch_pushdown_scatter(sa, ctx->stream);
    if (e != cudaSuccess) return cuda_fail("push-down scatter launch", e);
    ctx->launches++;
    return SEL_OK;
}

// Enqueues the push-down; the exact count lands in d_total (device).
static sel_status pushdown_enqueue(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                   const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                                   int64_t* dev_out_rowids, uint64_t max_rows, unsigned long long* d_total,
                                   const char* who) {
    if (!ctx || n_proj < 0 || n_proj > kPdMaxProj || (n_proj > 0 && (!proj_cols || !dev_out_cols))) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    sel_status s = check_pred_on_table(pred, table, who);
    if (s != SEL_OK) return s;
    PushdownArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int32_t j = 0; j < n_proj; ++j) {
        const int c = proj_cols[j];
        if (c < 0 || c >= table->n_cols) {
            set_error("%s: projected column %d out of range", who, c);
            return SEL_ERR_INVALID_ARG;
        }
        const sel_column& col = table->cols[c];
        if (col.type < SEL_I32 || col.type > SEL_DICT) {
            set_error("%s: projected column %d has an unknown type", who, c);
            return SEL_ERR_TYPE;
        }
        const uint32_t w = col.type == SEL_I64 ? 8u : 4u;
        const uintptr_t src = reinterpret_cast<uintptr_t>(col.data);
        const uintptr_t dst = reinterpret_cast<uintptr_t>(dev_out_cols[j]);
        if ((table->n_rows > 0 && (!src || src % w)) || (max_rows > 0 && (!dst || dst % w))) {
            set_error("%s: projected column %d: null or misaligned source/output pointer", who, c);
            return SEL_ERR_INVALID_ARG;
        }
        a.proj_src[j] = reinterpret_cast<const uint8_t*>(col.data);
        a.proj_dst[j] = static_cast<uint8_t*>(dev_out_cols[j]);
        a.proj_width[j] = w;
        a.proj_slot[j] = -1;
        for (size_t k = 0; k < pred->prog.slot_col.size(); ++k)
            if (pred->prog.slot_col[k] == c) a.proj_slot[j] = (int32_t)k;
    }
    if (dev_out_rowids && reinterpret_cast<uintptr_t>(dev_out_rowids) % 8) {
        set_error("%s: row id output is not 8-byte aligned", who);
        return SEL_ERR_INVALID_ARG;
    }
    s = pred_upload(pred);
    if (s != SEL_OK) return s;
    a.n_proj = (uint32_t)n_proj;
    if (ctx->pd_method != SEL_PD_ONE_PASS)
        return pushdown_two_pass(ctx, pred, table, a, dev_out_rowids, max_rows, d_total);
    TableArg ta;
    fill_table_arg(ta, pred->prog.slot_col, table);
    a.blob = static_cast<const uint8_t*>(pred->d_blob);
    a.instr_off = pred->instr_off;
    a.pool_off = pred->pool_off;
    a.blob_bytes = pred->blob_bytes;
    a.n_instr = (uint32_t)pred->prog.instrs.size();
    a.n_slots = ta.n_slots;
    a.row_bytes = ta.row_bytes;
    a.tma = ta.tma;
    // The persistent kernel: super-tiles (the largest multiple of the sub-tile
    // up to a target size) streamed in sub-tiles through shared-memory stages.
    // The target: the context's, else 384 KB of predicate columns (a CTA's
    // look-back of a super-tile takes a few microseconds: the super-tile
    // should stream for longer) but no more than 1/16 of a CTA's share of the
    // table (its last super-tile is looked back and written after the scan),
    // at least 32768 and at most 131072 rows; larger super-tiles take shared
    // memory (their row masks) from the stages.
    // Variant: the context's scan variant, else 12 consumer warps x 3 chunks
    // per pass (with the producer, look-back and 2 writer warps, 16 warps of
    // 128 registers: no spills in the evaluation loop; measured faster on
    // config 5's push-downs than 16 consumer warps of 96 registers, and 3
    // chunks a pass than 2), or 2 chunks when a requested sub-tile is a
    // multiple of 512 rows but not of 768.  Sub-tile and stages: the requested ones, else the count
    // scan's rule: 3 stages (2 if 3 do not fit) of the largest sub-tile, in
    // whole chunk groups, that fits in shared memory beside the row masks.  A
    // tile size the persistent kernel cannot use, or predicate columns too wide
    // for two stages, take the one-CTA-per-tile kernel (1024 rows or as
    // requested).
    {
        const int req = ctx->shape.tile_rows;
        const bool own = ctx->shape.warps > 0 && pushdown_persistent_ok(ctx->shape.warps, ctx->shape.group);
        const int W = own ? ctx->shape.warps : 12;
        const int G = own ? ctx->shape.group : (req > 0 && req % (3 * kChunkRows) != 0 ? 2 : 3);
        const int unit = kChunkRows * G;
        uint32_t target = ctx->pd_super_rows;
        if (target == 0) {
            const int64_t per = table->n_rows / (16 * (int64_t)std::max(1, ctx->n_sm));
            const int64_t by_bytes = (int64_t)(384u << 10) / std::max<int64_t>(1, ta.row_bytes);
            target = (uint32_t)std::max<int64_t>(std::min<int64_t>(std::min<int64_t>(per, by_bytes),
                                                                    kPdpMaxChunks * kChunkRows),
                                                  kPdpMinSuperRows);
        }
        target = target / kChunkRows * kChunkRows;
        int best_tr = 0, best_s = 0;
        if (pushdown_persistent_ok(W, G) && ta.row_bytes > 0) {
            const int tr0 = req > 0 ? req : (int)target / unit * unit;
            for (int S = ctx->shape.stages > 0 ? ctx->shape.stages : 3; S >= 2 && best_tr == 0; --S) {
                for (int tr = tr0; tr >= unit; tr -= unit) {
                    if (req > 0 && tr != req) break;
                    if (!pushdown_persistent_tile_ok((uint32_t)tr, G)) continue;
                    PushdownArgs p = a;
                    p.blob_bytes = pred->blob_bytes;
                    p.row_bytes = ta.row_bytes;
                    p.tile_rows = (uint32_t)tr;
                    p.stages = (uint32_t)S;
                    p.super_rows = pushdown_super_rows((uint32_t)tr, std::max<uint32_t>(target, (uint32_t)tr));
                    if (pushdown_persistent_layout(p) <= (size_t)ctx->max_smem_pdp) {
                        best_tr = tr;
                        best_s = S;
                        break;
                    }
                }
            }
        }
        if (best_tr > 0) {
            const int S = best_s;
            a.tile_rows = (uint32_t)best_tr;
            a.stages = (uint32_t)S;
            a.blob = static_cast<const uint8_t*>(pred->d_blob);
            a.instr_off = pred->instr_off;
            a.pool_off = pred->pool_off;
            a.blob_bytes = pred->blob_bytes;
            a.n_instr = (uint32_t)pred->prog.instrs.size();
            a.n_slots = ta.n_slots;
            a.row_bytes = ta.row_bytes;
            a.tma = ta.tma;
            a.super_rows = pushdown_super_rows(a.tile_rows, std::max<uint32_t>(target, a.tile_rows));
            pushdown_persistent_layout(a);
            uint32_t off = 0;
            for (uint32_t j = 0; j < ta.n_slots; ++j) {
                a.col[j] = ta.col[j];
                a.width[j] = ta.width[j];
                a.slot_off[j] = off;
                off += a.tile_rows * ta.width[j];
            }
            a.n_rows = table->n_rows;
            a.n_tiles = (table->n_rows + a.super_rows - 1) / a.super_rows;   // look-back unit: super-tiles
            a.n_proj = (uint32_t)n_proj;
            a.rowids = reinterpret_cast<long long*>(dev_out_rowids);
            a.max_rows = max_rows;
            a.skip_publish_tile = ctx->debug_skip_tile;
            a.wait_ns = ctx->debug_wait_ns;
            const size_t status_bytes = (size_t)a.n_tiles * 8;
            s = ctx->pd_scratch.ensure(status_bytes + 64, "push-down scratch");
            if (s != SEL_OK) return s;
            uint8_t* scr = static_cast<uint8_t*>(ctx->pd_scratch.p);
            a.status = reinterpret_cast<unsigned long long*>(scr);
            a.tile_counter64 = reinterpret_cast<unsigned long long*>(scr + status_bytes);
            a.total = d_total;
            a.err = static_cast<unsigned int*>(ctx->err.p);
            SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(scr, 0, status_bytes + 64, ctx->stream));
            SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(d_total, 0, 8, ctx->stream));
            const int grid = (int)std::min<int64_t>(a.n_tiles, (int64_t)ctx->n_sm);
            cudaError_t e = launch_pushdown_persistent(a, grid, W, G, ctx->stream);
            if (e != cudaSuccess) return cuda_fail("push-down launch", e);
            if (a.n_tiles > 0) ctx->launches++;
            return SEL_OK;
        }
    }
    a.tile_rows = ctx->shape.tile_rows > 0 ? (uint32_t)std::min(ctx->shape.tile_rows, kPdMaxTileRows) : 1024u;
    {   // shrink the tile until its stage fits in shared memory
        const size_t fixed = ((size_t)pred->blob_bytes + 127) / 128 * 128 + 1024;
        while (a.tile_rows > (uint32_t)kChunkRows && fixed + (size_t)a.tile_rows * ta.row_bytes > (size_t)ctx->max_smem)
            a.tile_rows -= kChunkRows;
    }
    uint32_t off = 0;
    for (uint32_t j = 0; j < ta.n_slots; ++j) {
        a.col[j] = ta.col[j];
        a.width[j] = ta.width[j];
        a.slot_off[j] = off;
        off += a.tile_rows * ta.width[j];
    }
    a.n_rows = table->n_rows;
    a.n_tiles = (table->n_rows + a.tile_rows - 1) / a.tile_rows;
    a.n_proj = (uint32_t)n_proj;
    a.rowids = reinterpret_cast<long long*>(dev_out_rowids);
    a.max_rows = max_rows;
    a.skip_publish_tile = ctx->debug_skip_tile;
    a.wait_ns = ctx->debug_wait_ns;
    const size_t smem = pushdown_layout(a);
    if (smem > (size_t)ctx->max_smem) {
        set_error("%s: %zu bytes of shared memory needed", who, smem);
        return SEL_ERR_UNSUPPORTED;
    }
    // scratch: status[n_tiles] | tile counter
    const size_t status_bytes = (size_t)a.n_tiles * 8;
    s = ctx->pd_scratch.ensure(status_bytes + 64, "push-down scratch");
    if (s != SEL_OK) return s;
    uint8_t* scr = static_cast<uint8_t*>(ctx->pd_scratch.p);
    a.status = reinterpret_cast<unsigned long long*>(scr);
    a.tile_counter = reinterpret_cast<unsigned int*>(scr + status_bytes);
    a.total = d_total;
    a.err = static_cast<unsigned int*>(ctx->err.p);
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(scr, 0, status_bytes + 64, ctx->stream));
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(d_total, 0, 8, ctx->stream));
    cudaError_t e = launch_pushdown(a, ctx->stream);
    if (e != cudaSuccess) return cuda_fail("push-down launch", e);
    if (a.n_tiles > 0) ctx->launches++;
    return SEL_OK;
}

extern "C" sel_status sel_pushdown_async(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                         const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                                         int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* dev_out_count) {
    if (!dev_out_count) {
        set_error("sel_pushdown_async: dev_out_count is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    return pushdown_enqueue(ctx, pred, table, proj_cols, n_proj, dev_out_cols, dev_out_rowids, max_rows,
                            reinterpret_cast<unsigned long long*>(dev_out_count), "sel_pushdown_async");
}

// ---------------------------------------------------------------------------
// V(R, A) and the join-size estimate of §1.1 / §3.2
// ---------------------------------------------------------------------------

namespace sel {
cudaError_t launch_distinct(const uint8_t* col, int type, int64_t n, unsigned long long* table, unsigned long long cap,
                            unsigned long long* n_new, unsigned int* flags, int n_sm, cudaStream_t st);
}

extern "C" sel_status sel_count_distinct(sel_ctx* ctx, const sel_table* table, int32_t col, const sel_pred* pred,
                                         uint64_t* out_distinct, uint64_t* out_rows) {
    const char* who = "sel_count_distinct";
    if (!ctx || !table || !out_distinct || col < 0 || col >= table->n_cols || table->n_rows < 0) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    const sel_column& c = table->cols[col];
    const int type = c.type == SEL_I64 ? 1 : c.type == SEL_F32 ? 2 : 0;
    const uint32_t width = c.type == SEL_I64 ? 8u : 4u;
    if (table->n_rows > 0 && (!c.data || reinterpret_cast<uintptr_t>(c.data) % width)) {
        set_error("%s: column %d: null or misaligned data", who, col);
        return SEL_ERR_INVALID_ARG;
    }
    const uint8_t* vals = static_cast<const uint8_t*>(c.data);
    uint64_t nv = (uint64_t)table->n_rows;
    if (pred) {   // the selected values, compacted by the push-down
        sel_status s = ctx->distinct_vals.ensure(std::max<size_t>(1, (size_t)table->n_rows) * width, who);
        if (s != SEL_OK) return s;
        void* dst = ctx->distinct_vals.p;
        const int32_t proj = col;
        uint64_t cnt = 0;
        s = sel_pushdown(ctx, pred, table, &proj, 1, &dst, nullptr, (uint64_t)table->n_rows, &cnt);
        if (s != SEL_OK) return s;
        vals = static_cast<const uint8_t*>(ctx->distinct_vals.p);
        nv = cnt;
    }
    unsigned long long cap = 1024;
    while (cap < 2 * (unsigned long long)nv) cap <<= 1;
    sel_status s = ctx->distinct_table.ensure((size_t)cap * 8 + 64, who);
    if (s != SEL_OK) return s;
    unsigned long long* tab = static_cast<unsigned long long*>(ctx->distinct_table.p);
    unsigned long long* n_new = tab + cap;
    unsigned int* flags = reinterpret_cast<unsigned int*>(tab + cap + 1);
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(tab, 0xFF, (size_t)cap * 8, ctx->stream));
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(n_new, 0, 64, ctx->stream));
    cudaError_t e = launch_distinct(vals, type, (int64_t)nv, tab, cap, n_new, flags, ctx->n_sm, ctx->stream);
    if (e != cudaSuccess) return cuda_fail("distinct launch", e);
    if (nv > 0) ctx->launches++;
    s = ensure_host(ctx, 2);
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_pinned, n_new, 8, cudaMemcpyDeviceToHost, ctx->stream));
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, flags, 4, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_and_check(ctx, who);
    if (s != SEL_OK) return s;
    if (*ctx->h_err & 1u) {
        set_error("%s: a probe sequence exceeded the table", who);
        return SEL_ERR_CUDA;
    }
    *out_distinct = ctx->h_pinned[0] + ((*ctx->h_err & 2u) ? 1u : 0u);
    if (out_rows) *out_rows = nv;
    return SEL_OK;
}

namespace sel {
cudaError_t launch_join_count(const uint8_t* build, int64_t n_build, const uint8_t* probe, int64_t n_probe, int type,
                              unsigned long long* keys, unsigned long long* mult, unsigned long long cap,
                              unsigned long long* counters, unsigned int* flags, int n_sm, cudaStream_t st);

// The key values of the selected rows of one side: the column itself, or the
// push-down's compaction of it into `buf`.
static sel_status join_side(sel_ctx* ctx, const sel_table* t, int32_t col, const sel_pred* pred, DevBuf& buf,
                            const uint8_t** vals, uint64_t* n, const char* who) {
    const sel_column& c = t->cols[col];
    const uint32_t width = c.type == SEL_I64 ? 8u : 4u;
    if (t->n_rows > 0 && (!c.data || reinterpret_cast<uintptr_t>(c.data) % width)) {
        set_error("%s: column %d: null or misaligned data", who, col);
        return SEL_ERR_INVALID_ARG;
    }
    *vals = static_cast<const uint8_t*>(c.data);
    *n = (uint64_t)t->n_rows;
    if (!pred) return SEL_OK;
    sel_status s = buf.ensure(std::max<size_t>(1, (size_t)t->n_rows) * width, who);
    if (s != SEL_OK) return s;
    void* dst = buf.p;
    uint64_t cnt = 0;
    s = sel_pushdown(ctx, pred, t, &col, 1, &dst, nullptr, (uint64_t)t->n_rows, &cnt);
    if (s != SEL_OK) return s;
    *vals = static_cast<const uint8_t*>(buf.p);
    *n = cnt;
    return SEL_OK;
}
}  // namespace sel

extern "C" sel_status sel_join_count(sel_ctx* ctx, const sel_table* r, int32_t col_r, const sel_pred* pred_r,
                                     const sel_table* s_tab, int32_t col_s, const sel_pred* pred_s,
                                     uint64_t* out_count, uint64_t* out_rows_r, uint64_t* out_rows_s) {
    const char* who = "sel_join_count";
    if (!ctx || !r || !s_tab || !out_count || col_r < 0 || col_r >= r->n_cols || col_s < 0 || col_s >= s_tab->n_cols) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    const bool fr = r->cols[col_r].type == SEL_F32, fs = s_tab->cols[col_s].type == SEL_F32;
    if (fr != fs) {
        set_error("%s: a float32 key joins only a float32 key", who);
        return SEL_ERR_TYPE;
    }
    const uint8_t *vr = nullptr, *vs = nullptr;
    uint64_t nr = 0, ns = 0;
    sel_status st = join_side(ctx, r, col_r, pred_r, ctx->distinct_vals, &vr, &nr, who);
    if (st != SEL_OK) return st;
    st = join_side(ctx, s_tab, col_s, pred_s, ctx->join_vals, &vs, &ns, who);
    if (st != SEL_OK) return st;
    // keys of different widths: widen both sides to the same 64-bit keys (type codes of distinct.cu)
    const int type_r = r->cols[col_r].type == SEL_I64 ? 1 : fr ? 2 : 0;
    const int type_s = s_tab->cols[col_s].type == SEL_I64 ? 1 : fs ? 2 : 0;
    if (type_r != type_s) {
        set_error("%s: int32 and int64 keys: join columns of the same width", who);
        return SEL_ERR_UNSUPPORTED;
    }
    const bool build_r = nr <= ns;
    const uint8_t* build = build_r ? vr : vs;
    const uint8_t* probe = build_r ? vs : vr;
    const uint64_t nb = build_r ? nr : ns, np = build_r ? ns : nr;
    unsigned long long cap = 1024;
    while (cap < 2 * (unsigned long long)nb) cap <<= 1;
    st = ctx->distinct_table.ensure((size_t)cap * 16 + 64, who);
    if (st != SEL_OK) return st;
    unsigned long long* keys = static_cast<unsigned long long*>(ctx->distinct_table.p);
    unsigned long long* mult = keys + cap;
    unsigned long long* counters = keys + 2 * cap;
    unsigned int* flags = reinterpret_cast<unsigned int*>(keys + 2 * cap + 2);
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(keys, 0xFF, (size_t)cap * 8, ctx->stream));
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(mult, 0, (size_t)cap * 8 + 64, ctx->stream));
    cudaError_t e = launch_join_count(build, (int64_t)nb, probe, (int64_t)np, type_r, keys, mult, cap, counters, flags,
                                      ctx->n_sm, ctx->stream);
    if (e != cudaSuccess) return cuda_fail("join count launch", e);
    ctx->launches += (nb > 0 ? 1 : 0) + (nb > 0 && np > 0 ? 1 : 0);
    st = ensure_host(ctx, 2);
    if (st != SEL_OK) return st;
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_pinned, counters, 8, cudaMemcpyDeviceToHost, ctx->stream));
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, flags, 4, cudaMemcpyDeviceToHost, ctx->stream));
    st = sync_and_check(ctx, who);
    if (st != SEL_OK) return st;
    if (*ctx->h_err & 1u) {
        set_error("%s: a probe sequence exceeded the table", who);
        return SEL_ERR_CUDA;
    }
    *out_count = ctx->h_pinned[0];
    if (out_rows_r) *out_rows_r = nr;
    if (out_rows_s) *out_rows_s = ns;
    return SEL_OK;
}

extern "C" double sel_join_size_estimate(uint64_t rows_r, uint64_t rows_s, uint64_t distinct_r, uint64_t distinct_s) {
    const uint64_t v = std::max(distinct_r, distinct_s);
    return v == 0 ? 0.0 : (double)rows_r * (double)rows_s / (double)v;
}

extern "C" sel_status sel_pushdown(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                                   const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                                   int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* out_count) {
    const char* who = "sel_pushdown";
    if (!ctx || !out_count) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    sel_status s = ctx->counts.ensure(64, "count buffer");
    if (s != SEL_OK) return s;
    unsigned long long* d_total = static_cast<unsigned long long*>(ctx->counts.p);
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(ctx->err.p, 0, 4, ctx->stream));
    s = pushdown_enqueue(ctx, pred, table, proj_cols, n_proj, dev_out_cols, dev_out_rowids, max_rows, d_total, who);
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_pinned, d_total, 8, cudaMemcpyDeviceToHost, ctx->stream));
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, ctx->err.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_and_check(ctx, who);
    if (s != SEL_OK) return s;
    if (*ctx->h_err) {
        set_error("%s: a look-back wait timed out", who);
        return SEL_ERR_TIMEOUT;
    }
    *out_count = ctx->h_pinned[0];
    if (*out_count > max_rows) {
        set_error("%s: count %llu > max_rows %llu", who, (unsigned long long)*out_count,
                  (unsigned long long)max_rows);
        return SEL_ERR_TOO_LARGE;
    }
    return SEL_OK;
}

// ---------------------------------------------------------------------------
// batched probes
// ---------------------------------------------------------------------------

namespace sel {

static std::string table_key(const sel_table* t) {
    std::string k = std::to_string(t->n_rows) + ":";
    for (int32_t c = 0; c < t->n_cols; ++c) {
        char b[48];
        std::snprintf(b, sizeof(b), "%p/%d,", t->cols[c].data, t->cols[c].type);
        k += b;
    }
    return k;
}

// One launch of the plan's probes on the given kernel (0 interpreter, 1 bucket).
static sel_status plan_launch(sel_batch_plan* p, int kernel, const Shape& sh, int* n_launches,
                              void* counts = nullptr) {
    unsigned long long* d_counts = static_cast<unsigned long long*>(counts ? counts : p->d_counts);
    if (kernel == 1) return run_bucket(p->ctx, p, sh, d_counts, n_launches);
    return run_scan(p->ctx, static_cast<const uint8_t*>(p->d_blob), p->blob_bytes, p->instr_off, p->pool_off,
                    p->n_progs, p->tables, d_counts, sh, n_launches);
}

static sel_status plan_time(sel_batch_plan* p, int kernel, const Shape& sh, int reps, float* ms) {
    sel_ctx* ctx = p->ctx;
    cudaEvent_t e0, e1;
    SEL_CUDA("cudaEventCreate", cudaEventCreate(&e0));
    SEL_CUDA("cudaEventCreate", cudaEventCreate(&e1));
    float best = 1e30f;
    sel_status s = SEL_OK;
    for (int r = 0; r <= reps && s == SEL_OK; ++r) {
        cudaEventRecord(e0, ctx->stream);
        cudaMemsetAsync(p->d_counts, 0, (size_t)p->n * 8, ctx->stream);
        s = plan_launch(p, kernel, sh, nullptr);
        cudaEventRecord(e1, ctx->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) s = cuda_fail("autotune", e);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0 || reps == 0) best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

// Captures the plan's launch (zeroing the counts, then the kernel) into a
// graph whose kernel writes the counts to `counts` (the plan's own buffer, or
// a caller's device buffer of n u64).
static sel_status plan_capture(sel_batch_plan* p, void* counts, cudaGraphExec_t* out) {
    sel_ctx* ctx = p->ctx;
    cudaStream_t cs;
    SEL_CUDA("cudaStreamCreate", cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    const uint64_t saved_launches = ctx->launches;
    ctx->stream = cs;
    cudaGraph_t g = nullptr;
    sel_status s = SEL_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) s = cuda_fail("cudaStreamBeginCapture", e);
    int nl = 0;
    if (s == SEL_OK) {
        cudaMemsetAsync(counts, 0, (size_t)p->n * 8, cs);
        if (p->parts.empty()) {
            s = plan_launch(p, p->kernel, p->shape, &nl, counts);
        } else {
            for (sel_batch_plan* q : p->parts) {   // every part adds its probes' counts to the same buffer
                int nq = 0;
                if (s == SEL_OK) s = plan_launch(q, q->kernel, q->shape, &nq, counts);
                nl += nq;
            }
        }
        e = cudaStreamEndCapture(cs, &g);
        if (s == SEL_OK && e != cudaSuccess) s = cuda_fail("cudaStreamEndCapture", e);
    }
    ctx->stream = saved;
    ctx->launches = saved_launches;
    if (s == SEL_OK) {
        e = cudaGraphInstantiate(out, g, 0);
        if (e != cudaSuccess) s = cuda_fail("cudaGraphInstantiate", e);
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    p->launches_per_run = nl;
    return s;
}

}  // namespace sel

namespace sel {

// Probes of one table a plan launch takes: one quad of the bucket kernel.
// Larger groups leave too little shared memory for the stages (measured on
// config 2: 512 probes in one launch counted 6x slower per probe than 256).
constexpr int kPlanPartProbes = 256;

// A plan of preds[0..n) over tables[0..n) whose counts go to outs[i] (null:
// i) of a counts buffer of n_total entries.
static sel_status plan_create(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                              int32_t n, int32_t autotune, const int32_t* omap, int32_t n_total,
                              sel_batch_plan** out) {
    const char* who = "sel_batch_plan_create";
    *out = nullptr;
    // group predicates by table (same data pointers and row count)
    std::vector<std::string> keys;
    std::map<std::string, int> gid;
    std::vector<int> group(n);
    std::vector<const sel_table*> gtab;
    for (int32_t i = 0; i < n; ++i) {
        const std::string k = table_key(tables[i]);
        auto it = gid.find(k);
        if (it == gid.end()) {
            it = gid.emplace(k, (int)gtab.size()).first;
            gtab.push_back(tables[i]);
        }
        group[i] = it->second;
    }
    std::unique_ptr<sel_batch_plan> p(new sel_batch_plan());
    p->ctx = ctx;
    p->n = n_total;
    std::vector<const Program*> progs;
    std::vector<std::vector<int32_t>> maps;
    std::vector<uint32_t> outs;
    std::vector<BkTableIn> bk_in(gtab.size());
    for (size_t g = 0; g < gtab.size(); ++g) {
        std::vector<int32_t> cols;
        for (int32_t i = 0; i < n; ++i)
            if (group[i] == (int)g)
                for (int32_t c : preds[i]->prog.slot_col) cols.push_back(c);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        if ((int)cols.size() > kMaxSlots) {
            set_error("%s: predicates on one table read more than 16 distinct columns", who);
            return SEL_ERR_UNSUPPORTED;
        }
        TableArg ta;
        fill_table_arg(ta, cols, gtab[g]);
        ta.prog_begin = (uint32_t)progs.size();
        for (int32_t i = 0; i < n; ++i) {
            if (group[i] != (int)g) continue;
            std::vector<int32_t> m;
            for (int32_t c : preds[i]->prog.slot_col)
                m.push_back((int32_t)(std::lower_bound(cols.begin(), cols.end(), c) - cols.begin()));
            const uint32_t o = omap ? (uint32_t)omap[i] : (uint32_t)i;
            progs.push_back(&preds[i]->prog);
            maps.push_back(m);
            outs.push_back(o);
            bk_in[g].progs.push_back(&preds[i]->prog);
            bk_in[g].slot_maps.push_back(m);
            bk_in[g].outs.push_back(o);
        }
        ta.prog_end = (uint32_t)progs.size();
        for (uint32_t j = 0; j < ta.n_slots; ++j) bk_in[g].slot_width.push_back(ta.width[j]);
        p->tables.push_back(ta);
    }
    p->n_progs = (uint32_t)progs.size();
    std::vector<uint8_t> blob;
    build_blob(progs, maps, blob, p->instr_off, p->pool_off, outs);
    p->blob_bytes = (uint32_t)blob.size();
    SEL_CUDA("cudaMalloc", dev_alloc(&p->d_blob, blob.size()));
    SEL_CUDA("cudaMemcpy", cudaMemcpy(p->d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice));
    SEL_CUDA("cudaMalloc", dev_alloc(&p->d_counts, (size_t)n_total * 8));
    uint32_t max_rb = 0;
    for (auto& t : p->tables) max_rb = std::max(max_rb, t.row_bytes);
    // the column-bucket form, when the probes fit it (bucket.h)
    bool bucket_ok = false;
    if (ctx->batch_kernel != 1) {
        BucketPlan bp;
        std::string why;
        const sel_status bs = build_bucket_plan(bk_in, &bp, &why);
        if (bs == SEL_OK) {
            BkHeader hdr;
            std::memcpy(&hdr, bp.blob.data(), sizeof(hdr));
            p->bk_blob_bytes = (uint32_t)bp.blob.size();
            p->bk_n_out = bp.n_out;
            p->bk_gb_slots = hdr.gb_slots;
            p->bk_gb_quad = hdr.gb_quad;
            SEL_CUDA("cudaMalloc", dev_alloc(&p->d_bk_blob, bp.blob.size()));
            SEL_CUDA("cudaMemcpy", cudaMemcpy(p->d_bk_blob, bp.blob.data(), bp.blob.size(), cudaMemcpyHostToDevice));
            bucket_ok = true;
        } else if (ctx->batch_kernel == 2) {
            set_error("%s: %s", who, why.c_str());
            return bs;
        }
    }
    // default shape, then the autotuner's candidates (stage size, stages, CTAs
    // per SM, consumer warps, chunks per instruction pass)
    // (stage_kb 0: the largest tile whose stages fit in shared memory); the
    // default shape is the single-probe count's, with the context's overrides
    Shape best = single_shape(ctx, max_rb);
    int best_kernel = 0;
    // 15 consumer warps (11 when a table takes the quad form: its passes hold
    // more registers), one chunk a pass, 3 stages that fill shared memory, or
    // the context's overrides (measured on config 2's 5 probes and config 5's
    // 256)
    Shape bucket_default;
    bucket_default.stages = ctx->shape.stages > 0 ? ctx->shape.stages : 3;
    bucket_default.ctas_per_sm = 1;
    bucket_default.tile_rows = ctx->shape.tile_rows > 0 ? ctx->shape.tile_rows : kMaxTileRows;
    bucket_default.auto_tile = ctx->shape.tile_rows <= 0;
    bucket_default.warps = p->bk_gb_quad ? 11 : 15;
    bucket_default.group = 1;
    if (bucket_variant_ok(ctx->shape.warps, ctx->shape.group > 0 ? ctx->shape.group : 1)) {
        bucket_default.warps = ctx->shape.warps;
        bucket_default.group = ctx->shape.group > 0 ? ctx->shape.group : 1;
    }
    if (bucket_ok) {   // the first shape that fits (tables too large for any: the interpreter)
        const int fallback[][3] = {{11, 1, 3}, {8, 1, 3}, {8, 1, 2}};   // warps, chunks per pass, stages
        sel_status rs = SEL_ERR_UNSUPPORTED;
        for (int c = -1; c < 3 && rs != SEL_OK; ++c) {
            Shape sh = bucket_default;
            if (c >= 0) {
                sh.warps = fallback[c][0];
                sh.group = fallback[c][1];
                sh.stages = fallback[c][2];
            }
            ScanArgs a;
            size_t smem = 0;
            rs = resolve_bucket(ctx, p.get(), p->tables, sh, &a, &smem, nullptr);
            if (rs == SEL_OK) bucket_default = sh;
        }
        if (rs == SEL_OK) {
            best = bucket_default;
            best_kernel = 1;
        } else if (ctx->batch_kernel == 2) {
            return rs;
        } else {
            bucket_ok = false;
        }
    }
    float best_ms = 0.f;
    if (autotune && bucket_ok) {
        struct BCand { int stage_kb, stages, warps, group; };
        const BCand bc[] = {{0, 3, 16, 1}, {0, 3, 15, 1}, {0, 3, 15, 2}, {0, 3, 11, 1}, {0, 3, 16, 2},
                            {0, 2, 15, 1}, {0, 4, 15, 2}, {0, 3, 8, 2}, {0, 3, 8, 1}};
        best_ms = 1e30f;
        for (const BCand& c : bc) {
            Shape sh = bucket_default;
            sh.stages = c.stages;
            sh.tile_rows = c.stage_kb > 0 ? default_tile_rows(max_rb, c.stage_kb * 1024) : kMaxTileRows;
            sh.warps = c.warps;
            sh.group = c.group;
            float ms = 0;
            sel_status st = plan_time(p.get(), 1, sh, 2, &ms);
            if (st == SEL_ERR_UNSUPPORTED) continue;
            if (st != SEL_OK) return st;
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
                best_kernel = 1;
            }
        }
    }
    if (autotune && ctx->batch_kernel != 2) {
        struct Cand { int stage_kb, stages, ctas, warps, group; };
        const Cand cands[] = {{0, 3, 1, 15, 3},  {0, 3, 1, 16, 2},  {64, 3, 1, 16, 2}, {48, 4, 1, 16, 2}, {96, 2, 1, 16, 2},
                              {64, 3, 1, 16, 1}, {48, 4, 1, 16, 1}, {32, 3, 2, 8, 2},  {24, 4, 2, 8, 2},
                              {32, 3, 2, 8, 1},  {24, 4, 2, 8, 1},  {16, 4, 3, 8, 1},  {64, 3, 1, 8, 4},
                              {48, 4, 1, 8, 4}};
        if (!bucket_ok) best_ms = 1e30f;
        bool first = true;
        for (const Cand& c : cands) {
            Shape sh;
            sh.stages = c.stages;
            sh.ctas_per_sm = c.ctas;
            sh.tile_rows = c.stage_kb > 0 ? default_tile_rows(max_rb, c.stage_kb * 1024) : kMaxTileRows;
            sh.auto_tile = true;
            sh.warps = c.warps;
            sh.group = c.group;
            float ms = 0;
            sel_status s = plan_time(p.get(), 0, sh, first && bucket_ok ? 0 : 2, &ms);
            if (s == SEL_ERR_UNSUPPORTED) continue;
            if (s != SEL_OK) return s;
            // the interpreter's other shapes are tried only when its default
            // comes within 25 % of the bucket kernel's best
            if (first && bucket_ok && ms > 1.25f * best_ms) break;
            first = false;
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
                best_kernel = 0;
            }
        }
    }
    p->kernel = best_kernel;
    if (best_kernel == 1) {   // the shape the plan's launches use (reported by sel_batch_plan_info)
        ScanArgs a;
        size_t smem = 0;
        const sel_status rs = resolve_bucket(ctx, p.get(), p->tables, best, &a, &smem, &p->shape);
        if (rs != SEL_OK) return rs;
    } else {   // the shape the plan's launches use (reported by sel_batch_plan_info)
        const sel_status rs = resolve_shape(ctx, p->blob_bytes, p->n_progs, p->tables, best, &p->shape);
        if (rs != SEL_OK) return rs;
    }
    p->ms = best_ms;
    sel_status s = plan_capture(p.get(), p->d_counts, &p->graph);
    if (s != SEL_OK) return s;
    *out = p.release();
    return SEL_OK;
}

}  // namespace sel

extern "C" sel_status sel_batch_plan_create(sel_ctx* ctx, const sel_pred* const* preds,
                                            const sel_table* const* tables, int32_t n, int32_t autotune,
                                            sel_batch_plan** out) {
    const char* who = "sel_batch_plan_create";
    if (!ctx || !out || n <= 0 || !preds || !tables) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int32_t i = 0; i < n; ++i) {
        sel_status s = check_pred_on_table(preds[i], tables[i], who);
        if (s != SEL_OK) return s;
    }
    // probes of each table, in order; part j takes the j-th kPlanPartProbes of every table
    std::map<std::string, std::vector<int32_t>> by_table;
    size_t most = 0;
    for (int32_t i = 0; i < n; ++i) {
        std::vector<int32_t>& v = by_table[table_key(tables[i])];
        v.push_back(i);
        most = std::max(most, v.size());
    }
    if (most <= (size_t)kPlanPartProbes) return plan_create(ctx, preds, tables, n, autotune, nullptr, n, out);
    std::unique_ptr<sel_batch_plan> p(new sel_batch_plan());
    p->ctx = ctx;
    p->n = n;
    const size_t n_parts = (most + kPlanPartProbes - 1) / kPlanPartProbes;
    for (size_t j = 0; j < n_parts; ++j) {
        std::vector<int32_t> idx;
        for (auto& kv : by_table)
            for (size_t k = j * kPlanPartProbes; k < std::min(kv.second.size(), (j + 1) * kPlanPartProbes); ++k)
                idx.push_back(kv.second[k]);
        std::sort(idx.begin(), idx.end());
        std::vector<const sel_pred*> pp;
        std::vector<const sel_table*> tt;
        for (int32_t i : idx) {
            pp.push_back(preds[i]);
            tt.push_back(tables[i]);
        }
        sel_batch_plan* q = nullptr;
        sel_status s = plan_create(ctx, pp.data(), tt.data(), (int32_t)idx.size(), autotune, idx.data(), n, &q);
        if (s != SEL_OK) return s;
        p->parts.push_back(q);
        p->ms += q->ms;
    }
    p->kernel = p->parts[0]->kernel;   // reported by sel_batch_plan_kernel / _info / _variant
    p->shape = p->parts[0]->shape;
    SEL_CUDA("cudaMalloc", dev_alloc(&p->d_counts, (size_t)n * 8));
    sel_status s = plan_capture(p.get(), p->d_counts, &p->graph);
    if (s != SEL_OK) return s;
    *out = p.release();
    return SEL_OK;
}

extern "C" sel_status sel_batch_plan_run(sel_batch_plan* p, uint64_t* dev_out_counts, uint64_t* host_out_counts) {
    if (!p || (!dev_out_counts && !host_out_counts)) {
        set_error("sel_batch_plan_run: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    sel_ctx* ctx = p->ctx;
    if (dev_out_counts) {
        // a graph whose kernel writes straight into the caller's buffer,
        // captured on the first run with that buffer (a few are kept)
        cudaGraphExec_t g = nullptr;
        for (auto& kv : p->out_graphs)
            if (kv.first == dev_out_counts) g = kv.second;
        if (!g) {
            if (p->out_graphs.size() >= 4) {
                cudaGraphExecDestroy(p->out_graphs.front().second);
                p->out_graphs.erase(p->out_graphs.begin());
            }
            sel_status s = plan_capture(p, dev_out_counts, &g);
            if (s != SEL_OK) return s;
            p->out_graphs.emplace_back(dev_out_counts, g);
        }
        SEL_CUDA("cudaGraphLaunch", cudaGraphLaunch(g, ctx->stream));
        ctx->launches += (uint64_t)p->launches_per_run;
        return SEL_OK;
    }
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(ctx->err.p, 0, 4, ctx->stream));
    SEL_CUDA("cudaGraphLaunch", cudaGraphLaunch(p->graph, ctx->stream));
    ctx->launches += (uint64_t)p->launches_per_run;
    const size_t bytes = (size_t)p->n * 8;
    sel_status s = ensure_host(ctx, (size_t)p->n);
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_pinned, p->d_counts, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, ctx->err.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    s = sync_and_check(ctx, "sel_batch_plan_run");
    if (s != SEL_OK) return s;
    if (*ctx->h_err) {
        set_error("sel_batch_plan_run: a device wait timed out");
        return SEL_ERR_TIMEOUT;
    }
    std::memcpy(host_out_counts, ctx->h_pinned, bytes);
    return SEL_OK;
}

extern "C" sel_status sel_batch_plan_info(const sel_batch_plan* p, int32_t* tile_rows, int32_t* stages,
                                          int32_t* ctas_per_sm, float* ms) {
    if (!p) {
        set_error("sel_batch_plan_info: plan is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    if (tile_rows) *tile_rows = p->shape.tile_rows;
    if (stages) *stages = p->shape.stages;
    if (ctas_per_sm) *ctas_per_sm = p->shape.ctas_per_sm;
    if (ms) *ms = p->ms;
    return SEL_OK;
}

extern "C" sel_status sel_batch_plan_variant(const sel_batch_plan* p, int32_t* consumer_warps,
                                             int32_t* chunks_per_pass) {
    if (!p) {
        set_error("sel_batch_plan_variant: plan is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    if (consumer_warps) *consumer_warps = p->shape.warps;
    if (chunks_per_pass) *chunks_per_pass = p->shape.group;
    return SEL_OK;
}

extern "C" sel_status sel_batch_plan_kernel(const sel_batch_plan* p, int32_t* kernel) {
    if (!p || !kernel) {
        set_error("sel_batch_plan_kernel: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    *kernel = p->kernel;
    return SEL_OK;
}

extern "C" sel_status sel_ctx_set_batch_kernel(sel_ctx* c, int32_t mode) {
    if (!c || mode < 0 || mode > 2) {
        set_error("sel_ctx_set_batch_kernel: mode must be 0, 1 or 2");
        return SEL_ERR_INVALID_ARG;
    }
    c->batch_kernel = mode;
    for (auto& kv : c->plans) sel_batch_plan_free(kv.second);   // cached plans were made under the old mode
    c->plans.clear();
    return SEL_OK;
}

extern "C" void sel_batch_plan_free(sel_batch_plan* p) { delete p; }

static sel_status batch_cached(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                               int32_t n, uint64_t* dev_out, uint64_t* host_out) {
    std::string key;
    for (int32_t i = 0; i < n; ++i) {
        if (!preds[i] || !tables[i]) {
            set_error("sel_count_batch: null predicate or table %d", i);
            return SEL_ERR_INVALID_ARG;
        }
        key += std::to_string(preds[i]->content) + "@" + table_key(tables[i]) + ";";
    }
    auto it = ctx->plans.find(key);
    if (it == ctx->plans.end()) {
        sel_batch_plan* p = nullptr;
        sel_status s = sel_batch_plan_create(ctx, preds, tables, n, 1, &p);
        if (s != SEL_OK) return s;
        if (ctx->plans.size() > 64) {   // bounded cache
            for (auto& kv : ctx->plans) sel_batch_plan_free(kv.second);
            ctx->plans.clear();
        }
        it = ctx->plans.emplace(key, p).first;
    }
    return sel_batch_plan_run(it->second, dev_out, host_out);
}

extern "C" sel_status sel_count_batch(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                                      int32_t n, uint64_t* out_counts) {
    if (!ctx || !preds || !tables || n <= 0 || !out_counts) {
        set_error("sel_count_batch: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    return batch_cached(ctx, preds, tables, n, nullptr, out_counts);
}

extern "C" sel_status sel_count_batch_async(sel_ctx* ctx, const sel_pred* const* preds,
                                            const sel_table* const* tables, int32_t n, uint64_t* dev_out_counts) {
    if (!ctx || !preds || !tables || n <= 0 || !dev_out_counts) {
        set_error("sel_count_batch_async: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    return batch_cached(ctx, preds, tables, n, dev_out_counts, nullptr);
}

extern "C" sel_status sel_ctx_synchronize(sel_ctx* ctx) {
    if (!ctx) {
        set_error("sel_ctx_synchronize: ctx is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    SEL_CUDA("cudaMemcpyAsync", cudaMemcpyAsync(ctx->h_err, ctx->err.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    sel_status s = sync_and_check(ctx, "sel_ctx_synchronize");
    if (s != SEL_OK) return s;
    SEL_CUDA("cudaMemsetAsync", cudaMemsetAsync(ctx->err.p, 0, 4, ctx->stream));
    if (*ctx->h_err) {
        set_error("sel_ctx_synchronize: a device wait timed out since the last check");
        return SEL_ERR_TIMEOUT;
    }
    return SEL_OK;
}
