// pushdown_noalloc.cu -- sel_pushdown_noalloc: the push-down for callers that
// cannot allocate device memory.
//
// The regular push-down keeps its scratch (one status word per tile for the
// look-back, a tile counter, the uploaded program, an error flag) in
// buffers its context allocates with cudaMalloc.  This entry point runs the
// same kernel with all of that scratch in one file-scope __device__ array of
// fixed size instead, so that it makes no cudaMalloc / cudaFree call and
// needs no context.  The caller passes the inputs and every output.
//
// The compiled program reaches the array through kernel parameters: a small
// copy kernel takes up to 16 KiB of the program by value per launch, so the
// call reads no host buffer after it returns (a cudaMemcpyAsync from pageable
// host memory could read it later, or wait for the GPU).
#include <cstring>
#include <mutex>

#include "internal.h"

namespace sel {
namespace {

constexpr size_t kNaBytes = size_t(4) << 20;          // the whole array: 4 MiB per device
constexpr size_t kNaBlobBytes = size_t(64) << 10;     // [0, 64 KiB): program blob
constexpr size_t kNaMiscOff = kNaBlobBytes;           // tile counter (4 B)
constexpr size_t kNaStatusOff = kNaBlobBytes + 256;   // [.., 4 MiB): one 8-byte status word per tile
constexpr size_t kNaMaxTiles = (kNaBytes - kNaStatusOff) / 8;

// The scratch array.  Every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device

// Device address of the array on the current device (first call per device
// looks it up; in host code the array's name is not a device address).
sel_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("sel_pushdown_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("sel_pushdown_noalloc: device %d out of range", dev);
        return SEL_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("sel_pushdown_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return SEL_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return SEL_OK;
}

// Lays out ProgDesc | Instr[] | pool for one program into dst (no allocation).
bool blob_into(const Program& p, uint8_t* dst, size_t cap, uint32_t* bytes, uint32_t* instr_off,
               uint32_t* pool_off) {
    auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
    const size_t io = up16(sizeof(ProgDesc));
    const size_t po = up16(io + p.instrs.size() * sizeof(Instr));
    const size_t total = up16(po + p.pool.size());
    if (total > cap) return false;
    std::memset(dst, 0, total);
    const ProgDesc pd{0u, (uint32_t)p.instrs.size(), 0u, 0u};
    std::memcpy(dst, &pd, sizeof(pd));
    if (!p.instrs.empty()) std::memcpy(dst + io, p.instrs.data(), p.instrs.size() * sizeof(Instr));
    if (!p.pool.empty()) std::memcpy(dst + po, p.pool.data(), p.pool.size());
    *bytes = (uint32_t)total;
    *instr_off = (uint32_t)io;
    *pool_off = (uint32_t)po;
    return true;
}

thread_local uint8_t t_blob[kNaBlobBytes];

// One piece of the program, passed by value to the copy kernel.
constexpr uint32_t kNaPieceBytes = 16u << 10;
struct BlobPiece {
    uint4* dst;
    uint32_t words;   // 16-byte words in this piece
    uint32_t pad;
    uint4 data[kNaPieceBytes / 16];
};

__global__ void __launch_bounds__(256) blob_piece_kernel(const __grid_constant__ BlobPiece p) {
    for (uint32_t i = threadIdx.x; i < p.words; i += blockDim.x) p.dst[i] = p.data[i];
}

// Enqueues the copy of the laid-out program (bytes, a multiple of 16) into dst.
cudaError_t upload_blob(uint8_t* dst, const uint8_t* src, uint32_t bytes, cudaStream_t st) {
    BlobPiece piece;
    for (uint32_t off = 0; off < bytes; off += kNaPieceBytes) {
        const uint32_t n = bytes - off < kNaPieceBytes ? bytes - off : kNaPieceBytes;
        piece.dst = reinterpret_cast<uint4*>(dst + off);
        piece.words = n / 16u;
        piece.pad = 0;
        std::memcpy(piece.data, src + off, n);
        blob_piece_kernel<<<1, 256, 0, st>>>(piece);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace sel

using namespace sel;

extern "C" sel_status sel_pushdown_noalloc(void* cuda_stream, const sel_pred* pred, const sel_table* table,
                                           const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                                           int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* dev_out_count,
                                           uint32_t* dev_out_error) {
    const char* who = "sel_pushdown_noalloc";
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (!pred || !table || !dev_out_count || !dev_out_error || n_proj < 0 || n_proj > kPdMaxProj ||
        (n_proj > 0 && (!proj_cols || !dev_out_cols)) || table->n_rows < 0 || table->n_cols < 0 ||
        (table->n_cols > 0 && !table->cols)) {
        set_error("%s: bad arguments", who);
        return SEL_ERR_INVALID_ARG;
    }
    const Program& prog = pred->prog;
    PushdownArgs a;
    std::memset(&a, 0, sizeof(a));
    uint32_t row_bytes = 0, tma = 1;
    for (size_t j = 0; j < prog.slot_col.size(); ++j) {
        const int c = prog.slot_col[j];
        if (c >= table->n_cols) {
            set_error("%s: predicate reads column %d, table has %d", who, c, table->n_cols);
            return SEL_ERR_INVALID_ARG;
        }
        if (table->cols[c].type != pred->col_types[c]) {
            set_error("%s: column %d has type %d, predicate was compiled for %d", who, c, table->cols[c].type,
                      pred->col_types[c]);
            return SEL_ERR_TYPE;
        }
        const uintptr_t p = reinterpret_cast<uintptr_t>(table->cols[c].data);
        if (table->n_rows > 0 && (!p || p % prog.slot_width[j])) {
            set_error("%s: column %d data pointer is null or not element-aligned", who, c);
            return SEL_ERR_INVALID_ARG;
        }
        if (p % 16) tma = 0;
        a.col[j] = reinterpret_cast<const uint8_t*>(table->cols[c].data);
        a.width[j] = prog.slot_width[j];
        row_bytes += prog.slot_width[j];
    }
    for (int32_t j = 0; j < n_proj; ++j) {
        const int c = proj_cols[j];
        if (c < 0 || c >= table->n_cols || table->cols[c].type < SEL_I32 || table->cols[c].type > SEL_DICT) {
            set_error("%s: projected column %d out of range or of unknown type", who, c);
            return SEL_ERR_INVALID_ARG;
        }
        const uint32_t w = table->cols[c].type == SEL_I64 ? 8u : 4u;
        const uintptr_t src = reinterpret_cast<uintptr_t>(table->cols[c].data);
        const uintptr_t dst = reinterpret_cast<uintptr_t>(dev_out_cols[j]);
        if ((table->n_rows > 0 && (!src || src % w)) || (max_rows > 0 && (!dst || dst % w))) {
            set_error("%s: projected column %d: null or misaligned source/output pointer", who, c);
            return SEL_ERR_INVALID_ARG;
        }
        a.proj_src[j] = reinterpret_cast<const uint8_t*>(table->cols[c].data);
        a.proj_dst[j] = static_cast<uint8_t*>(dev_out_cols[j]);
        a.proj_width[j] = w;
        a.proj_slot[j] = -1;
        for (size_t k = 0; k < prog.slot_col.size(); ++k)
            if (prog.slot_col[k] == c) a.proj_slot[j] = (int32_t)k;
    }
    if ((dev_out_rowids && reinterpret_cast<uintptr_t>(dev_out_rowids) % 8) ||
        reinterpret_cast<uintptr_t>(dev_out_count) % 8 || reinterpret_cast<uintptr_t>(dev_out_error) % 4) {
        set_error("%s: misaligned row id, count or error output", who);
        return SEL_ERR_INVALID_ARG;
    }
    uint32_t blob_bytes = 0;
    if (!blob_into(prog, t_blob, kNaBlobBytes, &blob_bytes, &a.instr_off, &a.pool_off)) {
        set_error("%s: compiled program larger than the %zu-byte program area", who, kNaBlobBytes);
        return SEL_ERR_UNSUPPORTED;
    }
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) {
        set_error("%s: %s", who, cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    // shared memory holds the program and the predicate columns of one tile
    // (outputs are not staged); 1 KiB is left for the kernel's static arrays
    a.tile_rows = 1024;
    auto up128 = [](size_t x) { return (x + 127) / 128 * 128; };
    while (a.tile_rows > (uint32_t)kChunkRows &&
           up128(blob_bytes) + up128((size_t)a.tile_rows * row_bytes) + 1024 > (size_t)max_smem)
        a.tile_rows -= kChunkRows;
    const int64_t n_tiles = (table->n_rows + a.tile_rows - 1) / a.tile_rows;
    if ((uint64_t)n_tiles > kNaMaxTiles) {
        set_error("%s: %lld rows need %lld tiles of %u rows; the fixed scratch holds at most %zu tiles (%llu rows)",
                  who, (long long)table->n_rows, (long long)n_tiles, a.tile_rows, kNaMaxTiles,
                  (unsigned long long)kNaMaxTiles * a.tile_rows);
        return SEL_ERR_UNSUPPORTED;
    }
    void* scratch = nullptr;
    sel_status s = scratch_address(&scratch);
    if (s != SEL_OK) return s;
    uint8_t* base = static_cast<uint8_t*>(scratch);
    uint32_t off = 0;
    for (size_t j = 0; j < prog.slot_col.size(); ++j) {
        a.slot_off[j] = off;
        off += a.tile_rows * a.width[j];
    }
    a.blob = base;
    a.blob_bytes = blob_bytes;
    a.n_instr = (uint32_t)prog.instrs.size();
    a.n_slots = (uint32_t)prog.slot_col.size();
    a.row_bytes = row_bytes;
    a.tma = tma;
    a.n_rows = table->n_rows;
    a.n_tiles = n_tiles;
    a.n_proj = (uint32_t)n_proj;
    a.rowids = reinterpret_cast<long long*>(dev_out_rowids);
    a.max_rows = max_rows;
    a.status = reinterpret_cast<unsigned long long*>(base + kNaStatusOff);
    a.tile_counter = reinterpret_cast<unsigned int*>(base + kNaMiscOff);
    a.err = reinterpret_cast<unsigned int*>(dev_out_error);
    a.total = reinterpret_cast<unsigned long long*>(dev_out_count);
    a.skip_publish_tile = -1;
    a.wait_ns = kWaitNs;
    if (pushdown_layout(a) + 1024 > (size_t)max_smem) {
        set_error("%s: tile does not fit in shared memory", who);
        return SEL_ERR_UNSUPPORTED;
    }
    // the array keeps the previous call's contents: clear what must start at zero
    if ((e = cudaMemsetAsync(base + kNaMiscOff, 0, 256 + (size_t)n_tiles * 8, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(dev_out_count, 0, 8, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(dev_out_error, 0, 4, st)) != cudaSuccess ||
        (e = upload_blob(base, t_blob, blob_bytes, st)) != cudaSuccess) {
        set_error("%s: %s", who, cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    e = launch_pushdown(a, st);
    if (e != cudaSuccess) {
        set_error("%s: launch: %s", who, cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    return SEL_OK;
}
