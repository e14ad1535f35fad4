// pushdown.cu -- selection push-down: the COUNT and the materialisation of
// sigma_P(pi_cols(R)) in one pass (§3.3 "Materialization": materialise while
// R's scan is still on the GPU; Algorithm 1, Execute with isSPD = true).
//
// One CTA per tile of tile_rows rows.  A CTA takes its tile id from an atomic
// counter (so tiles are started in order and the look-back below always
// waits on tiles that are already running), stages the predicate columns of
// its tile in shared memory (bulk copies for full aligned tiles), evaluates
// the program bit-sliced, and ranks its selected rows inside the tile.  The
// tile's output offset is found by decoupled look-back (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016): the tile
// publishes its aggregate, warp 0 walks back over predecessors' status words
// in windows of 32 until it meets an inclusive prefix, then publishes its own
// inclusive prefix.  Selected rows are gathered into shared memory in row
// order (projected columns that are predicate columns come from the staged
// tile, the others are read from HBM for selected rows only) and stored
// straight to their output positions.  Rows at output
// positions >= max_rows are not written; the count stays exact.
#include "kernels.h"
#include "lookback.cuh"
#include "rowmask.cuh"
#include "scan.cuh"

namespace sel {

__global__ void __launch_bounds__(kPdThreads, 6) pushdown_kernel(const __grid_constant__ PushdownArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned long long s_tile, s_excl;
    __shared__ uint32_t s_chunk_cnt[kPdThreads / 32 * 4];
    __shared__ uint32_t s_fail;
    __shared__ uint32_t s_slot_off[kMaxSlots];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, n_warps = blockDim.x >> 5;
    if (tid < kMaxSlots) s_slot_off[tid] = a.slot_off[tid];

    if (tid == 0) {
        s_tile = atomicAdd(a.tile_counter, 1u);
        s_fail = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    {
        uint4* dst = reinterpret_cast<uint4*>(smem + a.smem_prog_off);
        const uint4* src = reinterpret_cast<const uint4*>(a.blob);
        for (uint32_t i = tid; i < a.blob_bytes / 16u; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const long long t = static_cast<long long>(s_tile);
    const int64_t r0 = t * static_cast<int64_t>(a.tile_rows);
    const uint32_t valid = static_cast<uint32_t>((a.n_rows - r0 < (int64_t)a.tile_rows ? a.n_rows - r0 : (int64_t)a.tile_rows));
    uint8_t* st = smem + a.smem_stage_off;
    const bool bulk = a.tma && valid == a.tile_rows && a.row_bytes > 0;
    if (bulk) {
        if (tid == 0) {
            const uint64_t pol = policy_evict_first();
            mbar_arrive_expect_tx(&bar, a.tile_rows * a.row_bytes);
            for (uint32_t j = 0; j < a.n_slots; ++j)
                bulk_g2s(st + a.slot_off[j], a.col[j] + r0 * a.width[j], a.tile_rows * a.width[j], &bar, pol);
        }
        const bool ok = mbar_wait_bounded(&bar, 0);
        if (__syncthreads_or(!ok)) {
            // the copy did not land in time: report, drain (bounded) and leave a
            // published (invalid) prefix so that successors do not wait too
            if (tid == 0) {
                atomicOr(a.err, 1u);
                st_relaxed(&a.status[t], kFlagInc);
            }
            mbar_wait_bounded(&bar, 0);
            return;
        }
    } else {
        for (uint32_t j = 0; j < a.n_slots; ++j) {
            const uint32_t words = valid * a.width[j] / 4u;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(a.col[j] + r0 * a.width[j]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(st + a.slot_off[j]);
            for (uint32_t i = tid; i < words; i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
    }

    // --- evaluate: each warp handles chunks warp, warp + n_warps, ... ---
    const uint8_t* blob = smem + a.smem_prog_off;
    const Instr* ins = reinterpret_cast<const Instr*>(blob + a.instr_off);
    const uint8_t* pool = blob + a.pool_off;
    const uint32_t n_chunks = (valid + kChunkRows - 1) / kChunkRows;   // <= 4 per warp (tile_rows <= 4096)
    const uint32_t st_addr = smem_u32(st);
    uint32_t masks[4];
    uint32_t lane_pre[4];   // rank of the lane's first selected row inside its chunk (A and B halves packed)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        masks[q] = 0;
        lane_pre[q] = 0;
        const uint32_t ch = warp + q * n_warps;
        if (ch < n_chunks) {
            const uint32_t c0 = ch * kChunkRows;
            const uint32_t vm = (c0 + kChunkRows <= valid) ? 0xFFu : valid_mask(c0, lane, valid);
            const uint32_t m = eval_program(ins, a.n_instr, pool, st_addr, s_slot_off, c0, lane) & vm;
            masks[q] = m;
            // inclusive warp scan of (popc(A half) | popc(B half) << 16)
            const uint32_t mine = __popc(m & 0xFu) | (__popc(m >> 4) << 16);
            uint32_t x = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= static_cast<uint32_t>(o)) x += y;
            }
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, x, 31);
            const uint32_t ex = x - mine;
            // rows of half A come before rows of half B in the chunk
            lane_pre[q] = (ex & 0xFFFFu) | (((ex >> 16) + (tot & 0xFFFFu)) << 16);
            if (lane == 0) s_chunk_cnt[ch] = (tot & 0xFFFFu) + (tot >> 16);
        }
    }
    __syncthreads();
    // chunk prefix (chunks are in row order) and the tile aggregate
    __shared__ uint32_t s_chunk_pre[kPdThreads / 32 * 4];
    __shared__ uint32_t s_tile_cnt;
    if (tid == 0) {
        uint32_t acc = 0;
        for (uint32_t c = 0; c < n_chunks; ++c) {
            s_chunk_pre[c] = acc;
            acc += s_chunk_cnt[c];
        }
        s_tile_cnt = acc;
        if (t == 0) {
            s_excl = 0;
            if (t != a.skip_publish_tile) st_relaxed(&a.status[0], kFlagInc | acc);
        } else if (t != a.skip_publish_tile) {
            st_relaxed(&a.status[t], kFlagAgg | acc);
        }
    }
    __syncthreads();
    const uint32_t tile_cnt = s_tile_cnt;
    if (t > 0 && warp == 0) {
        unsigned long long excl;
        const bool ok = look_back(a, t, lane, &excl);
        if (lane == 0) {
            if (!ok) {
                atomicOr(a.err, 1u);
                s_fail = 1;
            }
            s_excl = excl;
            if (t != a.skip_publish_tile) st_relaxed(&a.status[t], kFlagInc | ((excl + tile_cnt) & kValMask));
        }
    }
    if (t == a.n_tiles - 1 && tid == 0 && t == 0) *a.total = tile_cnt;
    __syncthreads();
    const unsigned long long excl = s_excl;
    if (t == a.n_tiles - 1 && tid == 0 && t > 0) *a.total = excl + tile_cnt;
    if (tile_cnt == 0 || excl >= a.max_rows) return;

    if (s_fail) return;
    // --- write the selected rows straight to their output positions ---
    // Ranks follow row order, so a warp's stores for one mask bit land in a
    // short increasing run of output positions.
    const unsigned long long lim = a.max_rows;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t ch = warp + q * n_warps;
        if (ch >= n_chunks || masks[q] == 0) continue;
        const uint32_t c0 = ch * kChunkRows;
        const uint32_t m = masks[q];
        unsigned long long posA = excl + s_chunk_pre[ch] + (lane_pre[q] & 0xFFFFu);
        unsigned long long posB = excl + s_chunk_pre[ch] + (lane_pre[q] >> 16);
        for (uint32_t b = 0; b < 8; ++b) {
            if (!((m >> b) & 1u)) continue;
            const unsigned long long pos = (b < 4) ? posA++ : posB++;
            if (pos >= lim) continue;
            const uint32_t row = bit_row(c0, lane, b);
            for (uint32_t j = 0; j < a.n_proj; ++j) {
                const int32_t sl = a.proj_slot[j];
                if (a.proj_width[j] == 8) {
                    const uint64_t v = (sl >= 0)
                        ? *reinterpret_cast<const uint64_t*>(st + a.slot_off[sl] + static_cast<size_t>(row) * 8)
                        : __ldg(reinterpret_cast<const unsigned long long*>(a.proj_src[j]) + (r0 + row));
                    reinterpret_cast<uint64_t*>(a.proj_dst[j])[pos] = v;
                } else {
                    const uint32_t v = (sl >= 0)
                        ? *reinterpret_cast<const uint32_t*>(st + a.slot_off[sl] + static_cast<size_t>(row) * 4)
                        : __ldg(reinterpret_cast<const unsigned int*>(a.proj_src[j]) + (r0 + row));
                    reinterpret_cast<uint32_t*>(a.proj_dst[j])[pos] = v;
                }
            }
            if (a.rowids) a.rowids[pos] = static_cast<long long>(r0 + row);
        }
    }
}

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

size_t pushdown_layout(PushdownArgs& a) {
    a.smem_prog_off = 0;
    a.smem_stage_off = align_up(a.blob_bytes, 128u);
    a.smem_out_off = align_up(a.smem_stage_off + a.tile_rows * a.row_bytes, 128u);
    for (uint32_t j = 0; j <= a.n_proj; ++j) a.proj_stage_off[j] = 0;   // outputs are not staged
    a.smem_bytes = a.smem_out_off;
    return a.smem_bytes;
}

cudaError_t launch_pushdown(const PushdownArgs& a, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(pushdown_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(a.smem_bytes));
    if (e != cudaSuccess) return e;
    if (a.n_tiles <= 0) return cudaSuccess;
    pushdown_kernel<<<static_cast<unsigned>(a.n_tiles), kPdThreads, a.smem_bytes, st>>>(a);
    return cudaGetLastError();
}


// ===========================================================================
// Persistent push-down over super-tiles (the default path).
//
// The look-back unit is a super-tile: the largest multiple of the sub-tile
// (tile_rows rows) that is at most 32768 rows.  A CTA streams a super-tile
// through its shared-memory stages a sub-tile at a time and keeps only the row
// masks (1 bit per row, in row order) and the per-chunk counts of it, in one
// of three super-tile buffers.
//
//   producer warp   takes super-tile ids in increasing order from a global
//                   counter and bulk-copies each sub-tile's predicate columns
//                   into the next free stage (full[s]);
//   consumer warps  evaluate chunk groups of each sub-tile (ownership rotates
//                   from sub-tile to sub-tile), store each chunk's row masks
//                   (a byte per lane) into the super-tile's buffer and free
//                   the stage at once (empty[s]); after their part of super-tile j (evald[b])
//                   they go on with j+1 (once buffer b of j+1 is free);
//   look-back warp  sums super-tile j's chunk counts, finds its exclusive
//                   prefix by decoupled look-back, publishes the inclusive
//                   prefix and the chunk prefixes (done[b]) while the
//                   consumers already stream j+1 (the aggregate of j was
//                   published by the last consumer warp to finish it, so
//                   that no look-back waits behind another one);
//   writer warps    (kPdWriters) write the selected rows of each looked-back
//                   super-tile, reading the projected values of those rows
//                   from global memory, and release its buffer (freeb[b]).
// The write step ranks the super-tile's selected rows in row order and hands
// out batches of 32 consecutive ranks to the writer warps, kPdBatches at a
// time: a lane finds its rows from the chunk prefixes and the row-order mask
// words, all their loads are in flight together, and a batch's stores are
// contiguous.  The gathers' DRAM round trips never hold a consumer warp, so a
// stage is released as soon as it is evaluated and the stages keep streaming;
// up to kPdBufs super-tiles separate evaluation from writing.
// A CTA works on its super-tiles in increasing order, and what a super-tile
// waits for (free stages, a free buffer, the look-backs of the CTA's earlier
// super-tiles, the aggregates of smaller super-tiles) only involves smaller
// super-tiles, so the smallest unfinished super-tile always makes progress.
// Every wait is bounded; on a timeout the error flag is set, the CTA stops and
// the producer waits for its copies still in flight.
// ===========================================================================

namespace {

constexpr uint32_t kPdBufs = 4;      // super-tile buffers: evaluating j+1, look-back of j, writing j-1 and j-2
constexpr int kPdWriters = 2;        // writer warps: with 12 consumers, 16 warps a CTA and 128 registers a thread
constexpr uint32_t kPdBatches = 4;   // batches of 32 rows a writer lane has in flight
constexpr uint32_t kMaskWords = 8;   // 256 rows of a chunk, 32 per word, in row order

// Shared-memory layout (bytes from the dynamic base): a control block at
// fixed offsets (room for kPdMaxStages stages), so that every access to it is
// the shared base plus a constant, then the chunk prefixes and row masks of
// kPdBufs super-tiles of CH chunks.
constexpr uint32_t kPdMaxStages = 16;
namespace pdo {
constexpr uint32_t full = 0;
constexpr uint32_t empty = full + 8u * kPdMaxStages;
constexpr uint32_t evald = empty + 8u * kPdMaxStages;
constexpr uint32_t done = evald + 8u * kPdBufs;
constexpr uint32_t freeb = done + 8u * kPdBufs;
constexpr uint32_t tile = freeb + 8u * kPdBufs;
constexpr uint32_t st_id = tile + 8u * kPdMaxStages;
constexpr uint32_t excl = st_id + 8u * kPdBufs;
constexpr uint32_t nch = excl + 8u * kPdBufs;
constexpr uint32_t stot = nch + 4u * kPdBufs;
constexpr uint32_t claim = stot + 4u * kPdBufs;
constexpr uint32_t left = claim + 4u * kPdBufs;
constexpr uint32_t ngr = left + 4u * kPdBufs;
constexpr uint32_t evc = ngr + 4u * kPdBufs;
constexpr uint32_t cp = (evc + 4u * kPdBufs + 15u) & ~15u;
}  // namespace pdo
__host__ __device__ __forceinline__ uint32_t pd_mask_off(uint32_t CH) {
    return (pdo::cp + 4u * kPdBufs * CH + 15u) & ~15u;   // read as uint4
}
__host__ __device__ __forceinline__ uint32_t pd_ctrl_end(uint32_t CH) {
    return pd_mask_off(CH) + 4u * kPdBufs * CH * kMaskWords;
}

struct PdSmem {
    uint64_t *full, *empty;              // [S]
    uint64_t *evald, *done, *freeb;      // [kPdBufs]
    long long* tile;                     // [S] super-tile id of each stage (-1: no more work)
    long long* st_id;                    // [kPdBufs] super-tile id of each buffer (-1: end)
    unsigned long long* excl;            // [kPdBufs] exclusive prefix of each buffer's super-tile
    uint32_t* nch;                       // [kPdBufs] chunks of each buffer's super-tile that hold rows
    uint32_t* stot;                      // [kPdBufs] selected rows of each buffer's super-tile
    uint32_t* claim;                     // [kPdBufs] generation << 20 | next write group to hand out
    uint32_t* left;                      // [kPdBufs] write groups not yet finished
    uint32_t* ngr;                       // [kPdBufs] write groups of the buffer's super-tile
    uint32_t* evc;                       // [kPdBufs] consumer warps done with the buffer, over all its uses
    uint32_t* cp;                        // [kPdBufs][ch] chunk prefixes
    uint32_t* mask;                      // [kPdBufs][ch][kMaskWords] row masks (lane bytes, then row order)
    uint32_t ch;                         // chunks of a super-tile (super_rows / 256)
};

__device__ __forceinline__ PdSmem pd_smem(uint8_t* smem, uint32_t CH) {
    PdSmem m;
    m.ch = CH;
    m.full = reinterpret_cast<uint64_t*>(smem + pdo::full);
    m.empty = reinterpret_cast<uint64_t*>(smem + pdo::empty);
    m.evald = reinterpret_cast<uint64_t*>(smem + pdo::evald);
    m.done = reinterpret_cast<uint64_t*>(smem + pdo::done);
    m.freeb = reinterpret_cast<uint64_t*>(smem + pdo::freeb);
    m.tile = reinterpret_cast<long long*>(smem + pdo::tile);
    m.st_id = reinterpret_cast<long long*>(smem + pdo::st_id);
    m.excl = reinterpret_cast<unsigned long long*>(smem + pdo::excl);
    m.nch = reinterpret_cast<uint32_t*>(smem + pdo::nch);
    m.stot = reinterpret_cast<uint32_t*>(smem + pdo::stot);
    m.claim = reinterpret_cast<uint32_t*>(smem + pdo::claim);
    m.left = reinterpret_cast<uint32_t*>(smem + pdo::left);
    m.ngr = reinterpret_cast<uint32_t*>(smem + pdo::ngr);
    m.evc = reinterpret_cast<uint32_t*>(smem + pdo::evc);
    m.cp = reinterpret_cast<uint32_t*>(smem + pdo::cp);
    m.mask = reinterpret_cast<uint32_t*>(smem + pd_mask_off(CH));
    return m;
}

// Bounded wait by the whole warp; the warp goes on only if every lane saw the
// phase complete.  Every lane waits itself: a warp whose lane 0 waits alone
// while the other lanes park at a shuffle resumes much later after the phase
// completes (measured: the count-like loop of this kernel ran 1.7x slower).
// sleep_ns > 0: the waiters sleep between tries (waits off the critical path).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint32_t lane, uint32_t sleep_ns = 0) {
    (void)lane;
    const bool ok = sleep_ns ? mbar_wait_bounded_idle(bar, parity, sleep_ns) : mbar_wait_bounded(bar, parity);
    return __all_sync(0xFFFFFFFFu, ok);
}

// The same, but it also gives up (false) as soon as another warp of the CTA
// has flagged a failure: a wait on a role that stopped would otherwise last
// its full bound.  The sleep between tries doubles from sleep_ns up to
// max_sleep_ns: an idle writer would otherwise take issue slots from the
// consumers all through a scan that selects few rows.
__device__ __forceinline__ bool warp_wait_live(uint64_t* bar, uint32_t parity, const uint32_t* s_fail,
                                               uint32_t sleep_ns, uint32_t max_sleep_ns) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const unsigned long long t0 = global_ns();
        uint32_t ns = sleep_ns;
        while (true) {
            __nanosleep(ns);
            ns = ns * 2u < max_sleep_ns ? ns * 2u : max_sleep_ns;
            if (mbar_try_wait(bar, parity)) {
                ok = true;
                break;
            }
            if (*reinterpret_cast<const volatile uint32_t*>(s_fail) || global_ns() - t0 > kWaitNs) break;
        }
    }
    return __all_sync(0xFFFFFFFFu, ok);
}

__device__ __forceinline__ void fail_flag(const PushdownArgs& a, uint32_t* s_fail) {
    atomicOr(a.err, 1u);
    atomicOr(s_fail, 1u);
}

__device__ __forceinline__ bool volatile_flag(const uint32_t* f) { return *reinterpret_cast<const volatile uint32_t*>(f) != 0; }

// A chunk's row masks are first stored by the consumers as one byte per lane
// and turned into 8 row-order words by the look-back warp before the writers
// read them (rowmask.cuh).

// Row of rank r among the selected rows of the super-tile in buffer b.  lo:
// on entry a chunk whose prefix is <= r (0 always is), on return r's chunk,
// the last one whose prefix is <= r (cp[0] = 0).  The search gallops forward
// from lo and then halves: the ranks of a write group are consecutive, so
// starting from the previous rank's chunk takes a step or two where chunks
// hold many selected rows, and O(log distance) otherwise.
__device__ __forceinline__ int64_t rank_row(const PdSmem& sm, uint32_t b, int64_t R0, uint32_t r, uint32_t& lo) {
    const uint32_t nch = sm.nch[b];
    const uint32_t* cp = sm.cp + b * sm.ch;
    const uint32_t* mw = sm.mask + b * sm.ch * kMaskWords;
    uint32_t step = 1u;
    while (lo + step < nch && cp[lo + step] <= r) {
        lo += step;
        step <<= 1;
    }
    uint32_t hi = lo + step < nch ? lo + step : nch;   // cp[hi] > r, or hi = nch
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cp[mid] <= r) lo = mid;
        else hi = mid;
    }
    uint32_t o = r - cp[lo];
    const uint4* w4 = reinterpret_cast<const uint4*>(mw + lo * kMaskWords);
    const uint4 x = w4[0], y = w4[1];
    const uint32_t wv[kMaskWords] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    uint32_t word = 0, wbase = 0;
    bool found = false;
#pragma unroll
    for (uint32_t k = 0; k < kMaskWords; ++k) {
        const uint32_t c = __popc(wv[k]);
        if (!found) {
            if (o < c) {
                found = true;
                word = wv[k];
                wbase = 32u * k;
            } else {
                o -= c;
            }
        }
    }
    return R0 + static_cast<int64_t>(lo) * kChunkRows + wbase + select_bit(word, o);
}

// Writes group g of the selected rows of the super-tile in buffer b (first
// row R0): ranks g * 32 * kPdBatches .. + 32 * kPdBatches - 1 below n, to
// output positions excl + rank.  Every load of the group is issued before its
// first store.
__device__ __forceinline__ void scatter_group(const PushdownArgs& a, const PdSmem& sm, uint32_t b, int64_t R0,
                                              unsigned long long excl, uint32_t n, uint32_t g, uint32_t lane) {
    constexpr uint32_t K = kPdBatches;
    const uint32_t r0 = g * 32u * K;
    int64_t row[K];
    bool act[K];
    uint32_t lo = 0;   // the chunk of the lane's previous rank (the ranks increase)
#pragma unroll
    for (uint32_t k = 0; k < K; ++k) {
        const uint32_t r = r0 + 32u * k + lane;
        act[k] = r < n;
        row[k] = act[k] ? rank_row(sm, b, R0, r, lo) : 0;
    }
    for (uint32_t j0 = 0; j0 < a.n_proj; j0 += 4) {
        unsigned long long v[4][K];
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {   // all loads first: they are in flight together
            const uint32_t j = j0 + q;
#pragma unroll
            for (uint32_t k = 0; k < K; ++k) {
                v[q][k] = 0;
                if (act[k] && j < a.n_proj)
                    v[q][k] = a.proj_width[j] == 8
                                  ? __ldg(reinterpret_cast<const unsigned long long*>(a.proj_src[j]) + row[k])
                                  : __ldg(reinterpret_cast<const unsigned int*>(a.proj_src[j]) + row[k]);
            }
        }
#pragma unroll
        for (uint32_t q = 0; q < 4; ++q) {
            const uint32_t j = j0 + q;
            if (j >= a.n_proj) break;
#pragma unroll
            for (uint32_t k = 0; k < K; ++k) {
                if (!act[k]) continue;
                const unsigned long long pos = excl + r0 + 32u * k + lane;
                if (a.proj_width[j] == 8)
                    reinterpret_cast<unsigned long long*>(a.proj_dst[j])[pos] = v[q][k];
                else
                    reinterpret_cast<unsigned int*>(a.proj_dst[j])[pos] = static_cast<unsigned int>(v[q][k]);
            }
        }
    }
    if (a.rowids)
#pragma unroll
        for (uint32_t k = 0; k < K; ++k)
            if (act[k]) a.rowids[excl + r0 + 32u * k + lane] = static_cast<long long>(row[k]);
}

constexpr uint32_t kNoGroup = 0xFFFFFFFFu;

// Hands out the next write group of buffer b's super-tile of generation gen
// (the CTA's super-tile ordinal mod 4096): kNoGroup when all are handed out,
// or when the buffer has moved on to a later super-tile.  Called by one lane.
__device__ __forceinline__ uint32_t claim_group(uint32_t* word, uint32_t gen, uint32_t ngr) {
    uint32_t old = *reinterpret_cast<volatile uint32_t*>(word);
    while (true) {
        if ((old >> 20) != gen || (old & 0xFFFFFu) >= ngr) return kNoGroup;
        const uint32_t prev = atomicCAS(word, old, old + 1u);
        if (prev == old) return old & 0xFFFFFu;
        old = prev;
    }
}

__device__ __forceinline__ uint32_t atom_add_acq_rel_cta(uint32_t* p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v)
                 : "memory");
    return old;
}

// Claims and writes groups of buffer b's super-tile (its ordinal jj in the
// CTA's order) until none is left; the warp that finishes the last group
// frees the buffer (freeb[b]).  The buffer's look-back (done[b]) must have
// completed.  Returns the number of groups this warp wrote.
__device__ __forceinline__ uint32_t write_groups(const PushdownArgs& a, const PdSmem& sm, uint32_t b, uint32_t jj,
                                                 uint32_t SR, uint32_t lane, uint32_t max_groups) {
    const long long t = sm.st_id[b];
    const unsigned long long excl = sm.excl[b];
    const uint32_t ngr = sm.ngr[b];
    const uint32_t n = excl < a.max_rows ? (a.max_rows - excl < sm.stot[b] ? static_cast<uint32_t>(a.max_rows - excl)
                                                                           : sm.stot[b])
                                         : 0u;
    uint32_t done_groups = 0;
    while (done_groups < max_groups) {
        uint32_t g = 0;
        if (lane == 0) g = claim_group(&sm.claim[b], jj & 0xFFFu, ngr);
        g = __shfl_sync(0xFFFFFFFFu, g, 0);
        if (g == kNoGroup) break;
        scatter_group(a, sm, b, t * static_cast<int64_t>(SR), excl, n, g, lane);
        ++done_groups;
        __syncwarp();   // every lane's reads of the buffer come before its release
        if (lane == 0 && atom_add_acq_rel_cta(&sm.left[b], 0xFFFFFFFFu) == 1u) mbar_arrive(&sm.freeb[b]);
    }
    return done_groups;
}

}  // namespace

// W consumer warps; a warp evaluates groups of G chunks with one pass over the
// program, and group ownership rotates from sub-tile to sub-tile (as in the
// count scan), so the sub-tile size (a.tile_rows, a multiple of G chunks) is
// independent of W and G.
template <int W, int G>
__global__ void __launch_bounds__((W + kPdWriters + 2) * 32, 1)
    pushdown_persistent_kernel(const __grid_constant__ PushdownArgs a) {
    constexpr uint32_t PRODUCER = W + kPdWriters, LOOKBACK = W + kPdWriters + 1;
    const uint32_t TR = a.tile_rows;                   // rows per sub-tile
    const uint32_t NCH = TR / kChunkRows;              // chunks per sub-tile
    const uint32_t SR = a.super_rows;                  // rows per super-tile
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint32_t s_fail;
    __shared__ long long s_issued;
    __shared__ uint32_t s_slot_off[kMaxSlots];   // read by every leaf: keep it in shared memory
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t S = a.stages;
    const PdSmem sm = pd_smem(smem, SR / kChunkRows);
    if (tid < kMaxSlots) s_slot_off[tid] = a.slot_off[tid];
    uint8_t* stages = smem + a.smem_stage_off;
    const long long n_super = a.n_tiles;

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&sm.full[s], 1);
            mbar_init(&sm.empty[s], W);
        }
        for (uint32_t b = 0; b < kPdBufs; ++b) {
            mbar_init(&sm.evald[b], W);
            mbar_init(&sm.done[b], 1);
            mbar_init(&sm.freeb[b], 1);   // the warp that finishes the last write group (or the look-back)
            sm.evc[b] = 0;
        }
        fence_mbar_init();
        s_fail = 0;
        s_issued = 0;
    }
    {
        uint4* dst = reinterpret_cast<uint4*>(smem + a.smem_prog_off);
        const uint4* src = reinterpret_cast<const uint4*>(a.blob);
        for (uint32_t i = tid; i < a.blob_bytes / 16u; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const uint8_t* blob = smem + a.smem_prog_off;

    if (warp == PRODUCER) {
        // ------------------------------- producer -------------------------------
        const uint64_t pol = policy_evict_first();
        uint32_t s = 0, ph = 0;
        long long k = 0;   // stage fills issued
        bool stop = false;
        // the next super-tile id is taken one super-tile ahead, so that the
        // atomic's round trip does not stall the copies (taking it early changes
        // nothing for progress: it is still worked on after the CTA's smaller ids)
        unsigned long long next_id = 0;
        if (lane == 0) next_id = atomicAdd(a.tile_counter64, 1ull);
        while (!stop) {
            unsigned long long st_id = __shfl_sync(0xFFFFFFFFu, next_id, 0);
            if (lane == 0 && st_id < static_cast<unsigned long long>(n_super))
                next_id = atomicAdd(a.tile_counter64, 1ull);
            const bool last = st_id >= static_cast<unsigned long long>(n_super);
            const int64_t R0 = static_cast<int64_t>(st_id) * SR;
            const uint32_t n_sub = last ? 1u
                : static_cast<uint32_t>(((a.n_rows - R0 < (int64_t)SR ? a.n_rows - R0 : (int64_t)SR) + TR - 1) / TR);
            for (uint32_t u = 0; u < n_sub; ++u, ++k) {
                if (k >= static_cast<long long>(S) && !warp_wait(&sm.empty[s], ph ^ 1u, lane)) {
                    if (lane == 0) fail_flag(a, &s_fail);
                    stop = true;
                    break;
                }
                if (volatile_flag(&s_fail)) {
                    stop = true;
                    break;
                }
                if (last) {
                    if (lane == 0) {
                        sm.tile[s] = -1;
                        mbar_arrive(&sm.full[s]);   // release: the sentinel is visible to the waiters
                    }
                    stop = true;
                } else {
                    const int64_t r0 = R0 + static_cast<int64_t>(u) * TR;
                    const uint32_t valid =
                        static_cast<uint32_t>(a.n_rows - r0 < (int64_t)TR ? a.n_rows - r0 : (int64_t)TR);
                    uint8_t* st = stages + static_cast<size_t>(s) * a.stage_bytes;
                    if (lane == 0) sm.tile[s] = static_cast<long long>(st_id);
                    if (a.tma && valid == TR && a.row_bytes > 0) {
                        if (lane == 0) {
                            mbar_arrive_expect_tx(&sm.full[s], TR * a.row_bytes);
                            for (uint32_t j = 0; j < a.n_slots; ++j)
                                bulk_g2s(st + a.slot_off[j], a.col[j] + r0 * a.width[j], TR * a.width[j], &sm.full[s],
                                         pol);
                        }
                    } else {
                        for (uint32_t j = 0; j < a.n_slots; ++j) {
                            const uint32_t words = valid * a.width[j] / 4u;
                            const uint32_t* src = reinterpret_cast<const uint32_t*>(a.col[j] + r0 * a.width[j]);
                            uint32_t* dst = reinterpret_cast<uint32_t*>(st + a.slot_off[j]);
                            for (uint32_t i = lane; i < words; i += 32) dst[i] = src[i];
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sm.full[s]);
                    }
                }
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        if (lane == 0) s_issued = k;
    } else if (warp == LOOKBACK) {
        // ------------------------------- look-back ------------------------------
        for (uint32_t j = 0;; ++j) {
            const uint32_t b = j % kPdBufs, par = (j / kPdBufs) & 1u;
            if (!warp_wait(&sm.evald[b], par, lane, 500)) {   // a super-tile takes microseconds: sleep meanwhile
                if (lane == 0) fail_flag(a, &s_fail);
                break;
            }
            const long long t = sm.st_id[b];
            if (t < 0) {   // the end: pass the sentinel on to the writers
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.done[b]);
                break;
            }
            // chunk counts from the row words, their prefix in row order (chunks
            // past the super-tile's rows count 0) and the total
            const uint32_t nch = sm.nch[b];
            uint32_t carry = 0;
            for (uint32_t c0 = 0; c0 < sm.ch; c0 += 32) {
                const uint32_t c = c0 + lane;
                uint32_t v = 0;
                if (c < nch) {
                    uint4* w4 = reinterpret_cast<uint4*>(sm.mask + (b * sm.ch + c) * kMaskWords);
                    const uint4 x = w4[0], y = w4[1];
                    v = __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w) + __popc(y.x) + __popc(y.y) +
                        __popc(y.z) + __popc(y.w);
                    if (v) lane_bytes_to_rows(w4, x, y);   // a chunk with no rows is never ranked
                }
                uint32_t inc = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
                    if (lane >= static_cast<uint32_t>(o)) inc += y;
                }
                if (c < sm.ch) sm.cp[b * sm.ch + c] = carry + inc - v;
                carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
            }
            const uint32_t tile_cnt = carry;   // its aggregate is already published by the last consumer warp
            unsigned long long excl = 0;
            bool ok = true;
            if (t > 0) {
                ok = look_back(a, t, lane, &excl);
                if (lane == 0 && ok && t != a.skip_publish_tile)
                    st_relaxed(&a.status[t], kFlagInc | ((excl + tile_cnt) & kValMask));
            }
            // write groups of kPdBatches batches of 32 rows (none past max_rows)
            const bool writes = a.n_proj > 0 || a.rowids != nullptr;
            const unsigned long long n_write =
                (!writes || excl >= a.max_rows) ? 0ull
                                                : (a.max_rows - excl < tile_cnt ? a.max_rows - excl : tile_cnt);
            const uint32_t ngr = static_cast<uint32_t>((n_write + 32u * kPdBatches - 1) / (32u * kPdBatches));
            if (lane == 0) {
                if (!ok) fail_flag(a, &s_fail);
                sm.excl[b] = excl;
                sm.stot[b] = tile_cnt;
                sm.ngr[b] = ok ? ngr : 0u;
                sm.left[b] = ok ? ngr : 0u;
                sm.claim[b] = (j & 0xFFFu) << 20;
                if (t == n_super - 1) *a.total = excl + tile_cnt;
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sm.done[b]);                  // release: offsets and groups visible to the writers
                if (!ok || ngr == 0) mbar_arrive(&sm.freeb[b]);   // nothing to write: the buffer is free
            }
            if (!ok) break;
        }
    } else if (warp < W) {
        // ------------------------------- consumers ------------------------------
        const Instr* ins = reinterpret_cast<const Instr*>(blob + a.instr_off);
        const uint8_t* pool = blob + a.pool_off;
        uint32_t s = 0, ph = 0;
        uint32_t rot = 0;       // running group count: group k of a sub-tile belongs to warp (rot + k) % W
        for (uint32_t j = 0;; ++j) {
            const uint32_t b = j % kPdBufs;
            // ---- the buffer was last used by super-tile j - kPdBufs: until its rows are written,
            //      help write them (a consumer waiting here has nothing else to do) ----
            if (j >= kPdBufs) {
                const uint32_t par = ((j / kPdBufs) - 1) & 1u;
                const unsigned long long w0 = __shfl_sync(0xFFFFFFFFu, global_ns(), 0);
                bool ok = true;
                while (!__all_sync(0xFFFFFFFFu, mbar_try_wait(&sm.freeb[b], par))) {
                    if (__all_sync(0xFFFFFFFFu, mbar_try_wait(&sm.done[b], par)) &&
                        write_groups(a, sm, b, j - kPdBufs, SR, lane, 1u) > 0)
                        continue;
                    if (volatile_flag(&s_fail) || __shfl_sync(0xFFFFFFFFu, global_ns(), 0) - w0 > kWaitNs) {
                        ok = false;
                        break;
                    }
                    __nanosleep(200);   // nothing to write yet: leave the issue slots to the warps that have
                }
                if (!ok) {
                    if (lane == 0) fail_flag(a, &s_fail);
                    break;
                }
            }
            // ---- evaluate super-tile j, sub-tile by sub-tile ----
            long long t = -1;
            uint32_t n_sub = 1;
            bool fail = false;
            for (uint32_t u = 0; u < n_sub; ++u) {
                const uint32_t n_groups = NCH / G;
                const uint32_t first = (warp + W - rot % W) % W;
                if (!warp_wait(&sm.full[s], ph, lane)) {
                    if (lane == 0) fail_flag(a, &s_fail);
                    fail = true;
                    break;
                }
                if (u == 0) {
                    t = sm.tile[s];
                    if (t >= 0) {
                        const int64_t R0 = t * static_cast<int64_t>(SR);
                        const int64_t rows = a.n_rows - R0 < (int64_t)SR ? a.n_rows - R0 : (int64_t)SR;
                        n_sub = static_cast<uint32_t>((rows + TR - 1) / TR);
                    }
                }
                if (t < 0) break;   // sentinel (its stage is never reused)
                const int64_t r0 = t * static_cast<int64_t>(SR) + static_cast<int64_t>(u) * TR;
                const uint32_t valid = static_cast<uint32_t>(a.n_rows - r0 < (int64_t)TR ? a.n_rows - r0 : (int64_t)TR);
                for (uint32_t grp = first; grp < n_groups; grp += W) {
                    uint32_t c0[G], m[G];
#pragma unroll
                    for (int q = 0; q < G; ++q) c0[q] = (grp * G + q) * kChunkRows;
                    eval_program_g<G>(ins, a.n_instr, pool, smem_u32(stages + static_cast<size_t>(s) * a.stage_bytes),
                                      s_slot_off, c0, lane, m);
#pragma unroll
                    for (int q = 0; q < G; ++q) {
                        const uint32_t vm = (c0[q] + kChunkRows <= valid) ? 0xFFu
                                            : c0[q] >= valid             ? 0u
                                                                         : valid_mask(c0[q], lane, valid);
                        m[q] &= vm;
                        const uint32_t g = u * NCH + grp * G + q;   // chunk index in the super-tile (row order)
                        reinterpret_cast<uint8_t*>(sm.mask + (b * sm.ch + g) * kMaskWords)[lane] =
                            static_cast<uint8_t>(m[q]);
                    }
                }
                rot += n_groups;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[s]);   // the stage is no longer read
                if (++s == S) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (fail) break;
            if (warp == 0 && lane == 0) {
                sm.st_id[b] = t;
                sm.nch[b] = t >= 0 ? n_sub * NCH : 0u;
            }
            __syncwarp();
            // The last consumer warp done with super-tile j publishes its
            // aggregate right away: successors' look-backs then wait only for
            // the evaluation of their predecessors, never for this CTA's
            // look-back warp (busy with an earlier super-tile).
            uint32_t last = 0;
            if (lane == 0) last = atom_add_acq_rel_cta(&sm.evc[b], 1u) + 1u == W * (j / kPdBufs + 1u);
            last = __shfl_sync(0xFFFFFFFFu, last, 0);
            __syncwarp();   // lane 0's acquire orders the other warps' mask stores before the reads below
            if (last && t >= 0) {
                const uint32_t nch = n_sub * NCH;
                uint32_t v = 0;
                for (uint32_t c = lane; c < nch; c += 32) {
                    const uint4* w4 = reinterpret_cast<const uint4*>(sm.mask + (b * sm.ch + c) * kMaskWords);
                    const uint4 x = w4[0], y = w4[1];
                    v += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w) + __popc(y.x) + __popc(y.y) +
                         __popc(y.z) + __popc(y.w);
                }
                v = __reduce_add_sync(0xFFFFFFFFu, v);
                if (lane == 0 && t != a.skip_publish_tile)
                    st_relaxed(&a.status[t], (t == 0 ? kFlagInc : kFlagAgg) | v);
            }
            if (lane == 0) mbar_arrive(&sm.evald[b]);   // release: masks, counts, id (and the aggregate) visible
            if (t < 0 || volatile_flag(&s_fail)) break;
        }
    } else {
        // -------------------------------- writers -------------------------------
        for (uint32_t j = 0;; ++j) {
            const uint32_t b = j % kPdBufs;
            // idle writers sleep between tries: they would take issue slots from the consumers
            if (!warp_wait_live(&sm.done[b], (j / kPdBufs) & 1u, &s_fail, 100, 2000)) {
                if (lane == 0) fail_flag(a, &s_fail);
                break;
            }
            if (sm.st_id[b] < 0 || volatile_flag(&s_fail)) break;
            write_groups(a, sm, b, j, SR, lane, 0xFFFFFFFFu);
        }
    }
    __syncthreads();
    if (s_fail && warp == PRODUCER && lane == 0) {
        // copies issued for stages nobody consumed must land before the CTA exits
        const long long issued = s_issued;
        for (long long k = issued > (long long)S ? issued - S : 0; k < issued; ++k)
            mbar_wait_bounded(&sm.full[k % S], static_cast<uint32_t>((k / S) & 1));
    }
}

static inline uint32_t align_up_u32(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

bool pushdown_persistent_ok(int warps, int chunks_per_pass) {
    return ((warps == 8 || warps == 12 || warps == 16) && (chunks_per_pass == 1 || chunks_per_pass == 2)) ||
           (warps == 12 && chunks_per_pass == 3);
}

bool pushdown_persistent_tile_ok(uint32_t tile_rows, int chunks_per_pass) {
    const uint32_t unit = kChunkRows * static_cast<uint32_t>(chunks_per_pass);
    return tile_rows > 0 && tile_rows % unit == 0 && tile_rows <= static_cast<uint32_t>(kPdpMaxChunks * kChunkRows);
}

uint32_t pushdown_super_rows(uint32_t tile_rows, uint32_t target) {
    const uint32_t cap = target < (uint32_t)(kPdpMaxChunks * kChunkRows) ? target : kPdpMaxChunks * kChunkRows;
    if (tile_rows == 0 || tile_rows > cap) return 0u;
    return cap / tile_rows * tile_rows;
}

size_t pushdown_persistent_layout(PushdownArgs& a) {
    a.smem_prog_off = align_up_u32(pd_ctrl_end(a.super_rows / kChunkRows), 16u);
    a.smem_stage_off = align_up_u32(a.smem_prog_off + align_up_u32(a.blob_bytes, 16u), 128u);
    a.stage_bytes = align_up_u32(a.tile_rows * a.row_bytes, 128u);   // one sub-tile of the predicate columns
    a.smem_bytes = a.smem_stage_off + a.stages * a.stage_bytes;
    return a.smem_bytes;
}

template <int W, int Q>
static cudaError_t pdp_set_smem(int optin, int* dyn_max) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, pushdown_persistent_kernel<W, Q>);
    if (e != cudaSuccess) return e;
    const int lim = optin - static_cast<int>(fa.sharedSizeBytes);
    *dyn_max = *dyn_max < 0 ? lim : (lim < *dyn_max ? lim : *dyn_max);
    return cudaFuncSetAttribute(pushdown_persistent_kernel<W, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t pushdown_persistent_max_smem(int optin, int* dyn_max) {
    *dyn_max = -1;
    cudaError_t e = pdp_set_smem<8, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<8, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<12, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<12, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<12, 3>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<16, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = pdp_set_smem<16, 2>(optin, dyn_max);
    return e;
}

cudaError_t launch_pushdown_persistent(const PushdownArgs& a, int grid, int warps, int chunks_per_warp,
                                       cudaStream_t st) {
    if (a.n_tiles <= 0) return cudaSuccess;
    if (a.super_rows == 0 || a.super_rows % a.tile_rows != 0 ||
        a.super_rows > static_cast<uint32_t>(kPdpMaxChunks * kChunkRows) || a.stages < 1 || a.stages > kPdMaxStages)
        return cudaErrorInvalidValue;
    if (warps == 8 && chunks_per_warp == 1)
        pushdown_persistent_kernel<8, 1><<<grid, (8 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 8 && chunks_per_warp == 2)
        pushdown_persistent_kernel<8, 2><<<grid, (8 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 12 && chunks_per_warp == 1)
        pushdown_persistent_kernel<12, 1><<<grid, (12 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 12 && chunks_per_warp == 2)
        pushdown_persistent_kernel<12, 2><<<grid, (12 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 12 && chunks_per_warp == 3)
        pushdown_persistent_kernel<12, 3><<<grid, (12 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 16 && chunks_per_warp == 1)
        pushdown_persistent_kernel<16, 1><<<grid, (16 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else if (warps == 16 && chunks_per_warp == 2)
        pushdown_persistent_kernel<16, 2><<<grid, (16 + kPdWriters + 2) * 32, a.smem_bytes, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace sel
