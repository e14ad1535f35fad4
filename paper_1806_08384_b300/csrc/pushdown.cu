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
#include "scan.cuh"

namespace sel {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive prefix of tile t (t >= 1) by warp 0; false if a wait timed out.
__device__ bool look_back(const PushdownArgs& a, long long t, uint32_t lane, unsigned long long* excl_out) {
    unsigned long long excl = 0;
    long long base = t - 1;
    const unsigned long long t0 = global_ns();
    while (true) {
        const long long idx = base - static_cast<long long>(lane);
        unsigned long long v = (idx >= 0) ? ld_relaxed(&a.status[idx]) : kFlagInc;
        while (__any_sync(0xFFFFFFFFu, (v >> 62) == 0)) {
            if (global_ns() - t0 > a.wait_ns) {
                *excl_out = excl;
                return false;
            }
            if ((v >> 62) == 0) v = ld_relaxed(&a.status[idx]);
        }
        const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 2);
        if (inc) {
            const uint32_t k = __ffs(inc) - 1;   // nearest predecessor with an inclusive prefix
            unsigned long long x = (lane <= k) ? (v & kValMask) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
            excl += x;
            *excl_out = excl;
            return true;
        }
        unsigned long long x = v & kValMask;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
        excl += x;
        base -= 32;
    }
}

__global__ void __launch_bounds__(kPdThreads, 6) pushdown_kernel(const __grid_constant__ PushdownArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned long long s_tile, s_excl;
    __shared__ uint32_t s_chunk_cnt[kPdThreads / 32 * 4];
    __shared__ uint32_t s_fail;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, n_warps = blockDim.x >> 5;

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
            const uint32_t m = eval_program(ins, a.n_instr, pool, st_addr, a.slot_off, c0, lane) & vm;
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

}  // namespace sel
