// count.cu -- fused filtered COUNT scan (§3.1 "Selectivity Computation": the
// exact cardinality of a pushed-down selection is the result of
// SELECT COUNT(*) FROM R WHERE <predicates>), generalised to a batch of
// programs over up to kMaxTables tables in one persistent launch.
//
// Each CTA walks the launch's global tile sequence with stride gridDim.x.
// Thread 0 keeps `stages` tiles in flight: for a full, 16-byte aligned tile
// it issues one bulk copy per referenced column into a shared-memory stage
// and arms the stage's mbarrier with the byte count; any other tile (the
// ragged last tile of a table, or unaligned columns) is copied by the whole
// CTA with plain loads once the stage is free.  Every warp then evaluates
// every program of the tile's table on its 256-row chunks, bit-sliced (one
// bit per row), and adds popc of the masks to a per-program shared counter;
// the counters are added to the 64-bit global counts once per CTA.  Column
// tiles are therefore read from HBM exactly once per launch, whatever the
// number of programs on the table.
#include "kernels.h"
#include "scan.cuh"

namespace sel {

__device__ __forceinline__ int find_table(const ScanArgs& a, int64_t g) {
    int t = 0;
    while (t + 1 < static_cast<int>(a.n_tables) && g >= a.t[t + 1].tile_begin) ++t;
    return t;
}

__device__ __forceinline__ void issue_tile(const ScanArgs& a, int64_t g, uint32_t s, uint8_t* stages,
                                           uint64_t* full, uint64_t pol) {
    if (g >= a.total_tiles) return;
    const TableArg& T = a.t[find_table(a, g)];
    const int64_t r0 = (g - T.tile_begin) * static_cast<int64_t>(a.tile_rows);
    const bool whole = r0 + a.tile_rows <= T.n_rows;
    if (T.tma && whole && T.row_bytes > 0) {
        uint8_t* st = stages + static_cast<size_t>(s) * a.stage_bytes;
        mbar_arrive_expect_tx(&full[s], a.tile_rows * T.row_bytes);
        for (uint32_t j = 0; j < T.n_slots; ++j)
            bulk_g2s(st + T.slot_off[j], T.col[j] + r0 * T.width[j], a.tile_rows * T.width[j], &full[s], pol);
    } else {
        mbar_arrive(&full[s]);   // completes the phase; the CTA copies this tile itself
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_count_kernel(const __grid_constant__ ScanArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5, n_warps = blockDim.x >> 5;
    const uint32_t S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem + a.cnt_off);
    uint8_t* stages = smem + a.stage_off;

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x) cnt[p] = 0ull;
    const uint8_t* blob = a.blob;
    if (a.prog_in_smem) {
        uint4* dst = reinterpret_cast<uint4*>(smem + a.prog_off);
        const uint4* src = reinterpret_cast<const uint4*>(a.blob);
        for (uint32_t i = tid; i < a.blob_bytes / 16u; i += blockDim.x) dst[i] = src[i];
        blob = smem + a.prog_off;
    }
    __syncthreads();
    const ProgDesc* pd = reinterpret_cast<const ProgDesc*>(blob);
    const Instr* ins = reinterpret_cast<const Instr*>(blob + a.instr_off);
    const uint8_t* pool = blob + a.pool_off;

    const int64_t G = gridDim.x;
    const uint64_t pol = policy_evict_first();
    if (tid == 0)
        for (uint32_t s = 0; s < S; ++s) issue_tile(a, blockIdx.x + s * G, s, stages, full, pol);

    for (int64_t k = 0;; ++k) {
        const int64_t g = blockIdx.x + k * G;
        if (g >= a.total_tiles) break;
        const uint32_t s = static_cast<uint32_t>(k % S);
        const uint32_t parity = static_cast<uint32_t>((k / S) & 1);
        const TableArg& T = a.t[find_table(a, g)];
        const int64_t r0 = (g - T.tile_begin) * static_cast<int64_t>(a.tile_rows);
        const uint32_t valid = static_cast<uint32_t>((T.n_rows - r0 < (int64_t)a.tile_rows ? T.n_rows - r0 : (int64_t)a.tile_rows));
        const bool bulk = T.tma && valid == a.tile_rows && T.row_bytes > 0;
        const bool ok = mbar_wait_bounded(&full[s], parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(a.err, 1u);
            // let the copies already issued for the next stages land (bounded) before leaving
            for (uint32_t j = 1; j < S; ++j) {
                const int64_t kj = k + j;
                if (blockIdx.x + kj * G >= a.total_tiles) break;
                mbar_wait_bounded(&full[kj % S], static_cast<uint32_t>((kj / S) & 1));
            }
            break;   // every thread leaves together
        }
        uint8_t* st = stages + static_cast<size_t>(s) * a.stage_bytes;
        if (!bulk) {
            for (uint32_t j = 0; j < T.n_slots; ++j) {
                const uint32_t words = valid * T.width[j] / 4u;
                const uint32_t* src = reinterpret_cast<const uint32_t*>(T.col[j] + r0 * T.width[j]);
                uint32_t* dst = reinterpret_cast<uint32_t*>(st + T.slot_off[j]);
                for (uint32_t i = tid; i < words; i += blockDim.x) dst[i] = src[i];
            }
            __syncthreads();
        }
        const uint32_t n_chunks = (valid + kChunkRows - 1) / kChunkRows;
        const uint32_t st_addr = smem_u32(st);
        for (uint32_t ch = warp; ch < n_chunks; ch += n_warps) {
            const uint32_t c0 = ch * kChunkRows;
            const uint32_t vm = (c0 + kChunkRows <= valid) ? 0xFFu : valid_mask(c0, lane, valid);
            for (uint32_t p = T.prog_begin; p < T.prog_end; ++p) {
                const uint32_t m =
                    eval_program(ins + pd[p].instr_begin, pd[p].n_instr, pool, st_addr, T.slot_off, c0, lane) & vm;
                const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, static_cast<uint32_t>(__popc(m)));
                if (lane == 0 && c) atomicAdd(&cnt[p], static_cast<unsigned long long>(c));
            }
        }
        __syncthreads();   // stage s is free again
        if (tid == 0) issue_tile(a, g + static_cast<int64_t>(S) * G, s, stages, full, pol);
    }
    __syncthreads();
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x)
        if (cnt[p]) atomicAdd(&a.counts[pd[p].out], cnt[p]);
}

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

size_t scan_layout(ScanArgs& a) {
    a.cnt_off = align_up(8u * a.stages, 16u);
    a.prog_off = align_up(a.cnt_off + 8u * a.n_progs, 16u);
    const uint32_t prog_bytes = a.prog_in_smem ? align_up(a.blob_bytes, 16u) : 0u;
    a.stage_off = align_up(a.prog_off + prog_bytes, 128u);
    return static_cast<size_t>(a.stage_off) + static_cast<size_t>(a.stages) * a.stage_bytes;
}

cudaError_t scan_kernel_max_smem(int bytes) {
    return cudaFuncSetAttribute(scan_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_scan_count(const ScanArgs& a, int grid, size_t smem, cudaStream_t st) {
    scan_count_kernel<<<grid, kScanThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sel
