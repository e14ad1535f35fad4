// count.cu -- fused filtered COUNT scan (§3.1 "Selectivity Computation": the
// exact cardinality of a pushed-down selection is the result of
// SELECT COUNT(*) FROM R WHERE <predicates>), generalised to a batch of
// programs over up to kMaxTables tables in one persistent launch.
//
// Warp roles.  The last warp is the producer: it keeps `stages` tiles in
// flight -- for a full, 16-byte aligned tile its lane 0 issues one bulk copy
// per referenced column into a shared-memory stage, completing on the
// stage's `full` mbarrier; any other tile (the ragged last tile of a table,
// unaligned columns) is copied by the producer warp with plain loads, which
// then arrives on `full` itself.  The consumer warps evaluate every program
// of the tile's table on 256-row chunks, bit-sliced (one bit per row), add
// popc of the masks to per-program shared counters, and arrive on the
// stage's `empty` mbarrier; the producer refills a stage once every consumer
// warp has arrived.  Consumers never wait for each other, and chunk
// ownership rotates from tile to tile, so tiles with fewer chunks than warps
// leave no warp idle.  Each column tile is read from HBM exactly once per
// launch, whatever the number of programs on the table.
#include <algorithm>

#include "kernels.h"
#include "scan.cuh"

namespace sel {

// Consumer warps: evaluate every tile's chunk groups for all programs of the
// tile's table.  blob is the program blob (shared or global memory); the
// kernel calls this with a pointer the compiler can trace to shared memory
// when the blob is staged there, so instruction and pool reads are shared loads.
// MASK (one program on one table, the first pass of the two-pass push-down):
// every chunk stores its number of selected rows (ccnt) and, if it has some,
// its lane bytes (mask: byte l of chunk c is lane l's 8-bit mask, bit i < 4
// row 4l + i, bit 4 + i row 128 + 4l + i of the chunk), with no atomic; the
// total is left to the kernels that sum the chunk counts.
template <int W, int G, bool MASK>
__device__ __forceinline__ void consume_tiles(const ScanArgs& a, const uint8_t* blob, uint64_t* full, uint64_t* empty,
                                              unsigned long long* cnt, uint8_t* stages,
                                              const uint32_t (&s_off)[kMaxTables][kMaxSlots], uint32_t* s_fail,
                                              uint32_t warp, uint32_t lane) {
    const int64_t NB = gridDim.x;
    const uint32_t S = a.stages;
    const ProgDesc* pd = reinterpret_cast<const ProgDesc*>(blob);
    const Instr* ins = reinterpret_cast<const Instr*>(blob + a.instr_off);
    const uint8_t* pool = blob + a.pool_off;
    uint32_t rot = 0;   // running chunk count: chunk c of a tile belongs to warp (rot + c) % W
    uint32_t s = 0, parity = 0;
    for (int64_t k = 0;; ++k) {
        const int64_t g = blockIdx.x + k * NB;
        if (g >= a.total_tiles) break;
        const int ti = find_table(a, g);
        const TableArg& T = a.t[ti];
        const uint32_t valid = tile_valid(a, T, g);
        const uint32_t n_chunks = (valid + kChunkRows - 1) / kChunkRows;
        const uint32_t n_groups = (n_chunks + G - 1) / G;
        const uint32_t first = (warp + W - rot % W) % W;
        // every lane waits for the stage (a lane-0-only wait with the other
        // lanes parked at a shuffle resumes much later); one verdict per warp
        const bool okw = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(&full[s], parity));
        if (!okw) {
            if (lane == 0) {
                atomicOr(a.err, 1u);
                atomicOr(s_fail, 1u);
                mbar_wait_bounded(&full[s], parity);   // a copy still in flight lands before we leave
            }
            break;
        }
        if (*reinterpret_cast<volatile uint32_t*>(s_fail)) break;
        const uint32_t st_addr = smem_u32(stages + static_cast<size_t>(s) * a.stage_bytes);
        // MASK: the tile's first chunk's mask byte of this lane, and its count
        [[maybe_unused]] uint8_t* tile_mask = nullptr;
        [[maybe_unused]] uint16_t* tile_ccnt = nullptr;
        if constexpr (MASK) {
            const int64_t tc0 = (g - T.tile_begin) * static_cast<int64_t>(a.tile_rows / kChunkRows);
            tile_mask = a.mask + tc0 * 32 + lane;
            tile_ccnt = a.ccnt + tc0;
        }
        for (uint32_t grp = first; grp < n_groups; grp += W) {
            uint32_t c0[G], vm[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const uint32_t ch = grp * G + q;
                // a missing chunk of the last group re-reads the group's first chunk, masked out
                c0[q] = (ch < n_chunks ? ch : grp * G) * kChunkRows;
                vm[q] = ch >= n_chunks ? 0u
                        : (c0[q] + kChunkRows <= valid) ? 0xFFu
                                                          : valid_mask(c0[q], lane, valid);
            }
            for (uint32_t p = T.prog_begin; p < T.prog_end; ++p) {
                uint32_t m[G];
                eval_program_g<G>(ins + pd[p].instr_begin, pd[p].n_instr, pool, st_addr, s_off[ti], c0, lane, m);
                if constexpr (MASK) {
                    const uint32_t chunk0 = grp * G;   // in the tile
#pragma unroll
                    for (int q0 = 0; q0 < G; q0 += 2) {   // two chunk counts per reduction
                        const int q1 = q0 + 1 < G ? q0 + 1 : q0;   // G odd: the last pair has one chunk
                        const uint32_t m0 = m[q0] & vm[q0];
                        const uint32_t m1 = q0 + 1 < G ? m[q1] & vm[q1] : 0u;
                        const uint32_t both = __reduce_add_sync(0xFFFFFFFFu, __popc(m0) | (__popc(m1) << 16));
                        // predicated stores: a chunk without selected rows stores no mask, a
                        // missing chunk of a tile's last group nothing
                        const bool has0 = chunk0 + q0 < n_chunks;
                        const bool has1 = q0 + 1 < G && chunk0 + q0 + 1 < n_chunks;
                        uint8_t* mp = tile_mask + (chunk0 + q0) * 32u;
                        if (has0 && (both & 0xFFFFu)) mp[0] = static_cast<uint8_t>(m0);
                        if (has1 && (both >> 16)) mp[32] = static_cast<uint8_t>(m1);
                        if (lane == 0) {
                            if (has0) tile_ccnt[chunk0 + q0] = static_cast<uint16_t>(both & 0xFFFFu);
                            if (has1) tile_ccnt[chunk0 + q0 + 1] = static_cast<uint16_t>(both >> 16);
                        }
                    }
                } else {
                    uint32_t pc = 0;
#pragma unroll
                    for (int q = 0; q < G; ++q) pc += __popc(m[q] & vm[q]);
                    const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, pc);
                    if (lane == 0 && c) atomicAdd(&cnt[p], static_cast<unsigned long long>(c));
                }
            }
        }
        rot += n_groups;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            parity ^= 1u;
        }
    }
}

// W consumer warps (+1 producer warp); each consumer pass evaluates the
// programs on G chunks at once (G independent mask stacks share one
// instruction stream, which hides the interpreter's latency).
template <int W, int G, bool MASK>
__global__ void __launch_bounds__((W + 1) * 32, (W == 8 && G < 4) ? 2 : 1) scan_count_kernel(const __grid_constant__ ScanArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint32_t s_off[kMaxTables][kMaxSlots];
    __shared__ uint32_t s_fail;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem + a.cnt_off);
    uint8_t* stages = smem + a.stage_off;

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    for (uint32_t i = tid; i < kMaxTables * kMaxSlots; i += blockDim.x)
        s_off[i / kMaxSlots][i % kMaxSlots] = a.t[i / kMaxSlots].slot_off[i % kMaxSlots];
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x) cnt[p] = 0ull;
    const uint8_t* blob = a.blob;
    if (a.prog_in_smem) {
        uint4* dst = reinterpret_cast<uint4*>(smem + a.prog_off);
        const uint4* src = reinterpret_cast<const uint4*>(a.blob);
        for (uint32_t i = tid; i < a.blob_bytes / 16u; i += blockDim.x) dst[i] = src[i];
        blob = smem + a.prog_off;
    }
    __syncthreads();
    const int64_t NB = gridDim.x;

    if (warp == W) {
        // ------------------------------- producer -------------------------------
        const uint64_t pol = policy_evict_first();
        uint32_t s = 0, phase = 0;   // stage of tile k and the number of times it was reused, mod 2
        for (int64_t k = 0;; ++k) {
            const int64_t g = blockIdx.x + k * NB;
            if (g >= a.total_tiles) break;
            if (k >= S) {   // wait until every consumer warp released the stage's previous tile
                const bool ok = mbar_wait_bounded(&empty[s], phase ^ 1u);
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    // consumers waiting for tiles that are never produced give up on their own bound
                    if (lane == 0) {
                        atomicOr(a.err, 1u);
                        atomicOr(&s_fail, 1u);
                    }
                    break;
                }
            }
            produce_tile(a, g, s, stages, full, pol, lane);
            if (++s == S) {
                s = 0;
                phase ^= 1u;
            }
        }
    } else if (a.prog_in_smem) {
        // the program's address space is visible to the compiler: shared loads
        consume_tiles<W, G, MASK>(a, smem + a.prog_off, full, empty, cnt, stages, s_off, &s_fail, warp, lane);
    } else {
        consume_tiles<W, G, MASK>(a, a.blob, full, empty, cnt, stages, s_off, &s_fail, warp, lane);
    }
    __syncthreads();
    if (s_fail) return;   // counts are invalid; the error flag is set
    if constexpr (MASK) return;   // the chunk counts are the result
    const ProgDesc* pd = reinterpret_cast<const ProgDesc*>(blob);
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x)
        if (cnt[p]) atomicAdd(&a.counts[pd[p].out], cnt[p]);
}

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

size_t scan_layout(ScanArgs& a) {
    a.cnt_off = align_up(16u * a.stages, 16u);   // full[S] | empty[S]
    a.prog_off = align_up(a.cnt_off + 8u * a.n_progs, 16u);
    const uint32_t prog_bytes = a.prog_in_smem ? align_up(a.blob_bytes, 16u) : 0u;
    a.stage_off = align_up(a.prog_off + prog_bytes, 128u);
    return static_cast<size_t>(a.stage_off) + static_cast<size_t>(a.stages) * a.stage_bytes;
}

template <int W, int G, bool MASK>
static cudaError_t set_smem_limit_1(int optin, int* dyn_max) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, scan_count_kernel<W, G, MASK>);
    if (e != cudaSuccess) return e;
    const int lim = optin - static_cast<int>(fa.sharedSizeBytes);
    *dyn_max = *dyn_max < 0 ? lim : std::min(*dyn_max, lim);
    return cudaFuncSetAttribute(scan_count_kernel<W, G, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

template <int W, int G>
static cudaError_t set_smem_limit(int optin, int* dyn_max) {
    cudaError_t e = set_smem_limit_1<W, G, false>(optin, dyn_max);
    return e == cudaSuccess ? set_smem_limit_1<W, G, true>(optin, dyn_max) : e;
}

cudaError_t scan_kernel_max_smem(int optin, int* dyn_max) {
    *dyn_max = -1;
    cudaError_t e = set_smem_limit<8, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<8, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<16, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<16, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<8, 4>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<15, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = set_smem_limit<15, 3>(optin, dyn_max);
    return e;
}

// 16 consumer warps and the producer put 5 warps on one scheduler, which caps
// a thread at 96 registers (the 2-chunk pass spills a few words); 15 consumer
// warps make 4 a scheduler and 128 registers, room for 3 chunks a pass.
bool scan_variant_ok(int warps, int group) {
    return ((warps == 8 || warps == 16) && (group == 1 || group == 2)) || (warps == 8 && group == 4) ||
           (warps == 15 && (group == 2 || group == 3));
}

template <bool MASK>
static cudaError_t launch_scan_count_1(const ScanArgs& a, int grid, size_t smem, cudaStream_t st, int warps,
                                       int group) {
    if (warps == 8 && group == 1)
        scan_count_kernel<8, 1, MASK><<<grid, 9 * 32, smem, st>>>(a);
    else if (warps == 8 && group == 2)
        scan_count_kernel<8, 2, MASK><<<grid, 9 * 32, smem, st>>>(a);
    else if (warps == 16 && group == 1)
        scan_count_kernel<16, 1, MASK><<<grid, 17 * 32, smem, st>>>(a);
    else if (warps == 16 && group == 2)
        scan_count_kernel<16, 2, MASK><<<grid, 17 * 32, smem, st>>>(a);
    else if (warps == 8 && group == 4)
        scan_count_kernel<8, 4, MASK><<<grid, 9 * 32, smem, st>>>(a);
    else if (warps == 15 && group == 2)
        scan_count_kernel<15, 2, MASK><<<grid, 16 * 32, smem, st>>>(a);
    else if (warps == 15 && group == 3)
        scan_count_kernel<15, 3, MASK><<<grid, 16 * 32, smem, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_scan_count(const ScanArgs& a, int grid, size_t smem, cudaStream_t st, int warps, int group) {
    if (a.mask) {   // one program on one table
        if (a.n_tables != 1 || a.n_progs != 1 || a.tile_rows % kChunkRows != 0 || a.tile_rows > kMaxTileRows ||
            !a.ccnt)
            return cudaErrorInvalidValue;
        return launch_scan_count_1<true>(a, grid, smem, st, warps, group);
    }
    return launch_scan_count_1<false>(a, grid, smem, st, warps, group);
}

}  // namespace sel
