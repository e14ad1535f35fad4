// kernels.h -- launch interface between the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

namespace sel {

constexpr int kMaxTables = 8;
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any device wait
// Count-scan variants: consumer warps (8, 15 or 16, plus one producer warp)
// and chunks evaluated per instruction pass (1, 2, 3 or 4; scan_variant_ok).
constexpr int kScanDefaultWarps = 15;
constexpr int kMaxTileRows = 16384;
constexpr int kScanDefaultGroup = 3;

// One table of a scan launch: its referenced columns ("slots"), its tiles in
// the launch's global tile sequence and the programs evaluated on it.
struct TableArg {
    const uint8_t* col[kMaxSlots];   // device base pointer of each slot's column
    int64_t n_rows;
    int64_t tile_begin;              // first global tile index of this table
    int64_t n_tiles;                 // ceil(n_rows / tile_rows)
    uint32_t slot_off[kMaxSlots];    // byte offset of each slot inside a stage
    uint32_t width[kMaxSlots];       // bytes per element of each slot
    uint32_t prog_begin, prog_end;   // programs [prog_begin, prog_end) run on this table
    uint32_t n_slots;
    uint32_t row_bytes;              // sum of the slot widths
    uint32_t tma;                    // 1: every slot base is 16-byte aligned
    uint32_t pad;
};

// Program blob (device): ProgDesc[n_progs] | Instr[] at instr_off | pool at pool_off.
struct ScanArgs {
    const uint8_t* blob;
    uint32_t n_progs, instr_off, pool_off, blob_bytes;
    uint32_t tile_rows, stages, stage_bytes, prog_in_smem;
    uint32_t cnt_off, prog_off, stage_off, n_tables;
    uint32_t aux_off, aux_pad;       // bucket kernel: per-warp bucket-index buffers (0 bytes otherwise)
    int64_t total_tiles;
    unsigned long long* counts;      // n_progs, zeroed before the launch
    unsigned int* err;               // bit 0: a bounded wait timed out
    // Mask output of the two-pass push-down (one program on one table; null
    // otherwise): every chunk's selected-row count and the lane bytes of the
    // chunks that have some; counts is then not written.
    uint8_t* mask;                   // [chunks][32]
    uint16_t* ccnt;                  // [chunks]
    TableArg t[kMaxTables];
};

// Shared-memory bytes needed by a scan launch (and fills the *_off fields).
size_t scan_layout(ScanArgs& a);
bool scan_variant_ok(int warps, int group);
cudaError_t launch_scan_count(const ScanArgs& a, int grid, size_t smem, cudaStream_t st, int warps, int group);
// Sets every scan variant's dynamic shared-memory limit to the opt-in maximum
// minus its static shared memory; *dyn_max receives the smallest of them.
cudaError_t scan_kernel_max_smem(int optin, int* dyn_max);

// Batched count over the column-bucket form of the probes (bucket.h): a.blob
// is the bucket blob (staged in shared memory), a.n_progs its counter count.
// gb_bytes_per_warp: shared bytes of one warp's bucket-index buffer.  Variants:
// 8, 11, 15 or 16 consumer warps, 1 or 2 chunks per pass (bucket_variant_ok).
size_t bucket_layout(ScanArgs& a, int warps, uint32_t gb_bytes_per_warp);
bool bucket_variant_ok(int warps, int group);
cudaError_t launch_bucket_count(const ScanArgs& a, int grid, size_t smem, cudaStream_t st, int warps, int group);
cudaError_t bucket_kernel_max_smem(int optin, int* dyn_max);

// ---------------------------------------------------------------------------
// push-down (stable compaction with decoupled look-back)
// ---------------------------------------------------------------------------
constexpr int kPdThreads = 128;       // 4 warps: a 1024-row tile is one 256-row chunk per warp
constexpr int kPdMaxTileRows = 4096;  // at most 4 chunks per warp
constexpr int kPdMaxProj = 16;

struct PushdownArgs {
    const uint8_t* blob;             // single-program blob (ProgDesc | Instr | pool)
    uint32_t instr_off, pool_off, n_instr, blob_bytes;
    const uint8_t* col[kMaxSlots];   // predicate slots
    uint32_t width[kMaxSlots];
    uint32_t slot_off[kMaxSlots];
    uint32_t n_slots, row_bytes, tma, tile_rows;
    int64_t n_rows, n_tiles;
    // projection
    uint32_t n_proj;
    int32_t proj_slot[kPdMaxProj];   // slot index when the column is a predicate slot, else -1
    const uint8_t* proj_src[kPdMaxProj];
    uint8_t* proj_dst[kPdMaxProj];
    uint32_t proj_width[kPdMaxProj];
    uint32_t proj_stage_off[kPdMaxProj + 1];   // the last used entry is the row ids
    long long* rowids;               // may be null
    unsigned long long max_rows;
    // scratch
    unsigned long long* status;      // n_tiles, zeroed
    unsigned int* tile_counter;      // zeroed
    unsigned long long* total;       // count written by the last tile
    unsigned int* err;
    // fault injection for the timeout test: this tile never publishes
    long long skip_publish_tile;
    unsigned long long wait_ns;
    uint32_t smem_prog_off, smem_stage_off, smem_out_off, smem_bytes;
    // persistent kernel only: pipeline stages of tile_rows rows each; the
    // look-back unit (n_tiles of them) is a super-tile of super_rows rows
    uint32_t stages, stage_bytes, super_rows;
    unsigned long long* tile_counter64;   // zeroed; tiles handed out in order
};

size_t pushdown_layout(PushdownArgs& a);

// ---------------------------------------------------------------------------
// two-pass push-down: the count scan stores the row masks (ScanArgs.mask),
// a one-CTA kernel turns the segment counts into output offsets, and the
// scatter kernel writes the selected rows
// ---------------------------------------------------------------------------
constexpr uint32_t kSegChunks = 64;   // a segment: 64 chunks (16384 rows), one scatter warp
constexpr uint32_t kGrpSegs = 64;     // an offset group: 64 segments

struct ScatterArgs {
    const uint8_t* mask;                 // [chunks][32] lane bytes (of the chunks with selected rows)
    const uint16_t* ccnt;                // [chunks] selected rows per chunk
    const uint32_t* seg_cnt;             // [n_grp * kGrpSegs] selected rows per segment (zero past the table)
    const unsigned long long* grp_off;   // [n_grp] output offset of each group's first row
    int64_t n_rows, n_seg;
    uint32_t n_proj, pad;
    const uint8_t* src[kPdMaxProj];
    uint8_t* dst[kPdMaxProj];
    uint32_t width[kPdMaxProj];          // 4 or 8
    long long* rowids;                   // may be null
    unsigned long long max_rows;
};

// seg_cnt[s] = the sum of segment s's chunk counts, for all n_grp * kGrpSegs
// segments (0 past the table's n_chunks chunks).
cudaError_t launch_seg_sum(const uint16_t* ccnt, int64_t n_chunks, uint32_t* seg_cnt, int64_t n_grp, cudaStream_t st);
// grp_off[g] = sum of seg_cnt over the groups before g (n_grp groups);
// *total = the sum over all groups.
cudaError_t launch_seg_scan(const uint32_t* seg_cnt, unsigned long long* grp_off, int64_t n_grp,
                            unsigned long long* total, cudaStream_t st);
cudaError_t launch_pushdown_scatter(const ScatterArgs& a, cudaStream_t st);
cudaError_t launch_pushdown(const PushdownArgs& a, cudaStream_t st);

// Persistent push-down: one CTA per SM with W consumer warps (8, 12 or 16)
// evaluating groups of G chunks (1 or 2), a producer warp and a look-back warp;
// sub-tiles of tile_rows rows stream through `stages` shared-memory stages and
// the look-back unit (n_tiles, status words) is a super-tile of super_rows
// rows: the largest multiple of tile_rows that is at most a target of 32768
// to kPdpMaxChunks chunks (131072 rows).
constexpr int kPdpMaxChunks = 512;
constexpr int kPdpMinSuperRows = 32768;
bool pushdown_persistent_ok(int warps, int chunks_per_pass);
// tile_rows: a multiple of chunks_per_pass chunks, at most kPdpMaxChunks chunks.
bool pushdown_persistent_tile_ok(uint32_t tile_rows, int chunks_per_pass);
// The largest multiple of tile_rows that is at most min(target, kPdpMaxChunks
// chunks); 0 when tile_rows is larger.
uint32_t pushdown_super_rows(uint32_t tile_rows, uint32_t target);
// Fills the shared-memory offsets for a.stages stages of a.tile_rows rows and
// the row masks of super-tiles of a.super_rows rows; returns the bytes needed.
size_t pushdown_persistent_layout(PushdownArgs& a);
cudaError_t pushdown_persistent_max_smem(int optin, int* dyn_max);
cudaError_t launch_pushdown_persistent(const PushdownArgs& a, int grid, int warps, int chunks_per_warp,
                                       cudaStream_t st);

}  // namespace sel
