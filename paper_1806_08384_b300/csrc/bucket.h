// bucket.h -- the column-bucket form of a batch of count probes, shared by
// the host plan builder (bucket_plan.cpp) and the batched count kernel
// (bucket_count.cu).
//
// Every leaf of a compiled program tests one column value against a value
// set that is a union of intervals in the raw bit order of the column (an
// int32 range is one cyclic interval of uint32, a float32 range at most two
// intervals of its bit patterns, a set of codes a union of points).  For one
// table of a batch, the starts and ends of all those intervals on a column
// cut the column's raw domain into buckets; inside a bucket every leaf on
// that column has one value.  A row then needs one bucket index per column
// (a cell table indexed by the value's high bits followed by at most 3
// compares, a binary search over the sorted boundaries, or a linear count
// when there are few of them), and every leaf of every program follows from
// those indices.
//
// Programs are taken to disjunctive normal form (OR of AND-groups of
// possibly negated leaves, at most kBkGroups groups each).  The programs of a
// table are cut into blocks of at most 64; in a block, program k owns the
// 4-bit field k % 8 of group word k / 8, one bit per group.  For a block and
// a column, the table gm[bucket][word] holds, for every group bit, whether
// the group's leaves on that column hold in that bucket (1 when the group has
// no leaf there).  A row's group bits are the AND over the block's columns of
// those words (starting from the block's init mask, which clears unused
// bits); a program holds on the row when any bit of its field is set.  The
// per-field ORs are summed over the lane's rows and the warp (16-bit fields
// of a warp reduction) into per-CTA counters.
//
// Several blocks on one table share the column's global bucket search; a
// block whose leaves distinguish fewer buckets reads its gm table through a
// remap of global to local bucket indices (uint16).
//
// Tables with 3 or more blocks take the quad form instead: blocks are grouped
// by 4 into quads, and a quad's gm rows for a column are 128 bytes, block p's
// 8 group words at bytes 32p .. 32p + 31 (each block still indexed by its own
// local bucket, through a remap that gives the 4 local indices of a global
// bucket in 8 bytes).  In the kernel a quarter-warp evaluates one row for the
// whole quad: lane pair p reads block p's 32 bytes, so the 8 lanes of a
// quarter always read 8 different 16-byte bank groups (one wavefront), where
// the one-row-per-lane gathers of the block form collide in the banks about
// half the time.  The block's init mask is folded into the rows of the quad's
// first column, and each remap has two extra entries: k + 1 (rows past the
// table's end) reads an all-zero row.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sel.h"
#include "kernels.h"

namespace sel {

constexpr int kBkGroups = 4;         // groups per program (one 4-bit field)
constexpr int kBkProgsPerWord = 8;   // 8 fields of 4 bits
constexpr int kBkMaxWords = 8;       // group words per block
constexpr int kBkBlockProgs = kBkProgsPerWord * kBkMaxWords;   // 64 programs per block
constexpr int kBkLinear = 8;         // at most this many boundaries: a linear count can replace a search
constexpr int kBkMaxCells = 2048;    // cells of a BK_CELLS column
constexpr int kBkMaxOcc = 3;         // boundaries per cell for BK_CELLS
constexpr uint32_t kBkIdentity = 0xFFFFFFFFu;   // remap_off: global bucket = local bucket
constexpr int kBkQuadBlocks = 4;     // blocks of a quad
constexpr int kBkQuadMinBlocks = 3;  // tables with at least this many blocks take the quad form
constexpr int kBkQuadMaxSlots = 8;   // columns a quad table may read (bucket indices of a row: 16 bytes)
constexpr uint32_t kBkNoOut = 0xFFFFFFFFu;      // a quad program slot with no probe

// How a row's bucket on one column is found (BkSlot.mode).
enum BkMode : uint32_t {
    BK_LINEAR = 0,   // count the k boundaries <= x (k <= kBkLinear)
    BK_BINARY = 1,   // branch-free binary search over 2^steps - 1 padded boundaries
    BK_CELLS = 2,    // cell c = (x - lo) >> shift gives the buckets before the cell; at most occ
                     // boundaries inside one cell are then compared with x
    BK_CELLS_BIN = 3,  // the same cells, then a branch-free binary search of 2^steps - 1 boundaries
                       // from the cell's first (half = 2^(steps - 1); a cell holds fewer): boundaries
                       // of later cells are all above x, so the search never passes the cell
};

// Search data of one referenced column of a table (48 bytes).
struct BkSlot {
    uint32_t bnd_off;   // byte offset of the sorted boundaries (uint32 or uint64 by the slot width),
                        // padded with all-ones values (to 2^steps - 1 entries when searched, by occ
                        // entries for cells, by 2^steps - 1 for cells searched)
    uint32_t k;         // number of real boundaries; buckets 0..k
    uint32_t half;      // BK_BINARY, BK_CELLS_BIN: 2^(steps - 1)
    uint32_t mode;      // BkMode
    uint32_t cells_off; // BK_CELLS: byte offset of n_cells uint16 counts of boundaries before each cell
    uint32_t n_cells;
    uint32_t shift;
    uint32_t occ;       // largest number of boundaries in one cell
    uint64_t lo;        // BK_CELLS: the smallest boundary
    uint64_t pad;
};
// One block of at most 64 programs of a table.
struct BkBlock {
    uint32_t n_words;               // group words in use (1..8)
    uint32_t nw;                    // words read per gm row: 1, 2, 4 or 8
    uint32_t n_progs;               // programs in the block
    uint32_t out_off;               // byte offset of the uint32 output indices of its programs
    uint32_t n_used;                // columns the block reads
    uint32_t stride;                // words between gm rows: nw, or 12 for 8 (48-byte rows start on
                                    // all 8 16-byte bank groups, so random rows conflict less)
    uint32_t pad[2];
    uint32_t init[kBkMaxWords];     // group bits in use, per word
    uint32_t used[kMaxSlots];       // slot of each column the block reads
    uint32_t remap_off[kMaxSlots];  // per used column: uint16 global -> local bucket table, or kBkIdentity
    uint32_t gm_off[kMaxSlots];     // per used column: gm table [local bucket][stride] uint32
};

// Up to 4 blocks of a quad table (quad form above).  A quad reads every
// column of its table, in slot order (used[u] = u).
struct BkQuad {
    uint32_t n_used;                // columns the quad reads: the table's (<= kBkQuadMaxSlots)
    uint32_t out_off;               // byte offset of 256 uint32 output indices: program k of block p at 64p + k
                                    // (kBkNoOut: none)
    uint32_t pad[2];
    uint32_t used[kBkQuadMaxSlots];       // slot of each column the quad reads
    uint32_t remap_off[kBkQuadMaxSlots];  // per used column: (k + 2) x 4 uint16 local rows of blocks 0..3
    uint32_t gm_off[kBkQuadMaxSlots];     // per used column: 128-byte rows, block p's words at 32p
};

struct BkTable {
    uint32_t n_slots, n_blocks, block_off, max_buckets;   // block_off: byte offset of BkBlock[n_blocks]
    uint32_t n_quads, quad_off, pad[2];                   // quad form: BkQuad[n_quads] (n_blocks is then 0)
    BkSlot slot[kMaxSlots];
};

// Blob header; everything else is addressed by byte offsets from the blob start.
struct BkHeader {
    uint32_t n_tables;
    uint32_t n_out;       // per-CTA counters (one per probe of the launch)
    uint32_t gb_slots;    // >0: the kernel keeps global bucket indices of this many slots per warp in shared memory
    uint32_t gb_quad;     // 1: a quad table keeps a 16-byte record of bucket indices per row of a chunk per warp
    BkTable t[kMaxTables];
};

// Bytes of shared memory a consumer warp keeps bucket indices in, for G
// chunks a pass: global indices of gb_slots slots (block form), or one
// 16-byte record per row of a chunk (quad form; a chunk at a time).
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t bk_gb_bytes_per_warp(uint32_t gb_slots, uint32_t gb_quad, uint32_t G) {
    const uint32_t blocks = gb_slots * 8u * G * 32u * 2u, quads = gb_quad ? 256u * 16u : 0u;
    return blocks > quads ? blocks : quads;
}

// The host side of a bucket plan: one blob for one launch (at most kMaxTables tables).
struct BucketPlan {
    std::vector<uint8_t> blob;   // BkHeader | boundaries | output indices | remaps | gm tables | BkBlock arrays
    uint32_t n_out = 0;
};

struct Program;

// One table of a batch: its referenced columns (slots) and the programs run on it.
struct BkTableIn {
    std::vector<uint32_t> slot_width;              // bytes per value of each slot (4 or 8)
    std::vector<const Program*> progs;
    std::vector<std::vector<int32_t>> slot_maps;   // per program: its slot -> the table's slot
    std::vector<uint32_t> outs;                    // per program: index of its count
};

// Builds the blob; SEL_ERR_UNSUPPORTED (reason in *why) when the batch does
// not fit the bucket form.
sel_status build_bucket_plan(const std::vector<BkTableIn>& tables, BucketPlan* out, std::string* why);

// Evaluates a plan on the host over host column data (cols[table][slot],
// widths[table][slot]); adds each probe's count to counts[out].
void bucket_eval_host(const BucketPlan& plan, const std::vector<std::vector<const uint8_t*>>& cols,
                      const std::vector<std::vector<uint32_t>>& widths, const std::vector<int64_t>& n_rows,
                      uint64_t* counts);

}  // namespace sel
