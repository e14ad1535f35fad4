// internal.h -- host-side structures of the runtime (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/sel.h"
#include "kernels.h"
#include "program.h"

namespace sel {

void set_error(const char* fmt, ...);

// Every device and pinned host allocation of the library goes through these
// two; sel_debug_fail_allocation can make the n-th one fail with
// cudaErrorMemoryAllocation (reported as SEL_ERR_OOM) without allocating.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t host_alloc(void** p, size_t bytes);

// A comparison leaf of the normalised tree, kept for featurisation.
struct Clause {
    int32_t col;
    int32_t kind;       // SEL_N_CMP / SEL_N_BETWEEN / SEL_N_IN / SEL_N_LIKE
    int32_t op;         // SEL_N_CMP
    int32_t negated;
    int64_t i_lo, i_hi; // integer-like bounds (inclusive, for CMP/BETWEEN/IN as range of codes)
    float f_lo, f_hi;
    std::vector<int64_t> ivals;
    std::vector<float> fvals;
    int32_t code_lo, code_hi;   // LIKE: matching dictionary codes (range when contiguous)
    int32_t like_count;         // LIKE: number of matching codes
    // source-level description used by the learned estimator's features
    int32_t nnf_neg;            // the leaf sits under an odd number of NOTs
    int64_t raw_i0, raw_i1;     // constants as written (CMP: i0; BETWEEN: i0..i1)
    float raw_f0, raw_f1;
    std::vector<int32_t> like_codes;   // LIKE: every matching code
};

// Host program compiled by sel_compile_predicate.
struct Program {
    std::vector<Instr> instrs;
    std::vector<uint8_t> pool;
    std::vector<int32_t> slot_col;    // slot -> table column
    std::vector<uint32_t> slot_width; // slot -> bytes per element
    int32_t need = 0;                 // evaluation stack entries
    int32_t leaves = 0;
};

}  // namespace sel

struct sel_pred {
    uint64_t id;
    uint64_t content = 0;              // hash of the compiled program (plan cache key)
    std::vector<int32_t> col_types;    // schema the program was compiled against
    sel::Program prog;
    // clause structure for the learned estimator: OR of AND groups of leaves
    // (empty when the tree does not have that shape)
    std::vector<std::vector<sel::Clause>> dnf;
    bool dnf_ok = false;
    // the learned estimator's clause records, built on first use (under mu)
    bool feat_built = false, feat_ok = false;
    int32_t feat_max_col = -1;
    std::vector<uint8_t> feat_rec;
    std::vector<uint64_t> feat_keys;
    std::string text;
    // lazily uploaded device blob: ProgDesc | Instr[] | pool
    std::mutex mu;
    void* d_blob = nullptr;
    uint32_t blob_bytes = 0, instr_off = 0, pool_off = 0;
};

// Builds the host blob of a list of programs (slots already remapped).
// outs[i]: output index of program i (empty: i).
void build_blob(const std::vector<const sel::Program*>& progs, const std::vector<std::vector<int32_t>>& slot_maps,
                std::vector<uint8_t>& blob, uint32_t& instr_off, uint32_t& pool_off,
                const std::vector<uint32_t>& outs = {});

// Uploads the single-program blob of a predicate (first use).
sel_status pred_upload(const sel_pred* p);

namespace sel {
// The CUDA stream a context is bound to.
cudaStream_t ctx_stream(sel_ctx* ctx);

// Kernels launched by this host thread from the estimator's code.  The
// estimator's entry points add what they launched to their context's launch
// count (sel_ctx_launch_count) through a LaunchTally; when one entry point
// calls another, only the outermost tally adds.
uint64_t& thread_launches();
int& thread_tally_depth();
void ctx_add_launches(sel_ctx* ctx, uint64_t n);
struct LaunchTally {
    sel_ctx* ctx;
    uint64_t start;
    bool outer;
    explicit LaunchTally(sel_ctx* c) : ctx(c), start(thread_launches()), outer(thread_tally_depth()++ == 0) {}
    ~LaunchTally() {
        --thread_tally_depth();
        if (outer && ctx) ctx_add_launches(ctx, thread_launches() - start);
    }
    LaunchTally(const LaunchTally&) = delete;
    LaunchTally& operator=(const LaunchTally&) = delete;
};
}
