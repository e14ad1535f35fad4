// spd.cpp -- Algorithm 1, EvaluateAndPushDown: the selective selection
// push-down decision for the scanned relations of one query (Ch4 §4.2).
//
// Relations larger than PUSH_DOWN_MIN_TABLE_SIZE go into a priority queue by
// size (largest first; equal sizes in input order).  The largest one is the
// relation to be probed and is never pushed down.  Every other one with a
// pushed-down selection is executed with isSPD: its exact count is taken,
// and when the count is above maxSize (= floor(size x PUSH_DOWN_MAX_SELECTIVITY),
// or an absolute maxSize) the push-down is reverted, otherwise the selected
// rows of the projected columns are materialised.  Count and materialisation
// are one pass of the push-down kernel (sel_pushdown).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

extern "C" sel_status sel_evaluate_and_push_down(sel_ctx* ctx, const sel_spd_relation* rels, int32_t n,
                                                 const sel_spd_cfg* cfg, int32_t* decisions, uint64_t* counts,
                                                 uint64_t* max_sizes) {
    using namespace sel;
    if (!ctx || !cfg || n < 0 || (n > 0 && (!rels || !decisions || !counts)) ||
        !(cfg->max_selectivity >= 0.0) || !std::isfinite(cfg->max_selectivity)) {
        set_error("sel_evaluate_and_push_down: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    std::vector<int32_t> queue;
    for (int32_t i = 0; i < n; ++i) {
        if (!rels[i].table) {
            set_error("sel_evaluate_and_push_down: relation %d has no table", i);
            return SEL_ERR_INVALID_ARG;
        }
        decisions[i] = SEL_SPD_TOO_SMALL;
        counts[i] = 0;
        if (max_sizes) max_sizes[i] = 0;
        if ((uint64_t)rels[i].table->n_rows > cfg->min_table_size) queue.push_back(i);
    }
    std::stable_sort(queue.begin(), queue.end(),
                     [&](int32_t a, int32_t b) { return rels[a].table->n_rows > rels[b].table->n_rows; });
    if (queue.empty()) return SEL_OK;
    decisions[queue[0]] = SEL_SPD_PROBE;   // the largest relation is probed, never pushed down
    for (size_t qi = 1; qi < queue.size(); ++qi) {
        const int32_t i = queue[qi];
        const sel_spd_relation& r = rels[i];
        if (!r.pred) {
            decisions[i] = SEL_SPD_NO_PREDICATE;
            continue;
        }
        const uint64_t size = (uint64_t)r.table->n_rows;
        const uint64_t max_size =
            cfg->max_rows ? cfg->max_rows : (uint64_t)std::floor((double)size * cfg->max_selectivity);
        if (max_sizes) max_sizes[i] = max_size;
        uint64_t count = 0;
        const sel_status s = sel_pushdown(ctx, r.pred, r.table, r.proj_cols, r.n_proj, r.dev_out_cols,
                                          r.dev_out_rowids, max_size, &count);
        counts[i] = count;
        if (s == SEL_ERR_TOO_LARGE) {
            decisions[i] = SEL_SPD_REVERTED;   // count > maxSize: keep the selection above the joins
        } else if (s == SEL_OK) {
            decisions[i] = SEL_SPD_PUSHED;
        } else {
            return s;
        }
    }
    return SEL_OK;
}
