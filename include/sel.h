/*
 * sel.h -- exact selectivity computation and selection push-down on one GPU.
 *
 * The method (Ch3 "A Novel Query Optimization Paradigm"): instead of
 * estimating the cardinality of a pushed-down selection from statistics, the
 * optimiser runs SELECT COUNT(*) FROM R WHERE <pushed-down predicates> during
 * optimisation (§3.1 "Selectivity Computation"), compares the exact count with
 * maxSize = R.size * PUSH_DOWN_MAX_SELECTIVITY and, if the count is not above
 * it, materialises sigma_P(pi_cols(R)) right away while R's scan is still on
 * the GPU (§3.3 "Materialization"; Algorithm 1, functions Execute and
 * EvaluateAndPushDown).
 *
 * Conventions for every entry point:
 *  - All functions return sel_status; no exception ever crosses this ABI.
 *    sel_last_error() gives a human-readable reason for the last non-OK
 *    status on the calling host thread.
 *  - Column data are BORROWED device pointers (e.g. from torch tensors); the
 *    library never frees them.  Columns are plain arrays of n_rows elements:
 *    int32 (SEL_I32, SEL_DATE, SEL_DICT) / int64 (SEL_I64) / binary32
 *    (SEL_F32).  A base address that is 16-byte aligned takes the fast bulk
 *    (TMA) path; any element-aligned address is accepted.
 *  - sel_ctx, sel_pred and sel_batch_plan are library-owned handles, released
 *    with sel_ctx_destroy / sel_pred_free / sel_batch_plan_free.
 *  - A context binds one CUDA stream; all device work of a call is enqueued
 *    on it.  Synchronous calls (sel_count, sel_pushdown, sel_count_batch,
 *    sel_batch_plan_run with host output) return after the result is on the
 *    host.  Use one context per host thread.
 *  - Row counts and row ids are 64-bit everywhere.
 */
#ifndef SEL_H
#define SEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sel_status {
    SEL_OK = 0,
    SEL_ERR_INVALID_ARG = 1,   /* null pointer, bad size, malformed tree, bad column index   */
    SEL_ERR_TYPE = 2,          /* constant or operator does not fit the column's type        */
    SEL_ERR_UNSUPPORTED = 3,   /* a documented limit is exceeded (tree depth, list sizes ...) */
    SEL_ERR_OOM = 4,           /* a device or pinned-host allocation failed                  */
    SEL_ERR_CUDA = 5,          /* a CUDA runtime call failed (no device, launch error ...)    */
    SEL_ERR_TOO_LARGE = 6,     /* push-down: count > max_rows (Algorithm 1's thrown exception) */
    SEL_ERR_TIMEOUT = 7        /* a bounded device-side wait gave up; results are invalid      */
} sel_status;

typedef enum sel_type {
    SEL_I32 = 0,   /* int32                                                          */
    SEL_I64 = 1,   /* int64                                                          */
    SEL_F32 = 2,   /* IEEE-754 binary32; compared in binary32 without promotion       */
    SEL_DATE = 3,  /* int32 days since 1970-01-01, compared as an integer             */
    SEL_DICT = 4   /* int32 code into a dictionary of strings (code -> string)         */
} sel_type;

/* One column.  dict/dict_size describe a SEL_DICT column's dictionary (host
 * strings, NUL-terminated, entry i is the string of code i); they are only
 * read by sel_compile_predicate (to resolve LIKE) and may be NULL when no
 * LIKE refers to the column.  A byte-wise sorted dictionary turns a prefix
 * into one code range; an unsorted one into a code bitmap. */
typedef struct sel_column {
    int32_t type;                 /* sel_type                                   */
    int32_t dict_size;            /* SEL_DICT only                              */
    const void* data;             /* device pointer to n_rows elements          */
    const char* const* dict;      /* SEL_DICT only, host, may be NULL           */
} sel_column;

typedef struct sel_table {
    const sel_column* cols;       /* host array of n_cols descriptors           */
    int32_t n_cols;
    int64_t n_rows;               /* >= 0                                       */
} sel_table;

/* Predicate trees are passed as a flat POSTFIX array of nodes (children
 * before their parent), the WHERE clause of the COUNT query of §3.1.
 * Leaves: comparison with a constant, BETWEEN (inclusive both ends), IN-list
 * and prefix LIKE ('prefix%': byte-wise, case-sensitive) on dictionary
 * columns.  Inner nodes: n-ary AND / OR (n_children >= 1 operands popped),
 * NOT.  Logic is two-valued (columns hold no NULLs). */
typedef enum sel_node_kind {
    SEL_N_CMP = 1,      /* col op i_lo (integer-like) / col op f_lo (SEL_F32)          */
    SEL_N_BETWEEN = 2,  /* i_lo <= col <= i_hi  /  f_lo <= col <= f_hi                 */
    SEL_N_IN = 3,       /* col in values[0 .. n_values)  (empty list: FALSE)           */
    SEL_N_LIKE = 4,     /* dictionary string of col starts with prefix                 */
    SEL_N_AND = 5,
    SEL_N_OR = 6,
    SEL_N_NOT = 7,
    SEL_N_TRUE = 8,
    SEL_N_FALSE = 9
} sel_node_kind;

typedef enum sel_op { SEL_EQ = 0, SEL_NE = 1, SEL_LT = 2, SEL_LE = 3, SEL_GT = 4, SEL_GE = 5 } sel_op;

typedef struct sel_node {
    int32_t kind;          /* sel_node_kind                                          */
    int32_t col;           /* leaves: column index in the table                      */
    int32_t op;            /* SEL_N_CMP: sel_op                                       */
    int32_t n_children;    /* SEL_N_AND / SEL_N_OR: operands popped (>= 1)            */
    int64_t i_lo, i_hi;    /* integer constants (int32/int64/date/dict columns)      */
    float f_lo, f_hi;      /* binary32 constants (SEL_F32 columns)                    */
    int32_t n_values;      /* SEL_N_IN: number of values (<= SEL_MAX_IN_VALUES)       */
    int32_t reserved;
    const void* values;    /* SEL_N_IN: host int64_t[] (integer-like) / float[] (F32) */
    const char* prefix;    /* SEL_N_LIKE: NUL-terminated literal prefix (no wildcard)  */
} sel_node;

#define SEL_MAX_NODES 512         /* postfix nodes per predicate                       */
#define SEL_MAX_LEAVES 64         /* leaves per predicate                              */
#define SEL_MAX_IN_VALUES 4096    /* values per IN list                                */
#define SEL_MAX_SLOTS 16          /* distinct columns referenced by one predicate      */

typedef struct sel_ctx sel_ctx;
typedef struct sel_pred sel_pred;
typedef struct sel_batch_plan sel_batch_plan;

/* Last error message of the calling host thread ("" if none). */
const char* sel_last_error(void);
const char* sel_status_str(sel_status s);

/* Create a context bound to a CUDA stream (a cudaStream_t; NULL = the legacy
 * default stream) on the current device.  The context owns small device
 * scratch (result counters, error flag, tile status of the push-down scan,
 * row masks of the two-pass push-down, grown on demand) and pinned host
 * buffers for results.  It also sets the calling process's L2 fetch
 * granularity hint on the device (cudaLimitMaxL2FetchGranularity) to 32
 * bytes: the push-down's gathers of single values then read a quarter of the
 * DRAM bytes.  The hint belongs to the process's CUDA context, ends with it,
 * and can be changed back with cudaDeviceSetLimit. */
sel_status sel_ctx_create(void* cuda_stream, sel_ctx** out);
void sel_ctx_destroy(sel_ctx* ctx);

/* a1 -- compile a postfix tree against a table schema (column types and
 * dictionaries; data pointers and n_rows are not read).  Host-only work: NOT
 * is pushed to the leaves (negation normal form), comparisons become
 * inclusive ranges of the column's type, LIKE becomes a code range or bitmap,
 * operands are ordered to bound the evaluation stack.  The program is
 * uploaded to the device on first use.  Errors: SEL_ERR_INVALID_ARG
 * (malformed postfix, column out of range), SEL_ERR_TYPE (LIKE on a non-dict
 * column, dict needed but absent), SEL_ERR_UNSUPPORTED (limits above). */
sel_status sel_compile_predicate(const sel_table* schema, const sel_node* postfix, int32_t n_nodes,
                                 sel_pred** out);
void sel_pred_free(sel_pred* pred);

/* Text dump of the compiled program (for tests and debugging); writes at most
 * cap bytes including the terminating NUL and returns SEL_OK. */
sel_status sel_pred_describe(const sel_pred* pred, char* buf, int64_t cap);

/* a2 -- exact count = |{ i in [0, n_rows) : P(row i) }| (§3.1 COUNT query).
 * The table must have the column types the predicate was compiled for.
 * Synchronous: *out_count (host) holds the count on SEL_OK. */
sel_status sel_count(sel_ctx* ctx, const sel_pred* pred, const sel_table* table, uint64_t* out_count);

/* Same scan, enqueued only: the count is written to dev_out_count (device,
 * 8 bytes, caller-owned) when the stream reaches it.  A timed-out device wait
 * is reported by the next synchronous call on this context. */
sel_status sel_count_async(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                           uint64_t* dev_out_count);

/* a3 + a4 -- selection push-down (Algorithm 1, Execute with isSPD = true):
 * computes the exact count and writes the rows of sigma_P(R) (in two passes
 * or one fused pass: sel_ctx_set_pushdown_method),
 * projected on proj_cols[0 .. n_proj), in ascending row order
 * into caller-allocated device buffers dev_out_cols[j] (capacity max_rows
 * elements of column proj_cols[j]'s type), plus their int64 row ids into
 * dev_out_rowids when it is not NULL.  *out_count (host) always receives the
 * exact count.  If count > max_rows the call returns SEL_ERR_TOO_LARGE (the
 * paper's thrown exception: the caller reverts the push-down) and the output
 * buffers hold unspecified data; nothing is written beyond max_rows
 * elements.  Synchronous. */
sel_status sel_pushdown(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                        const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                        int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* out_count);

/* Same push-down, enqueued only: the exact count is written to dev_out_count
 * (device, 8 bytes) and nothing waits for it; the caller compares it with
 * max_rows (rows past max_rows are never written).  A timed-out device wait
 * (a look-back, or a stage of the scan) is reported by sel_ctx_synchronize.
 * The two-pass method keeps its scratch in the context: calls on one
 * context run in its stream's order. */
sel_status sel_pushdown_async(sel_ctx* ctx, const sel_pred* pred, const sel_table* table,
                              const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                              int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* dev_out_count);

/* Push-down for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a library convenience).  Some callers must not call
 * cudaMalloc: code that runs inside its own device memory manager (a
 * database buffer pool, an allocator callback) where a nested allocation
 * would re-enter that manager or break its accounting, and latency-critical
 * query pipelines where an allocation may synchronise the whole device.
 * This entry point needs no sel_ctx and makes no cudaMalloc / cudaFree or
 * other allocating call: its scratch (look-back status words, tile counter,
 * program) lives in one fixed 4 MiB __device__ array inside the library,
 * which every GPU that loads the library holds until exit.  The compiled
 * program is handed to the GPU as kernel parameters (a copy kernel per
 * 16 KiB), so no host buffer is read after the call returns.
 * Limit: the table may have at most 516,064 tiles of 1024 rows, i.e.
 * 528,449,536 rows; larger tables and programs above 64 KiB return
 * SEL_ERR_UNSUPPORTED with a message.  The caller passes the stream
 * (cudaStream_t, NULL = legacy default stream), the inputs, and all outputs,
 * all caller-owned device memory: dev_out_cols / dev_out_rowids as for
 * sel_pushdown, dev_out_count (8 bytes, receives the exact count; compare it
 * with max_rows -- rows past max_rows are never written) and dev_out_error
 * (4 bytes, required: NULL gives SEL_ERR_INVALID_ARG; nonzero after the
 * stream reaches the end of the call means a look-back wait timed out and
 * the count and rows are invalid).  Enqueue only: nothing waits for the GPU.
 * The first call on each device looks up the array's device address, so make
 * that first call before any stream capture; later calls can be captured in
 * a CUDA graph (the graph holds the program).  All calls share the one array:
 * each call clears the parts that must start at zero, and calls that overlap
 * on the GPU (different streams, or different host threads on one device)
 * race on it -- order them on one stream. */
sel_status sel_pushdown_noalloc(void* cuda_stream, const sel_pred* pred, const sel_table* table,
                                const int32_t* proj_cols, int32_t n_proj, void* const* dev_out_cols,
                                int64_t* dev_out_rowids, uint64_t max_rows, uint64_t* dev_out_count,
                                uint32_t* dev_out_error);

/* a5 -- batched probes: counts of n predicates, preds[i] evaluated over
 * tables[i], in one persistent launch that reads every referenced column of
 * each distinct table once for all predicates on that table (tables are the
 * same when their descriptors point to the same column data and n_rows).
 * The launch shape (tile rows, pipeline stages, CTAs per SM) is picked by
 * the library's autotuner on first use of the plan and the launch is
 * captured in a CUDA graph that later runs replay.  out_counts: host, n. */
sel_status sel_count_batch(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                           int32_t n, uint64_t* out_counts);

/* Same as sel_count_batch, enqueued only: counts go to dev_out_counts
 * (device, n u64).  Plans are cached per context by the compiled programs'
 * content and the tables' column pointers, so recompiling the same probes
 * reuses the tuned shape and the captured graph. */
sel_status sel_count_batch_async(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                                 int32_t n, uint64_t* dev_out_counts);

/* Waits for all work enqueued on the context's stream and reports (then
 * clears) a device wait that timed out in an enqueue-only call since the
 * last check: SEL_ERR_TIMEOUT. */
sel_status sel_ctx_synchronize(sel_ctx* ctx);

/* The plan behind sel_count_batch, for callers that run the same probe set
 * many times.  The predicates and table descriptors must outlive the plan.
 * autotune: 1 = time the candidate launch shapes now and keep the fastest,
 * 0 = use the default shape.  A plan with more than 256 probes on one table
 * runs as parts of at most 256 probes a table, one launch each (all in its
 * graph), which add into the same counts; sel_batch_plan_kernel, _info and
 * _variant then report the first part. */
sel_status sel_batch_plan_create(sel_ctx* ctx, const sel_pred* const* preds, const sel_table* const* tables,
                                 int32_t n, int32_t autotune, sel_batch_plan** out);
/* Runs the plan: counts to dev_out_counts (device, n u64, enqueue only) when
 * it is not NULL, else to host_out_counts (synchronous).  With a device
 * buffer the replayed graph's kernel writes the counts straight into it: the
 * first run with a buffer captures that graph (the plan keeps the graphs of
 * its last 4 buffers), later runs are one graph launch. */
sel_status sel_batch_plan_run(sel_batch_plan* plan, uint64_t* dev_out_counts, uint64_t* host_out_counts);
/* Launch shape chosen by the plan and its measured time per launch (ms, 0 if
 * not autotuned). */
sel_status sel_batch_plan_info(const sel_batch_plan* plan, int32_t* tile_rows, int32_t* stages,
                               int32_t* ctas_per_sm, float* ms);
/* Count-scan kernel variant chosen by the plan (see sel_ctx_set_scan_variant). */
sel_status sel_batch_plan_variant(const sel_batch_plan* plan, int32_t* consumer_warps, int32_t* chunks_per_pass);
/* The kernel the plan runs: 0 = the program interpreter (count.cu), 1 = the
 * column-bucket kernel (bucket_count.cu): every predicate taken to an OR of at
 * most 4 AND-groups, each row's bucket per referenced column found once, and
 * every probe's leaves read from per-bucket group masks.  Both give the same
 * exact counts; plan creation picks the faster (measured when autotuning,
 * else the bucket kernel whenever the probes fit it). */
sel_status sel_batch_plan_kernel(const sel_batch_plan* plan, int32_t* kernel);
/* Which kernels later batch plans of this context may use: 0 = the faster of
 * both (default), 1 = the interpreter only, 2 = the bucket kernel only
 * (plans whose probes do not fit it fail with SEL_ERR_UNSUPPORTED).  Clears
 * the context's cache of sel_count_batch plans. */
sel_status sel_ctx_set_batch_kernel(sel_ctx* ctx, int32_t mode);
void sel_batch_plan_free(sel_batch_plan* plan);

/* Launch configuration override for sel_count / sel_count_async / sel_pushdown
 * (0 = keep the library default: 3 stages of the largest tile that fits in
 * shared memory).  tile_rows must be a multiple of 256 and at most 16384; a
 * larger tile than fits is shrunk.  The push-down's persistent kernel takes
 * tiles that are whole chunk groups (256 x chunks_per_pass rows); other
 * tiles run on its one-CTA-per-tile kernel, which uses at most 4096 rows. */
sel_status sel_ctx_set_scan_shape(sel_ctx* ctx, int32_t tile_rows, int32_t stages, int32_t ctas_per_sm);

/* Count-scan kernel variant for sel_count / sel_count_async (both 0 = the
 * library default): consumer_warps 8 or 16 (plus one producer warp per CTA)
 * and chunks_per_pass 1 or 2 (256-row chunks a warp evaluates with one pass
 * over the program's instructions), 8 warps with 4 chunks per pass, or 15
 * warps with 2 or 3 chunks per pass.  Any other pair: SEL_ERR_INVALID_ARG.
 * The same pair selects the persistent push-down kernel's consumer warps and
 * chunks per pass where that kernel has the variant (8, 12 or 16 warps, 1 or
 * 2 chunks, and 12 x 3; default 12 x 3, or 12 x 2 for a requested tile that is
 * not a multiple of 768 rows; with 8 x 4 the push-down keeps its default).
 * The batch plans' column-bucket kernel also takes 11 or 15 consumer warps
 * (1 or 2 chunks per pass), and the push-down 12 warps (1, 2 or 3 chunks); with pairs a kernel
 * does not have, sel_count, sel_pushdown and the batch plans keep their
 * defaults.  Results do not depend on the variant. */
sel_status sel_ctx_set_scan_variant(sel_ctx* ctx, int32_t consumer_warps, int32_t chunks_per_pass);

/* Number of kernels this context has launched so far (all entry points). */
uint64_t sel_ctx_launch_count(const sel_ctx* ctx);

/* Super-tile size of the persistent push-down kernel (its look-back unit,
 * Algorithm 1's output offsets are found per super-tile): the largest multiple
 * of the kernel's sub-tile that is at most `rows` rows.  0 (the default):
 * 384 KB of the predicate's columns, but at most 1/16 of a CTA's share of the
 * table, and at least 32768 and at most 131072 rows.  rows must be
 * 0 or a multiple of 256 up to 131072, else SEL_ERR_INVALID_ARG.  Results do
 * not depend on it. */
sel_status sel_ctx_set_pushdown_super_rows(sel_ctx* ctx, int32_t rows);

/* Push-down method of sel_pushdown / sel_pushdown_async; results do not
 * depend on it.
 *   SEL_PD_AUTO      (0, the default) the library's choice: two passes.
 *   SEL_PD_TWO_PASS  (1) the count scan (sel_count's kernel and launch shape)
 *                    also stores each 256-row chunk's row mask and count and
 *                    each 16384-row segment's count (1/8 byte per row plus
 *                    2 bytes per chunk of context scratch); a one-CTA kernel
 *                    turns the segment counts into output offsets; a scatter
 *                    kernel (one warp per segment) writes the selected rows.
 *                    No device wait on another CTA.
 *   SEL_PD_ONE_PASS  (2) count and compaction in one pass: the persistent
 *                    kernel, output offsets by decoupled look-back over
 *                    super-tiles (sel_ctx_set_pushdown_super_rows), or the
 *                    one-CTA-per-tile kernel for tile sizes the persistent
 *                    kernel does not take (sel_ctx_set_scan_shape).
 * Any other value: SEL_ERR_INVALID_ARG. */
enum { SEL_PD_AUTO = 0, SEL_PD_TWO_PASS = 1, SEL_PD_ONE_PASS = 2 };
sel_status sel_ctx_set_pushdown_method(sel_ctx* ctx, int32_t method);

/* Timing hook: when cuda_event (a cudaEvent_t of the context's device) is
 * not NULL, every two-pass push-down enqueued on this context records it on
 * the context's stream between its count pass and the rest (offsets and
 * scatter), so that the caller can time the passes separately with events of
 * its own before and after the call.  The event is recorded when the call
 * enqueues its work; NULL (the default) turns the hook off.  The caller owns
 * the event and clears the hook before destroying it. */
sel_status sel_ctx_set_pushdown_split_event(sel_ctx* ctx, void* cuda_event);

/* Test hook for the bounded waits of the push-down look-back (SEL_PD_ONE_PASS): look-back unit
 * skip_tile (a super-tile of the persistent kernel -- see
 * sel_ctx_set_pushdown_super_rows --, a tile of the one-CTA-per-tile kernel;
 * -1: none) never publishes its prefix, and a waiting tile gives up after
 * wait_ns nanoseconds (0: the default of 2 s), so that later sel_pushdown
 * calls on this context return SEL_ERR_TIMEOUT instead of waiting forever.
 * The context stays usable; set skip_tile back to -1 to disarm. */
sel_status sel_ctx_debug_pushdown_fault(sel_ctx* ctx, int64_t skip_tile, uint64_t wait_ns);

/* ---------------------------------------------------------------------------
 * Join-size estimate (§1.1, §3.2): |R join S| = |R||S| / max(V(R,A), V(S,A)),
 * V(R, A) the number of distinct values of the join attribute.
 * ------------------------------------------------------------------------- */

/* V(sigma_P(R), col): distinct values of column `col` over the rows that
 * satisfy `pred` (NULL: all rows), and (when out_rows is not NULL) the number
 * of those rows.  float32 -0.0 and +0.0 count as one value.  With a predicate
 * the selected values are compacted by the push-down first.  Device scratch
 * (owned by the context): the selected values and a hash set of at least
 * twice as many 8-byte slots.  Synchronous. */
sel_status sel_count_distinct(sel_ctx* ctx, const sel_table* table, int32_t col, const sel_pred* pred,
                              uint64_t* out_distinct, uint64_t* out_rows);

/* The exact COUNT(*) of sigma_P(R) join sigma_Q(S) on R.col_r = S.col_s (the
 * two-relation COUNT query of the paper's experiments, Ch5): the selected keys
 * of both sides (compacted by the push-down when a predicate is given), a
 * key -> multiplicity hash map of the side with fewer rows, probed with the
 * other side.  Keys are compared as values: both columns int32-like (int32,
 * date, dictionary code) or both int64 or both float32 (-0.0 == +0.0; a
 * float32 key with an integer key: SEL_ERR_TYPE; int32 with int64:
 * SEL_ERR_UNSUPPORTED).  out_rows_r / out_rows_s (nullable): the selected row
 * counts.  Device scratch owned by the context.  Synchronous. */
sel_status sel_join_count(sel_ctx* ctx, const sel_table* r, int32_t col_r, const sel_pred* pred_r,
                          const sel_table* s, int32_t col_s, const sel_pred* pred_s, uint64_t* out_count,
                          uint64_t* out_rows_r, uint64_t* out_rows_s);

/* rows_r * rows_s / max(distinct_r, distinct_s); 0 when both are 0. */
double sel_join_size_estimate(uint64_t rows_r, uint64_t rows_s, uint64_t distinct_r, uint64_t distinct_s);

/* ---------------------------------------------------------------------------
 * Algorithm 1, EvaluateAndPushDown (Ch4 §4.2): the push-down decision for the
 * scanned relations of one query.  Relations whose size is greater than
 * min_table_size (PUSH_DOWN_MIN_TABLE_SIZE) are ordered by size, largest
 * first (equal sizes keep their input order); the largest is the probed
 * relation and is never pushed down.  Each other one with a predicate is
 * pushed down with sel_pushdown and maxSize = floor(size * max_selectivity)
 * (PUSH_DOWN_MAX_SELECTIVITY as a ratio), or max_rows when that is not 0 (the
 * absolute form the paper also names): count > maxSize reverts the push-down
 * (its outputs are then unspecified), otherwise the projected columns of the
 * selected rows are in the relation's outputs.
 * ------------------------------------------------------------------------- */
typedef enum {
    SEL_SPD_PROBE = 0,          /* the largest relation: not pushed down */
    SEL_SPD_TOO_SMALL = 1,      /* size <= min_table_size: not considered */
    SEL_SPD_NO_PREDICATE = 2,   /* nothing to push down */
    SEL_SPD_PUSHED = 3,         /* count <= maxSize: rows materialised */
    SEL_SPD_REVERTED = 4        /* count > maxSize: push-down reverted */
} sel_spd_decision;

typedef struct {
    const sel_table* table;        /* the scanned relation (device columns) */
    const sel_pred* pred;          /* its pushed-down selection; NULL: none */
    const int32_t* proj_cols;      /* columns needed above the relation (host) */
    int32_t n_proj;
    void* const* dev_out_cols;     /* caller-owned device outputs, capacity >= maxSize rows each */
    int64_t* dev_out_rowids;       /* caller-owned, capacity >= maxSize; may be NULL */
} sel_spd_relation;

typedef struct {
    uint64_t min_table_size;       /* PUSH_DOWN_MIN_TABLE_SIZE */
    double max_selectivity;        /* PUSH_DOWN_MAX_SELECTIVITY (ratio, >= 0) */
    uint64_t max_rows;             /* absolute maxSize instead of the ratio when not 0 */
} sel_spd_cfg;

/* decisions[i] (sel_spd_decision), counts[i] (exact count of each relation that
 * was executed, else 0) and, when not NULL, max_sizes[i] are written for the n
 * relations.  Synchronous.  Errors of a push-down (other than the count being
 * too large) stop the pass and are returned. */
sel_status sel_evaluate_and_push_down(sel_ctx* ctx, const sel_spd_relation* rels, int32_t n, const sel_spd_cfg* cfg,
                                      int32_t* decisions, uint64_t* counts, uint64_t* max_sizes);

/* ---------------------------------------------------------------------------
 * Learned estimator (not in the paper, whose selectivity is always the exact
 * COUNT of §3.1): a small MLP answers from predicate features and the exact
 * batched count answers whenever the MLP's predicted uncertainty is above a
 * threshold, so exactness stays available for every probe.
 *
 * Features (a6): per column (the first 8 columns of the table) an empirical
 * CDF from sample_rows rows drawn with SplitMix64, idx_i = splitmix64(seed +
 * (col + 1) * 2^40 + i) mod n_rows.  A predicate whose negation normal form
 * is an OR of at most 3 ANDs of at most 6 leaves in total gets 144 features:
 * per leaf slot a column one-hot (8), an operator one-hot (= <> < <= > >=
 * BETWEEN IN LIKE) plus a NOT flag (10), [F_lo, F_hi] = sample fractions
 * bounding the leaf's value set (2), the AND group one-hot (3) and the leaf's
 * log selectivity ln(max(p, 1/(2m))) / ln(2m) with p = F_hi - F_lo (its
 * complement for <> and for a negated leaf).  Other predicates are "not
 * featurizable" and always answered exactly.  sel_mlp_train starts an
 * untrained model's output biases at the targets' mean and log-variance.
 * Network (a7, a8): 144 -> 256 -> 256 -> 256 (ReLU) -> 2 = (mu, log sigma^2)
 * of y = ln(1 + count); BF16 operands with FP32 accumulation on the tensor
 * cores; Gaussian negative log-likelihood; Adam on FP32 master weights.
 * ------------------------------------------------------------------------- */
typedef struct sel_mlp sel_mlp;

typedef struct sel_train_cfg {
    int32_t epochs;        /* sel_mlp_train: passes over the training predicates          */
    int32_t batch;         /* rows per minibatch, a positive multiple of 8                */
    float lr, beta1, beta2, eps;   /* Adam                                                */
    uint64_t seed;         /* minibatch shuffling                                         */
    int32_t apply_update;  /* sel_mlp_train_step: 1 = Adam step (gradients are then cleared),
                              0 = only accumulate gradients (inspect with sel_mlp_get_grads) */
    int32_t reserved;
} sel_train_cfg;

/* Builds the CDF tables from `table` (device columns; sample_rows a power of
 * two in [2, 8192]) and seeded initial weights.  The model keeps no pointer
 * to the table. */
sel_status sel_mlp_create(sel_ctx* ctx, const sel_table* table, int32_t sample_rows, uint64_t seed, sel_mlp** out);
void sel_mlp_free(sel_mlp* m);
/* a6: features of n predicates into dev_features (device BF16, n x 144,
 * caller-owned) and, when dev_ok is not NULL, 1/0 featurizable flags (device,
 * n bytes).  Predicates must be compiled against the model's table schema.
 * Asynchronous on the context's stream: the host builds the clause records,
 * copies them through a pinned staging block owned by the model (a later call
 * waits for the previous copy out of it) and launches the feature kernel. */
sel_status sel_mlp_featurize(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds, int32_t n, void* dev_features,
                             uint8_t* dev_ok);
/* a7: dev_out (device FP32, n x 2) = (mu, raw log-variance) per feature row.
 * dev_features 16-byte aligned.  Enqueued on the context's stream.  One
 * kernel runs the three hidden layers and the head for 128 rows per CTA
 * (activations in shared memory, accumulators in TMEM). */
sel_status sel_mlp_forward(sel_ctx* ctx, sel_mlp* m, const void* dev_features, int32_t n, float* dev_out);
/* Debug: on = 0 makes the model's inference (sel_mlp_forward,
 * sel_mlp_estimate) run layer by layer like the training pass (three GEMM
 * launches and a head kernel, activations through global memory) instead of
 * the fused kernel; 1 restores the default.  Both give the same bits. */
sel_status sel_debug_mlp_fused(sel_mlp* m, int32_t on);
/* a8: one minibatch (n rows, a multiple of 8) of features and targets
 * y = ln(1 + count) (device FP32): gradients of the mean Gaussian NLL, then
 * an Adam step when cfg->apply_update.  *loss_out = the batch's mean loss.
 * Synchronous. */
sel_status sel_mlp_train_step(sel_ctx* ctx, sel_mlp* m, const void* dev_features, const float* dev_y, int32_t n,
                              const sel_train_cfg* cfg, float* loss_out);
/* a8 driver: featurizes the n predicates, targets ln(1 + exact_counts[i])
 * (host), shuffled minibatches for cfg->epochs epochs (non-featurizable
 * predicates skipped).  *final_loss = mean loss of the last epoch. */
sel_status sel_mlp_train(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds, const uint64_t* exact_counts,
                         int64_t n, const sel_train_cfg* cfg, float* final_loss);
/* a9: est[i] (host) = the exact count of preds[i] over `table` when the
 * predicate is not featurizable or sigma_i = exp(lv_i / 2) > tau (lv clamped
 * to [-8, 8]); otherwise max(0, exp(mu_i) - 1).  sigma (host, may be NULL)
 * gets sigma_i (+inf when not featurizable), used_exact (host, may be NULL)
 * 1 where the exact batched scan answered.  Synchronous. */
sel_status sel_mlp_estimate(sel_ctx* ctx, sel_mlp* m, const sel_pred* const* preds, const sel_table* table,
                            int32_t n, float tau, double* est, float* sigma, uint8_t* used_exact);
/* a9 calibration of tau (the paper has no learned part; reading of the
 * uncertainty rule): given held-out predicates' sigma (as returned by
 * sel_mlp_estimate; +inf = no feature form, never accepted), the network's
 * estimates est = max(0, exp(mu) - 1) and their exact counts, *tau_out = the
 * largest sigma value t for which the `quantile`-th percentile (linear
 * interpolation between order statistics, in double) of the q-errors
 * max(e, c) / min(e, c) (e, c clamped to >= 1) of the predicates with
 * sigma <= t is at most max_q; 0 when no t qualifies (everything exact).
 * answered_out (may be NULL) = the fraction of the n predicates accepted at
 * that tau.  Host only, no GPU work; SEL_ERR_INVALID_ARG on NULL inputs or a
 * quantile outside [0, 100]. */
sel_status sel_mlp_choose_tau(const float* sigma, const double* est, const uint64_t* exact, int64_t n,
                              double max_q, double quantile, float* tau_out, double* answered_out);
/* Parameters as one FP32 array (W1 256x144, b1 256, W2 256x256, b2, W3
 * 256x256, b3, W4 2x256, b4 2; row-major, [out][in]) of sel_mlp_param_count()
 * floats.  set also clears gradients and Adam state. */
int64_t sel_mlp_param_count(void);
sel_status sel_mlp_get_params(const sel_mlp* m, float* host_params, int64_t n_floats);
sel_status sel_mlp_set_params(sel_ctx* ctx, sel_mlp* m, const float* host_params, int64_t n_floats);
sel_status sel_mlp_get_grads(const sel_mlp* m, float* host_grads, int64_t n_floats);
/* Checkpoint: weights, Adam state, step and CDF tables in one binary file. */
sel_status sel_mlp_save(const sel_mlp* m, const char* path);
sel_status sel_mlp_load(sel_ctx* ctx, const char* path, sel_mlp** out);

/* Test hook for the tensor-core matrix product behind the learned estimator
 * (the paper has none): C[M x N] = A[M x K] * B[N x K]^T with A, B row-major
 * BF16 device matrices (16-byte aligned, K a multiple of 8) and C row-major
 * FP32 (device, caller-owned), FP32 accumulation, k_splits-way split over K
 * (1..64).  Enqueued on cuda_stream; *dev_err (device, 4 bytes) becomes
 * nonzero if a bounded wait inside the kernel gave up. */
sel_status sel_debug_gemm_bf16(void* cuda_stream, const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                               float* C, int32_t k_splits, uint32_t* dev_err);

/* Test hook for allocation failures (failure injection on the host; no GPU
 * fault): the nth device or pinned-host allocation the library makes from
 * now on (1 = the next one; process-wide, every context and thread) fails as
 * if the device were out of memory, without allocating; the entry point that
 * made it returns SEL_ERR_OOM and frees what it had allocated, and the
 * context stays usable.  0 disarms; negative: SEL_ERR_INVALID_ARG.  The hook
 * fires once. */
sel_status sel_debug_fail_allocation(int64_t nth);

/* Test hook for the column-bucket form of a batch (host only, no GPU): the
 * exact counts of preds[0..n) over `table`, whose column pointers are HOST
 * memory here, evaluated on the CPU from the same bucket tables the GPU
 * kernel reads (counts: host, n entries; n_blocks, may be NULL: blocks of 64
 * probes the form used; n_quads, may be NULL: quads of 4 blocks when the
 * table took the quad form, else 0).  SEL_ERR_UNSUPPORTED (message in
 * sel_last_error) when the probes do not fit the form. */
sel_status sel_debug_bucket_count_host(const sel_pred* const* preds, int32_t n, const sel_table* table,
                                       uint64_t* counts, int32_t* n_blocks, int32_t* n_quads);

#ifdef __cplusplus
}
#endif

#endif /* SEL_H */
