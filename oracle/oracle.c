/*
 * oracle.c -- plain, slow, row-by-row CPU oracle for exact selectivity
 * computation and selection push-down.  TEST INFRASTRUCTURE ONLY: it is
 * loaded by the tests, by __graft_entry__.smoke() and by the bench's CPU
 * baseline, never by the library's product path.  It shares no code, header
 * or table with the CUDA library.
 *
 * What it computes (Ch3 §3.1 "Selectivity Computation", the COUNT query
 * built over the pushed-down selection; §3.3 "Materialization"; Algorithm 1,
 * function Execute):
 *
 *   count(P, R)        = |{ i in [0, n) : P(R[i]) }|                  (exact u64)
 *   select(P, R)       = ascending list of i with P(R[i])             (row ids of sigma_P(R))
 *   pushdown status    = TOO_LARGE iff count > maxSize  (Algorithm 1, Execute: "count > maxSize")
 *
 * The predicate is evaluated for every row by a recursive walk over the
 * UNCOMPILED tree: AND/OR/NOT nodes and leaf comparisons, exactly as written
 * in the query's WHERE clause (§1.1 listing "Selection with complicate
 * predicates", §3.1 listing "Selectivity computation").
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   - no NULLs: two-valued logic;
 *   - float32 columns are compared to float32 constants with IEEE-754 ordered
 *     compares in binary32 (no promotion, no fast-math);
 *   - integer-like columns (int32, int64, date, dictionary code) are compared
 *     to 64-bit integer constants after widening the value to 64 bits;
 *   - BETWEEN is inclusive on both ends; lo > hi selects nothing;
 *   - IN is set membership; an empty list is FALSE;
 *   - LIKE 'p%' on a dictionary column: byte-wise, case-sensitive prefix test
 *     of the row's dictionary string; a code outside [0, dict_size) is no
 *     match; an empty prefix matches every in-range code.
 *
 * Build: gcc -O2 -fPIC -shared -pthread oracle.c -o liboracle.so
 * (no -ffast-math: float compares must stay IEEE).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_AND = 1, O_OR = 2, O_NOT = 3, O_CMP = 4, O_BETWEEN = 5, O_IN = 6, O_LIKE = 7,
       O_TRUE = 8, O_FALSE = 9 };
enum { O_EQ = 0, O_NE = 1, O_LT = 2, O_LE = 3, O_GT = 4, O_GE = 5 };
enum { T_I32 = 0, T_I64 = 1, T_F32 = 2, T_DATE = 3, T_DICT = 4 };

typedef struct {
    int32_t type;
    int32_t n_dict;
    const void* data;
    const char* const* dict;      /* NUL-terminated strings, dictionary code -> string */
} ocol;

typedef struct {
    int32_t kind;
    int32_t col;
    int32_t op;
    int32_t n_child;
    const int32_t* child;         /* indices of the children in the node array */
    int64_t i0, i1;               /* integer constants (CMP: i0; BETWEEN: i0..i1) */
    float f0, f1;                 /* float32 constants */
    int32_t n_vals;
    const int64_t* ivals;         /* IN list, integer-like column */
    const float* fvals;           /* IN list, float32 column */
    const char* prefix;           /* LIKE prefix */
} onode;

static int64_t ival(const ocol* c, int64_t row) {
    if (c->type == T_I64) return ((const int64_t*)c->data)[row];
    return (int64_t)((const int32_t*)c->data)[row];
}

static int cmp_int(int op, int64_t v, int64_t k) {
    switch (op) {
    case O_EQ: return v == k;
    case O_NE: return v != k;
    case O_LT: return v < k;
    case O_LE: return v <= k;
    case O_GT: return v > k;
    case O_GE: return v >= k;
    }
    return 0;
}

static int cmp_flt(int op, float v, float k) {
    switch (op) {
    case O_EQ: return v == k;
    case O_NE: return v != k;
    case O_LT: return v < k;
    case O_LE: return v <= k;
    case O_GT: return v > k;
    case O_GE: return v >= k;
    }
    return 0;
}

/* P(R[row]) for the sub-tree rooted at node idx. */
static int eval_node(const onode* nodes, int32_t idx, const ocol* cols, int64_t row) {
    const onode* nd = &nodes[idx];
    const ocol* c = (nd->col >= 0) ? &cols[nd->col] : NULL;
    switch (nd->kind) {
    case O_TRUE: return 1;
    case O_FALSE: return 0;
    case O_AND:
        for (int32_t i = 0; i < nd->n_child; i++)
            if (!eval_node(nodes, nd->child[i], cols, row)) return 0;
        return 1;
    case O_OR:
        for (int32_t i = 0; i < nd->n_child; i++)
            if (eval_node(nodes, nd->child[i], cols, row)) return 1;
        return 0;
    case O_NOT:
        return !eval_node(nodes, nd->child[0], cols, row);
    case O_CMP:
        if (c->type == T_F32) return cmp_flt(nd->op, ((const float*)c->data)[row], nd->f0);
        return cmp_int(nd->op, ival(c, row), nd->i0);
    case O_BETWEEN:
        if (c->type == T_F32) {
            float v = ((const float*)c->data)[row];
            return nd->f0 <= v && v <= nd->f1;
        } else {
            int64_t v = ival(c, row);
            return nd->i0 <= v && v <= nd->i1;
        }
    case O_IN:
        if (c->type == T_F32) {
            float v = ((const float*)c->data)[row];
            for (int32_t i = 0; i < nd->n_vals; i++)
                if (v == nd->fvals[i]) return 1;
            return 0;
        } else {
            int64_t v = ival(c, row);
            for (int32_t i = 0; i < nd->n_vals; i++)
                if (v == nd->ivals[i]) return 1;
            return 0;
        }
    case O_LIKE: {
        int32_t code = ((const int32_t*)c->data)[row];
        if (code < 0 || code >= c->n_dict) return 0;
        size_t m = strlen(nd->prefix);
        return strncmp(c->dict[code], nd->prefix, m) == 0;
    }
    }
    return 0;
}

uint64_t oracle_count(const onode* nodes, int32_t root, const ocol* cols,
                      int64_t row_begin, int64_t row_end) {
    uint64_t n = 0;
    for (int64_t i = row_begin; i < row_end; i++)
        n += (uint64_t)eval_node(nodes, root, cols, i);
    return n;
}

/* Writes the ascending row ids i in [row_begin, row_end) with P(R[i]) into
 * out (capacity cap); returns the number of such rows (which may exceed cap:
 * only the first cap are written). */
int64_t oracle_select(const onode* nodes, int32_t root, const ocol* cols,
                      int64_t row_begin, int64_t row_end, int64_t* out, int64_t cap) {
    int64_t k = 0;
    for (int64_t i = row_begin; i < row_end; i++) {
        if (eval_node(nodes, root, cols, i)) {
            if (k < cap) out[k] = i;
            k++;
        }
    }
    return k;
}

/* ---- the same two functions split over host threads by row range ---- */

typedef struct {
    const onode* nodes; int32_t root; const ocol* cols;
    int64_t b, e; int64_t* out; int64_t cap; int64_t result;
} job;

static void* count_job(void* p) {
    job* j = (job*)p;
    j->result = (int64_t)oracle_count(j->nodes, j->root, j->cols, j->b, j->e);
    return NULL;
}

static void* select_job(void* p) {
    job* j = (job*)p;
    j->result = oracle_select(j->nodes, j->root, j->cols, j->b, j->e, j->out, j->cap);
    return NULL;
}

static void split(int64_t b, int64_t e, int t, int T, int64_t* jb, int64_t* je) {
    int64_t n = e - b;
    *jb = b + n * t / T;
    *je = b + n * (t + 1) / T;
}

uint64_t oracle_count_mt(const onode* nodes, int32_t root, const ocol* cols,
                         int64_t row_begin, int64_t row_end, int32_t n_threads) {
    if (n_threads < 1) n_threads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    job* js = (job*)calloc((size_t)n_threads, sizeof(job));
    for (int t = 0; t < n_threads; t++) {
        js[t].nodes = nodes; js[t].root = root; js[t].cols = cols;
        split(row_begin, row_end, t, n_threads, &js[t].b, &js[t].e);
        pthread_create(&th[t], NULL, count_job, &js[t]);
    }
    uint64_t total = 0;
    for (int t = 0; t < n_threads; t++) {
        pthread_join(th[t], NULL);
        total += (uint64_t)js[t].result;
    }
    free(th);
    free(js);
    return total;
}

/* Two passes: per-range counts, then each range writes at its offset. */
int64_t oracle_select_mt(const onode* nodes, int32_t root, const ocol* cols,
                         int64_t row_begin, int64_t row_end, int64_t* out, int64_t cap,
                         int32_t n_threads) {
    if (n_threads < 1) n_threads = 1;
    pthread_t* th = (pthread_t*)calloc((size_t)n_threads, sizeof(pthread_t));
    job* js = (job*)calloc((size_t)n_threads, sizeof(job));
    for (int t = 0; t < n_threads; t++) {
        js[t].nodes = nodes; js[t].root = root; js[t].cols = cols;
        split(row_begin, row_end, t, n_threads, &js[t].b, &js[t].e);
        pthread_create(&th[t], NULL, count_job, &js[t]);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    int64_t off = 0;
    for (int t = 0; t < n_threads; t++) {
        int64_t c = js[t].result;
        js[t].out = out + (off < cap ? off : cap);
        js[t].cap = (off < cap) ? ((cap - off) < c ? (cap - off) : c) : 0;
        off += c;
        pthread_create(&th[t], NULL, select_job, &js[t]);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
    free(th);
    free(js);
    return off;
}
