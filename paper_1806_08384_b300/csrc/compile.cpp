// compile.cpp -- predicate compiler (host).
//
// Turns the WHERE clause of the §3.1 COUNT query, given as a postfix array of
// sel_node, into the program the scan kernels interpret:
//   1. parse the postfix array into a tree, checking arity;
//   2. push NOT down to the leaves (negation normal form; exact in the
//      two-valued logic of NULL-free columns);
//   3. lower each leaf to one device operation on the column's own type:
//      comparisons and BETWEEN become inclusive ranges intersected with the
//      type's value range, IN becomes a range / bitmap / value list, prefix
//      LIKE becomes the dictionary codes whose string starts with the prefix
//      (one code range for a sorted dictionary, else a bitmap);
//   4. fold constants, flatten nested AND / OR, order operands by the stack
//      depth they need (Sethi-Ullman) and emit postfix instructions.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <sstream>

#include "internal.h"

namespace sel {
namespace {

typedef __int128 i128;

enum { K_AND = 1, K_OR, K_NOT, K_LEAF, K_TRUE, K_FALSE };

struct TNode {
    int kind;
    bool neg = false;
    std::vector<int> kids;
    const sel_node* src = nullptr;
};

struct Leaf {          // a lowered leaf, or a constant
    bool is_const = false;
    bool cval = false;
    Instr ins{};
    std::vector<uint8_t> pool;
    int col = -1;
};

struct ENode {
    int kind;          // K_AND / K_OR / K_LEAF / K_TRUE / K_FALSE
    Leaf leaf;
    std::vector<ENode> kids;
    int need = 1;
};

struct Fail {
    sel_status st;
    std::string msg;
};

[[noreturn]] void fail(sel_status st, const std::string& m) { throw Fail{st, m}; }

template <typename T>
void put(std::vector<uint8_t>& v, T x) {
    const uint8_t* p = reinterpret_cast<const uint8_t*>(&x);
    v.insert(v.end(), p, p + sizeof(T));
}

uint32_t fbits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}

Leaf make_const(bool v) {
    Leaf l;
    l.is_const = true;
    l.cval = v;
    return l;
}

Leaf int_range(int col, int type, i128 lo, i128 hi, bool neg) {
    const i128 tmin = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::min() : (i128)INT32_MIN;
    const i128 tmax = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::max() : (i128)INT32_MAX;
    lo = std::max(lo, tmin);
    hi = std::min(hi, tmax);
    if (lo > hi) return make_const(neg);
    if (lo == tmin && hi == tmax) return make_const(!neg);
    Leaf l;
    l.col = col;
    l.ins.neg = neg ? 1 : 0;
    if (type == SEL_I64) {
        l.ins.opc = OP_RANGE64;
        put<uint64_t>(l.pool, (uint64_t)(int64_t)lo);
        put<uint64_t>(l.pool, (uint64_t)(hi - lo));
    } else {
        l.ins.opc = OP_RANGE32;
        l.ins.a = (uint32_t)(int32_t)lo;
        l.ins.b = (uint32_t)(hi - lo);
    }
    return l;
}

// Perfect multiply-shift hash of a value set: slot(x) = (uint32)(key(x) * mult)
// >> shift over a table of 2^(32 - shift) entries, key(x) = x for 32-bit
// columns and lo32(x) ^ hi32(x) for int64.  Multipliers are drawn from a fixed
// SplitMix64 stream (the same set always compiles to the same table) until one
// puts every value in its own slot; the table doubles (up to 8 KB) when a size
// finds none.  Empty slots hold the first value, which cannot match there
// because that value hashes to its own slot.
constexpr size_t kMaxHashKeys = 128;

bool perfect_hash(Leaf& l, const std::vector<i128>& v, bool wide) {
    const size_t max_entries = wide ? 1024 : 2048;
    uint64_t state = 0x5E1EC7ull;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    std::vector<uint32_t> keys;
    for (i128 x : v) {
        const uint64_t u = (uint64_t)(int64_t)x;
        keys.push_back(wide ? (uint32_t)u ^ (uint32_t)(u >> 32) : (uint32_t)u);
    }
    int bits = 1;
    while (((size_t)1 << bits) < 2 * v.size()) ++bits;
    std::vector<int> slot_of;
    for (; ((size_t)1 << bits) <= max_entries; ++bits) {
        const size_t m = (size_t)1 << bits;
        const uint32_t shift = 32u - (uint32_t)bits;
        std::vector<uint8_t> used(m);
        for (int attempt = 0; attempt < 4000; ++attempt) {
            const uint32_t mult = (uint32_t)next() | 1u;
            std::fill(used.begin(), used.end(), 0);
            bool ok = true;
            for (uint32_t k : keys) {
                const uint32_t h = (k * mult) >> shift;
                if (used[h]) {
                    ok = false;
                    break;
                }
                used[h] = 1;
            }
            if (!ok) continue;
            l.ins.opc = wide ? OP_HASH64 : OP_HASH32;
            l.ins.a = mult;
            l.ins.b = shift;
            l.pool.clear();
            std::vector<uint64_t> table(m, (uint64_t)(int64_t)v.front());
            for (size_t i = 0; i < v.size(); ++i) table[(keys[i] * mult) >> shift] = (uint64_t)(int64_t)v[i];
            for (uint64_t t : table) {
                if (wide)
                    put<uint64_t>(l.pool, t);
                else
                    put<uint32_t>(l.pool, (uint32_t)t);
            }
            return true;
        }
    }
    return false;
}

Leaf int_set(int col, int type, std::vector<i128> v, bool neg) {
    const i128 tmin = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::min() : (i128)INT32_MIN;
    const i128 tmax = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::max() : (i128)INT32_MAX;
    v.erase(std::remove_if(v.begin(), v.end(), [&](i128 x) { return x < tmin || x > tmax; }), v.end());
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    if (v.empty()) return make_const(neg);
    const i128 span = v.back() - v.front();
    if (span == (i128)(v.size() - 1)) return int_range(col, type, v.front(), v.back(), neg);
    Leaf l;
    l.col = col;
    l.ins.neg = neg ? 1 : 0;
    if (type != SEL_I64 && span < 32) {   // the whole set in one 32-bit word of the instruction
        uint32_t word = 0;
        for (i128 x : v) word |= 1u << (uint32_t)(x - v.front());
        l.ins.opc = OP_MASK32;
        l.ins.a = (uint32_t)(int32_t)v.front();
        l.ins.b = word;
        return l;
    }
    if (v.size() >= 3 && v.size() <= kMaxHashKeys && perfect_hash(l, v, type == SEL_I64)) return l;
    if (type != SEL_I64 && v.size() > 8 && span < (i128)(1 << 20)) {
        const uint32_t nbits = (uint32_t)(span + 1);
        std::vector<uint32_t> words((nbits + 31) / 32, 0u);
        for (i128 x : v) {
            const uint32_t d = (uint32_t)(x - v.front());
            words[d >> 5] |= 1u << (d & 31);
        }
        l.ins.opc = OP_BITMAP;
        l.ins.a = (uint32_t)(int32_t)v.front();
        l.ins.b = nbits;
        for (uint32_t w : words) put<uint32_t>(l.pool, w);
        return l;
    }
    l.ins.a = (uint32_t)v.size();
    if (type == SEL_I64) {
        l.ins.opc = OP_IN64;
        for (i128 x : v) put<uint64_t>(l.pool, (uint64_t)(int64_t)x);
    } else {
        l.ins.opc = OP_IN32;
        for (i128 x : v) put<uint32_t>(l.pool, (uint32_t)(int32_t)x);
    }
    return l;
}

Leaf float_range(int col, float lo, float hi, bool neg) {
    if (std::isnan(lo) || std::isnan(hi) || lo > hi) return make_const(neg);
    Leaf l;
    l.col = col;
    l.ins.opc = OP_RANGEF;
    l.ins.neg = neg ? 1 : 0;
    l.ins.a = fbits(lo);
    l.ins.b = fbits(hi);
    return l;
}

const float kInf = std::numeric_limits<float>::infinity();

Leaf lower_leaf(const sel_node& nd, const sel_table& schema, bool neg, Clause& cl) {
    const int col = nd.col;
    const sel_column& c = schema.cols[col];
    const int type = c.type;
    cl = Clause{};
    cl.col = col;
    cl.kind = nd.kind;
    cl.op = nd.op;
    cl.negated = neg ? 1 : 0;
    cl.nnf_neg = neg ? 1 : 0;
    cl.raw_i0 = nd.i_lo;
    cl.raw_i1 = nd.i_hi;
    cl.raw_f0 = nd.f_lo;
    cl.raw_f1 = nd.f_hi;
    if (type == SEL_F32) {
        if (nd.kind == SEL_N_LIKE) fail(SEL_ERR_TYPE, "LIKE on a float32 column");
        if (nd.kind == SEL_N_CMP) {
            const float k = nd.f_lo;
            float lo = k, hi = k;
            bool n = neg;
            switch (nd.op) {
            case SEL_EQ: break;
            case SEL_NE: n = !n; break;
            case SEL_LT:
                if (std::isnan(k) || k == -kInf) return make_const(neg);
                lo = -kInf; hi = std::nextafter(k, -kInf); break;
            case SEL_LE: lo = -kInf; hi = k; break;
            case SEL_GT:
                if (std::isnan(k) || k == kInf) return make_const(neg);
                lo = std::nextafter(k, kInf); hi = kInf; break;
            case SEL_GE: lo = k; hi = kInf; break;
            default: fail(SEL_ERR_INVALID_ARG, "bad comparison operator");
            }
            cl.f_lo = lo; cl.f_hi = hi; cl.negated = n ? 1 : 0;
            return float_range(col, lo, hi, n);
        }
        if (nd.kind == SEL_N_BETWEEN) {
            cl.f_lo = nd.f_lo; cl.f_hi = nd.f_hi;
            return float_range(col, nd.f_lo, nd.f_hi, neg);
        }
        // IN
        if (nd.n_values < 0 || nd.n_values > SEL_MAX_IN_VALUES) fail(SEL_ERR_UNSUPPORTED, "IN list too long");
        if (nd.n_values > 0 && !nd.values) fail(SEL_ERR_INVALID_ARG, "IN list without values");
        std::vector<float> v;
        const float* src = static_cast<const float*>(nd.values);
        for (int i = 0; i < nd.n_values; ++i)
            if (!std::isnan(src[i])) v.push_back(src[i]);
        std::sort(v.begin(), v.end());
        std::vector<float> u;
        for (float x : v)
            if (u.empty() || !(u.back() == x)) u.push_back(x);   // -0.0 == +0.0: one entry
        cl.fvals = u;
        if (u.empty()) return make_const(neg);
        if (u.size() == 1) return float_range(col, u[0], u[0], neg);
        Leaf l;
        l.col = col;
        l.ins.opc = OP_INF;
        l.ins.neg = neg ? 1 : 0;
        l.ins.a = (uint32_t)u.size();
        for (float x : u) put<float>(l.pool, x);
        return l;
    }
    // integer-like: int32, int64, date, dictionary code
    if (nd.kind == SEL_N_CMP) {
        const i128 k = nd.i_lo;
        const i128 big = (i128)1 << 100;
        i128 lo = k, hi = k;
        bool n = neg;
        switch (nd.op) {
        case SEL_EQ: break;
        case SEL_NE: n = !n; break;
        case SEL_LT: lo = -big; hi = k - 1; break;
        case SEL_LE: lo = -big; hi = k; break;
        case SEL_GT: lo = k + 1; hi = big; break;
        case SEL_GE: lo = k; hi = big; break;
        default: fail(SEL_ERR_INVALID_ARG, "bad comparison operator");
        }
        const i128 tmin = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::min() : (i128)INT32_MIN;
        const i128 tmax = (type == SEL_I64) ? (i128)std::numeric_limits<int64_t>::max() : (i128)INT32_MAX;
        cl.i_lo = (int64_t)std::max(std::min(lo, tmax), tmin);
        cl.i_hi = (int64_t)std::min(std::max(hi, tmin), tmax);
        cl.negated = n ? 1 : 0;
        return int_range(col, type, lo, hi, n);
    }
    if (nd.kind == SEL_N_BETWEEN) {
        cl.i_lo = nd.i_lo;
        cl.i_hi = nd.i_hi;
        return int_range(col, type, nd.i_lo, nd.i_hi, neg);
    }
    if (nd.kind == SEL_N_IN) {
        if (nd.n_values < 0 || nd.n_values > SEL_MAX_IN_VALUES) fail(SEL_ERR_UNSUPPORTED, "IN list too long");
        if (nd.n_values > 0 && !nd.values) fail(SEL_ERR_INVALID_ARG, "IN list without values");
        std::vector<i128> v;
        const int64_t* src = static_cast<const int64_t*>(nd.values);
        for (int i = 0; i < nd.n_values; ++i) {
            v.push_back(src[i]);
            cl.ivals.push_back(src[i]);
        }
        return int_set(col, type, v, neg);
    }
    // LIKE 'prefix%'
    if (type != SEL_DICT) fail(SEL_ERR_TYPE, "LIKE on a column that is not dictionary-encoded");
    if (!c.dict || c.dict_size <= 0) fail(SEL_ERR_TYPE, "LIKE needs the column's dictionary");
    if (!nd.prefix) fail(SEL_ERR_INVALID_ARG, "LIKE without a prefix");
    const size_t m = std::strlen(nd.prefix);
    std::vector<i128> codes;
    for (int32_t i = 0; i < c.dict_size; ++i) {
        if (!c.dict[i]) fail(SEL_ERR_INVALID_ARG, "null dictionary entry");
        if (std::strncmp(c.dict[i], nd.prefix, m) == 0) codes.push_back(i);
    }
    cl.like_count = (int32_t)codes.size();
    for (i128 x : codes) cl.like_codes.push_back((int32_t)x);
    cl.code_lo = codes.empty() ? 0 : (int32_t)codes.front();
    cl.code_hi = codes.empty() ? -1 : (int32_t)codes.back();
    if (codes.empty()) return make_const(neg);
    if (codes.back() - codes.front() == (i128)(codes.size() - 1))
        return int_range(col, SEL_I32, codes.front(), codes.back(), neg);
    // scattered codes (unsorted dictionary): bitmap over [first, last]
    Leaf l;
    l.col = col;
    l.ins.opc = OP_BITMAP;
    l.ins.neg = neg ? 1 : 0;
    const uint32_t nbits = (uint32_t)(codes.back() - codes.front() + 1);
    std::vector<uint32_t> words((nbits + 31) / 32, 0u);
    for (i128 x : codes) {
        const uint32_t d = (uint32_t)(x - codes.front());
        words[d >> 5] |= 1u << (d & 31);
    }
    l.ins.a = (uint32_t)(int32_t)codes.front();
    l.ins.b = nbits;
    for (uint32_t w : words) put<uint32_t>(l.pool, w);
    return l;
}

struct Compiler {
    const sel_table& schema;
    const sel_node* nodes;
    int n_nodes;
    std::vector<TNode> t;     // parsed tree
    std::vector<TNode> nnf;   // negation normal form
    std::vector<std::vector<Clause>> dnf;
    bool dnf_ok = true;

    int parse() {
        std::vector<int> st;
        for (int i = 0; i < n_nodes; ++i) {
            const sel_node& nd = nodes[i];
            TNode x;
            switch (nd.kind) {
            case SEL_N_CMP: case SEL_N_BETWEEN: case SEL_N_IN: case SEL_N_LIKE:
                if (nd.col < 0 || nd.col >= schema.n_cols)
                    fail(SEL_ERR_INVALID_ARG, "node " + std::to_string(i) + ": column out of range");
                if (nd.kind == SEL_N_CMP && (nd.op < SEL_EQ || nd.op > SEL_GE))
                    fail(SEL_ERR_INVALID_ARG, "node " + std::to_string(i) + ": bad comparison operator");
                x.kind = K_LEAF;
                x.src = &nd;
                break;
            case SEL_N_TRUE: x.kind = K_TRUE; break;
            case SEL_N_FALSE: x.kind = K_FALSE; break;
            case SEL_N_NOT:
                if (st.empty()) fail(SEL_ERR_INVALID_ARG, "NOT without operand");
                x.kind = K_NOT;
                x.kids.push_back(st.back());
                st.pop_back();
                break;
            case SEL_N_AND: case SEL_N_OR: {
                const int k = nd.n_children;
                if (k < 1 || k > (int)st.size())
                    fail(SEL_ERR_INVALID_ARG, "node " + std::to_string(i) + ": bad operand count");
                x.kind = nd.kind == SEL_N_AND ? K_AND : K_OR;
                x.kids.assign(st.end() - k, st.end());
                st.resize(st.size() - k);
                break;
            }
            default:
                fail(SEL_ERR_INVALID_ARG, "node " + std::to_string(i) + ": unknown kind");
            }
            t.push_back(x);
            st.push_back((int)t.size() - 1);
        }
        if (st.size() != 1) fail(SEL_ERR_INVALID_ARG, "postfix array does not reduce to one tree");
        return st.back();
    }

    int to_nnf(int x, bool neg) {
        const TNode& n = t[x];
        TNode y;
        switch (n.kind) {
        case K_NOT: return to_nnf(n.kids[0], !neg);
        case K_TRUE: y.kind = neg ? K_FALSE : K_TRUE; break;
        case K_FALSE: y.kind = neg ? K_TRUE : K_FALSE; break;
        case K_LEAF: y = n; y.neg = neg; break;
        default: {
            const bool is_and = (n.kind == K_AND) != neg;
            y.kind = is_and ? K_AND : K_OR;
            for (int k : n.kids) y.kids.push_back(to_nnf(k, neg));
        }
        }
        nnf.push_back(y);
        return (int)nnf.size() - 1;
    }

    ENode lower(int x) {
        const TNode& n = nnf[x];
        ENode e;
        if (n.kind == K_TRUE || n.kind == K_FALSE) {
            e.kind = n.kind;
            return e;
        }
        if (n.kind == K_LEAF) {
            Clause cl;
            e.leaf = lower_leaf(*n.src, schema, n.neg, cl);
            if (e.leaf.is_const) e.kind = e.leaf.cval ? K_TRUE : K_FALSE;
            else e.kind = K_LEAF;
            return e;
        }
        // AND / OR: fold constants and flatten
        const bool is_and = n.kind == K_AND;
        e.kind = n.kind;
        for (int k : n.kids) {
            ENode c = lower(k);
            if (c.kind == (is_and ? K_FALSE : K_TRUE)) {
                ENode r;
                r.kind = c.kind;
                return r;
            }
            if (c.kind == (is_and ? K_TRUE : K_FALSE)) continue;
            if (c.kind == n.kind) {
                for (auto& g : c.kids) e.kids.push_back(std::move(g));
            } else {
                e.kids.push_back(std::move(c));
            }
        }
        if (e.kids.empty()) {
            ENode r;
            r.kind = is_and ? K_TRUE : K_FALSE;
            return r;
        }
        if (e.kids.size() == 1) return std::move(e.kids[0]);
        return e;
    }

    static void order(ENode& e) {
        if (e.kind != K_AND && e.kind != K_OR) {
            e.need = 1;
            return;
        }
        for (auto& k : e.kids) order(k);
        std::stable_sort(e.kids.begin(), e.kids.end(), [](const ENode& a, const ENode& b) { return a.need > b.need; });
        e.need = e.kids[0].need;
        for (size_t i = 1; i < e.kids.size(); ++i) e.need = std::max(e.need, e.kids[i].need + 1);
    }

    void emit(const ENode& e, Program& p, const std::vector<int>& col_slot) {
        if (e.kind == K_TRUE || e.kind == K_FALSE) {
            Instr in{};
            in.opc = OP_CONST;
            in.neg = e.kind == K_FALSE ? 1 : 0;
            p.instrs.push_back(in);
            return;
        }
        if (e.kind == K_LEAF) {
            const std::string key = leaf_key(e.leaf);
            auto done = memo_slot.find(key);
            if (done != memo_slot.end()) {   // evaluated before: reuse its saved mask
                Instr ld{};
                ld.opc = OP_LOAD;
                ld.a = (uint32_t)done->second;
                p.instrs.push_back(ld);
                return;
            }
            Instr in = e.leaf.ins;
            in.slot = (uint8_t)col_slot[e.leaf.col];
            if (!e.leaf.pool.empty()) {
                const size_t al = (in.opc == OP_RANGE64 || in.opc == OP_IN64 || in.opc == OP_HASH64) ? 8 : 4;
                while (p.pool.size() % al) p.pool.push_back(0);
                in.off = (uint32_t)p.pool.size();
                p.pool.insert(p.pool.end(), e.leaf.pool.begin(), e.leaf.pool.end());
            }
            p.instrs.push_back(in);
            p.leaves++;
            if (occurrences[key] > 1 && (int)memo_slot.size() < kMemoSlots) {
                const int k = (int)memo_slot.size();
                memo_slot[key] = k;
                Instr sv{};
                sv.opc = OP_SAVE;
                sv.a = (uint32_t)k;
                p.instrs.push_back(sv);
            }
            return;
        }
        emit(e.kids[0], p, col_slot);
        for (size_t i = 1; i < e.kids.size(); ++i) {
            emit(e.kids[i], p, col_slot);
            Instr in{};
            in.opc = e.kind == K_AND ? OP_AND : OP_OR;
            p.instrs.push_back(in);
        }
    }

    // Identity of a lowered leaf: column, operation, negation and constants.
    static std::string leaf_key(const Leaf& l) {
        std::string k(reinterpret_cast<const char*>(&l.ins), sizeof(Instr));
        k += std::to_string(l.col) + ":";
        k.append(reinterpret_cast<const char*>(l.pool.data()), l.pool.size());
        return k;
    }

    std::map<std::string, int> occurrences;   // leaf key -> number of occurrences in the tree
    std::map<std::string, int> memo_slot;     // leaf key -> memo slot holding its mask

    void count_leaves(const ENode& e) {
        if (e.kind == K_LEAF) occurrences[leaf_key(e.leaf)]++;
        for (auto& k : e.kids) count_leaves(k);
    }

    static void columns(const ENode& e, std::vector<int>& cols) {
        if (e.kind == K_LEAF) cols.push_back(e.leaf.col);
        for (auto& k : e.kids) columns(k, cols);
    }

    // Clause structure (OR of ANDs of leaves) of the NNF tree, for features.
    void capture_dnf(int root) {
        auto leaf_clause = [&](int x, std::vector<Clause>& out) -> bool {
            const TNode& n = nnf[x];
            if (n.kind != K_LEAF) return false;
            Clause cl;
            lower_leaf(*n.src, schema, n.neg, cl);
            out.push_back(cl);
            return true;
        };
        auto and_group = [&](int x, std::vector<Clause>& out) -> bool {
            const TNode& n = nnf[x];
            if (n.kind == K_LEAF) return leaf_clause(x, out);
            if (n.kind != K_AND) return false;
            for (int k : n.kids)
                if (!leaf_clause(k, out)) return false;
            return true;
        };
        const TNode& r = nnf[root];
        dnf.clear();
        if (r.kind == K_OR) {
            for (int k : r.kids) {
                std::vector<Clause> g;
                if (!and_group(k, g)) { dnf_ok = false; return; }
                dnf.push_back(g);
            }
        } else {
            std::vector<Clause> g;
            if (!and_group(root, g)) { dnf_ok = false; return; }
            dnf.push_back(g);
        }
    }
};

// Peephole over the postfix program: an instruction that pushes a mask (a
// leaf, CONST or LOAD) directly followed by AND / OR combines its mask into
// the top of the stack instead (Instr.comb), which saves the binary
// operator's dispatch and a push and pop of the mask stack.  The pushed mask
// is always the operator's second operand, so the result is the same.
static void combine_into_top(Program& p) {
    std::vector<Instr> out;
    out.reserve(p.instrs.size());
    for (size_t i = 0; i < p.instrs.size(); ++i) {
        Instr in = p.instrs[i];
        const bool pushes = in.opc != OP_AND && in.opc != OP_OR && in.opc != OP_SAVE;
        if (pushes && !out.empty() && i + 1 < p.instrs.size() &&
            (p.instrs[i + 1].opc == OP_AND || p.instrs[i + 1].opc == OP_OR)) {
            in.comb = p.instrs[i + 1].opc;
            ++i;
        }
        out.push_back(in);
    }
    p.instrs.swap(out);
}

std::string describe(const Program& p) {
    std::ostringstream o;
    static const char* names[] = {"?", "AND", "OR", "CONST", "RANGE32", "RANGE64", "RANGEF",
                                  "IN32", "IN64", "INF", "BITMAP", "SAVE", "LOAD", "MASK32", "HASH32", "HASH64"};
    o << "slots:";
    for (size_t s = 0; s < p.slot_col.size(); ++s) o << " " << p.slot_col[s] << "/" << p.slot_width[s];
    o << "\nneed: " << p.need << "\nleaves: " << p.leaves << "\n";
    for (const Instr& in : p.instrs) {
        o << names[in.opc <= OP_HASH64 ? in.opc : 0];
        if (in.opc == OP_SAVE || in.opc == OP_LOAD) o << " m=" << in.a;
        if (in.opc != OP_AND && in.opc != OP_OR && in.opc != OP_SAVE && in.opc != OP_LOAD) {
            if (in.opc != OP_CONST) o << " slot=" << (int)in.slot;
            o << " neg=" << (int)in.neg;
        }
        switch (in.opc) {
        case OP_RANGE32: o << " lo=" << (int32_t)in.a << " span=" << in.b; break;
        case OP_RANGE64: {
            uint64_t lo, sp;
            std::memcpy(&lo, &p.pool[in.off], 8);
            std::memcpy(&sp, &p.pool[in.off + 8], 8);
            o << " lo=" << (int64_t)lo << " span=" << sp;
            break;
        }
        case OP_RANGEF: {
            float lo, hi;
            std::memcpy(&lo, &in.a, 4);
            std::memcpy(&hi, &in.b, 4);
            o << " lo=" << lo << " hi=" << hi << " bits=0x" << std::hex << in.a << ",0x" << in.b << std::dec;
            break;
        }
        case OP_IN32: case OP_IN64: case OP_INF: {
            o << " n=" << in.a << " vals=";
            for (uint32_t k = 0; k < in.a; ++k) {
                if (k) o << ",";
                if (in.opc == OP_IN32) {
                    int32_t v;
                    std::memcpy(&v, &p.pool[in.off + 4 * k], 4);
                    o << v;
                } else if (in.opc == OP_IN64) {
                    int64_t v;
                    std::memcpy(&v, &p.pool[in.off + 8 * k], 8);
                    o << v;
                } else {
                    uint32_t v;
                    std::memcpy(&v, &p.pool[in.off + 4 * k], 4);
                    o << "0x" << std::hex << v << std::dec;
                }
            }
            break;
        }
        case OP_MASK32: o << " lo=" << (int32_t)in.a << " word=0x" << std::hex << in.b << std::dec; break;
        case OP_HASH32: case OP_HASH64: {
            const uint32_t entries = 1u << (32u - in.b);
            o << " mult=0x" << std::hex << in.a << std::dec << " shift=" << in.b << " table=";
            for (uint32_t k = 0; k < entries; ++k) {
                if (k) o << ",";
                if (in.opc == OP_HASH32) {
                    int32_t v;
                    std::memcpy(&v, &p.pool[in.off + 4 * k], 4);
                    o << v;
                } else {
                    int64_t v;
                    std::memcpy(&v, &p.pool[in.off + 8 * k], 8);
                    o << v;
                }
            }
            break;
        }
        case OP_BITMAP: {
            o << " lo=" << (int32_t)in.a << " nbits=" << in.b << " words=";
            for (uint32_t k = 0; k < (in.b + 31) / 32; ++k) {
                uint32_t w;
                std::memcpy(&w, &p.pool[in.off + 4 * k], 4);
                o << (k ? "," : "") << "0x" << std::hex << w << std::dec;
            }
            break;
        }
        default: break;
        }
        if (in.comb == OP_AND) o << " +AND";
        else if (in.comb == OP_OR) o << " +OR";
        o << "\n";
    }
    return o.str();
}

std::atomic<uint64_t> g_next_id{1};

}  // namespace
}  // namespace sel

using namespace sel;

extern "C" sel_status sel_compile_predicate(const sel_table* schema, const sel_node* postfix, int32_t n_nodes,
                                            sel_pred** out) {
    if (!out) {
        set_error("sel_compile_predicate: out is NULL");
        return SEL_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!schema || !postfix || n_nodes <= 0 || (schema->n_cols > 0 && !schema->cols) || schema->n_cols < 0) {
        set_error("sel_compile_predicate: null schema/postfix or empty tree");
        return SEL_ERR_INVALID_ARG;
    }
    if (n_nodes > SEL_MAX_NODES) {
        set_error("sel_compile_predicate: %d nodes > SEL_MAX_NODES", n_nodes);
        return SEL_ERR_UNSUPPORTED;
    }
    for (int32_t c = 0; c < schema->n_cols; ++c) {
        const int ty = schema->cols[c].type;
        if (ty < SEL_I32 || ty > SEL_DICT) {
            set_error("sel_compile_predicate: column %d has unknown type %d", c, ty);
            return SEL_ERR_TYPE;
        }
    }
    try {
        Compiler cp{*schema, postfix, n_nodes, {}, {}, {}, true};
        const int root = cp.parse();
        const int nroot = cp.to_nnf(root, false);
        ENode e = cp.lower(nroot);
        Compiler::order(e);
        Program prog;
        std::vector<int> cols;
        Compiler::columns(e, cols);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        if ((int)cols.size() > kMaxSlots) fail(SEL_ERR_UNSUPPORTED, "predicate reads more than 16 columns");
        std::vector<int> col_slot(schema->n_cols, -1);
        for (size_t s = 0; s < cols.size(); ++s) {
            col_slot[cols[s]] = (int)s;
            prog.slot_col.push_back(cols[s]);
            prog.slot_width.push_back(schema->cols[cols[s]].type == SEL_I64 ? 8u : 4u);
        }
        prog.need = e.need;
        cp.count_leaves(e);
        cp.emit(e, prog, col_slot);
        combine_into_top(prog);
        if (prog.leaves > SEL_MAX_LEAVES) fail(SEL_ERR_UNSUPPORTED, "more than SEL_MAX_LEAVES leaves");
        if (prog.need > kMaxDepth) fail(SEL_ERR_UNSUPPORTED, "tree needs a deeper evaluation stack than 8");
        if (prog.pool.size() > (1u << 20)) fail(SEL_ERR_UNSUPPORTED, "constant pool above 1 MiB");
        cp.capture_dnf(nroot);
        sel_pred* p = new sel_pred();
        p->id = g_next_id++;
        for (int32_t c = 0; c < schema->n_cols; ++c) p->col_types.push_back(schema->cols[c].type);
        p->prog = std::move(prog);
        p->dnf = std::move(cp.dnf);
        p->dnf_ok = cp.dnf_ok;
        p->text = describe(p->prog);
        // FNV-1a over the program (instructions, pool, slot columns and schema types)
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](const void* d, size_t n) {
            const uint8_t* b = static_cast<const uint8_t*>(d);
            for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
        };
        mix(p->prog.instrs.data(), p->prog.instrs.size() * sizeof(Instr));
        mix(p->prog.pool.data(), p->prog.pool.size());
        mix(p->prog.slot_col.data(), p->prog.slot_col.size() * sizeof(int32_t));
        mix(p->col_types.data(), p->col_types.size() * sizeof(int32_t));
        p->content = h;
        *out = p;
        return SEL_OK;
    } catch (const Fail& f) {
        set_error("sel_compile_predicate: %s", f.msg.c_str());
        return f.st;
    } catch (const std::bad_alloc&) {
        set_error("sel_compile_predicate: host allocation failed");
        return SEL_ERR_OOM;
    }
}

extern "C" void sel_pred_free(sel_pred* p) {
    if (!p) return;
    if (p->d_blob) cudaFree(p->d_blob);
    delete p;
}

extern "C" sel_status sel_pred_describe(const sel_pred* p, char* buf, int64_t cap) {
    if (!p || !buf || cap <= 0) {
        set_error("sel_pred_describe: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    const size_t n = std::min<size_t>(p->text.size(), (size_t)cap - 1);
    std::memcpy(buf, p->text.data(), n);
    buf[n] = 0;
    return SEL_OK;
}

// ---------------------------------------------------------------------------
// blobs
// ---------------------------------------------------------------------------

void build_blob(const std::vector<const Program*>& progs, const std::vector<std::vector<int32_t>>& slot_maps,
                std::vector<uint8_t>& blob, uint32_t& instr_off, uint32_t& pool_off,
                const std::vector<uint32_t>& outs) {
    std::vector<ProgDesc> pd;
    std::vector<Instr> ins;
    std::vector<uint8_t> pool;
    for (size_t i = 0; i < progs.size(); ++i) {
        const Program& p = *progs[i];
        while (pool.size() % 8) pool.push_back(0);
        const uint32_t pbase = (uint32_t)pool.size();
        pool.insert(pool.end(), p.pool.begin(), p.pool.end());
        pd.push_back(ProgDesc{(uint32_t)ins.size(), (uint32_t)p.instrs.size(), (uint32_t)(outs.empty() ? i : outs[i]), 0u});
        for (Instr in : p.instrs) {
            if (in.opc != OP_AND && in.opc != OP_OR && in.opc != OP_CONST && in.opc != OP_SAVE && in.opc != OP_LOAD) {
                in.slot = (uint8_t)slot_maps[i][in.slot];
                in.off += pbase;
            }
            ins.push_back(in);
        }
    }
    blob.clear();
    auto pad16 = [&]() { while (blob.size() % 16) blob.push_back(0); };
    blob.insert(blob.end(), reinterpret_cast<uint8_t*>(pd.data()),
                reinterpret_cast<uint8_t*>(pd.data()) + pd.size() * sizeof(ProgDesc));
    pad16();
    instr_off = (uint32_t)blob.size();
    blob.insert(blob.end(), reinterpret_cast<uint8_t*>(ins.data()),
                reinterpret_cast<uint8_t*>(ins.data()) + ins.size() * sizeof(Instr));
    pad16();
    pool_off = (uint32_t)blob.size();
    blob.insert(blob.end(), pool.begin(), pool.end());
    pad16();
}

// A non-blocking stream per device for the predicate uploads: a copy on the
// legacy default stream would wait for every kernel queued before it (the
// caller's earlier scans), and the host with it.
static cudaStream_t upload_stream(cudaError_t* err) {
    static std::mutex mu;
    static std::map<int, cudaStream_t> streams;
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    auto it = streams.find(dev);
    if (it != streams.end()) return it->second;
    cudaStream_t st = nullptr;
    *err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (*err != cudaSuccess) return nullptr;
    streams[dev] = st;
    return st;
}

sel_status pred_upload(const sel_pred* cp) {
    sel_pred* p = const_cast<sel_pred*>(cp);
    std::lock_guard<std::mutex> g(p->mu);
    if (p->d_blob) return SEL_OK;
    std::vector<uint8_t> blob;
    std::vector<int32_t> ident(kMaxSlots);
    for (int i = 0; i < kMaxSlots; ++i) ident[i] = i;
    build_blob({&p->prog}, {ident}, blob, p->instr_off, p->pool_off);
    void* d = nullptr;
    cudaError_t e = dev_alloc(&d, blob.size());
    if (e != cudaSuccess) {
        set_error("predicate upload: cudaMalloc: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? SEL_ERR_OOM : SEL_ERR_CUDA;
    }
    // the copy is complete when this returns: later launches on any stream read it
    cudaStream_t st = upload_stream(&e);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(d);
        set_error("predicate upload: %s", cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    p->blob_bytes = (uint32_t)blob.size();
    p->d_blob = d;
    return SEL_OK;
}
