// bucket_plan.cpp -- host builder of the column-bucket form of a batch of
// count probes (the layout is described in bucket.h), and a host evaluator
// of that form used by the CPU tests.
//
// Steps for each table of the batch:
//   1. every program (already in negation normal form, postfix) is taken to
//      disjunctive normal form over literals (a leaf and a negation flag);
//      identical leaves of different programs become one leaf;
//   2. every leaf's value set is turned into its change points in the raw bit
//      order of its column (the values x where membership of x and of x - 1
//      differ); the union of a column's change points are its bucket
//      boundaries;
//   3. each leaf's membership is evaluated at the first value of every
//      bucket, with the same semantics as the interpreter's leaf (program.h);
//      as a check of step 2 it is also evaluated at the last value and the two
//      must agree;
//   4. programs are cut into blocks of 64; for every block and column the gm
//      table holds the group bits of every bucket (deduplicated into local
//      buckets through a uint16 remap when the table has several blocks).
// A batch that does not fit (a program with more than 4 groups after
// simplification, more than 4096 boundaries on a column, more than 8 tables)
// is reported as SEL_ERR_UNSUPPORTED and runs on the interpreter instead.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "bucket.h"
#include "internal.h"

namespace sel {

namespace {

constexpr size_t kMaxBoundaries = 4096;
constexpr size_t kMaxDnfGroups = 64;   // intermediate DNF size during the conversion

typedef uint32_t Lit;                  // leaf index << 1 | negated
typedef std::vector<Lit> Group;        // sorted, unique
typedef std::vector<Group> Dnf;        // OR of groups; empty = FALSE; an empty group = TRUE

// A distinct leaf of a table: the instruction (slot remapped to the table's
// slot), its pool bytes, and its membership per global bucket.
struct LeafRec {
    Instr in;
    std::vector<uint8_t> pool;   // the leaf's own pool bytes (offset 0)
    uint32_t slot;
    std::vector<uint8_t> member; // per global bucket of its slot
};

uint32_t f2u(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u;
}
float u2f(uint32_t u) {
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// Bytes of the pool a leaf reads (from its instruction's offset).
size_t leaf_pool_bytes(const Instr& in) {
    switch (in.opc) {
    case OP_RANGE64: return 16;
    case OP_IN32: case OP_INF: return (size_t)in.a * 4;
    case OP_IN64: return (size_t)in.a * 8;
    case OP_BITMAP: return (size_t)((in.b + 31) / 32) * 4;
    case OP_HASH32: return ((size_t)1 << (32 - in.b)) * 4;
    case OP_HASH64: return ((size_t)1 << (32 - in.b)) * 8;
    default: return 0;
    }
}

bool is_leaf(uint8_t opc) {
    return opc == OP_RANGE32 || opc == OP_RANGE64 || opc == OP_RANGEF || opc == OP_IN32 || opc == OP_IN64 ||
           opc == OP_INF || opc == OP_BITMAP || opc == OP_MASK32 || opc == OP_HASH32 || opc == OP_HASH64;
}

template <typename T>
T rd(const std::vector<uint8_t>& p, size_t off) {
    T v;
    std::memcpy(&v, p.data() + off, sizeof(T));
    return v;
}

// Membership of raw value x (the column's bits, zero-extended) in the leaf's
// value set, before its negation flag: the interpreter's leaf semantics.
bool member(const LeafRec& L, uint64_t x) {
    const Instr& in = L.in;
    const uint32_t x32 = (uint32_t)x;
    switch (in.opc) {
    case OP_RANGE32: return (uint32_t)(x32 - in.a) <= in.b;
    case OP_RANGE64: return x - rd<uint64_t>(L.pool, 0) <= rd<uint64_t>(L.pool, 8);
    case OP_RANGEF: {
        const float v = u2f(x32);
        return u2f(in.a) <= v && v <= u2f(in.b);
    }
    case OP_IN32:
        for (uint32_t k = 0; k < in.a; ++k)
            if (rd<uint32_t>(L.pool, 4 * k) == x32) return true;
        return false;
    case OP_IN64:
        for (uint32_t k = 0; k < in.a; ++k)
            if (rd<uint64_t>(L.pool, 8 * k) == x) return true;
        return false;
    case OP_INF:
        for (uint32_t k = 0; k < in.a; ++k)
            if (u2f(rd<uint32_t>(L.pool, 4 * k)) == u2f(x32)) return true;
        return false;
    case OP_BITMAP: {
        const uint32_t d = x32 - in.a;
        return d < in.b && ((rd<uint32_t>(L.pool, 4 * (d >> 5)) >> (d & 31u)) & 1u);
    }
    case OP_MASK32: {
        const uint32_t d = x32 - in.a;
        return d < 32 && ((in.b >> d) & 1u);
    }
    case OP_HASH32: return rd<uint32_t>(L.pool, 4 * (size_t)((x32 * in.a) >> in.b)) == x32;
    case OP_HASH64: {
        const uint32_t k = (uint32_t)x ^ (uint32_t)(x >> 32);
        return rd<uint64_t>(L.pool, 8 * (size_t)((k * in.a) >> in.b)) == x;
    }
    default: return false;
    }
}

// Values where membership changes (x with member(x) != member(x - 1)), as a
// superset; 0 (the start of the domain) is never listed.
void change_points(const LeafRec& L, uint32_t width, std::vector<uint64_t>& out) {
    const Instr& in = L.in;
    const uint64_t top = width == 8 ? ~0ull : 0xFFFFFFFFull;   // largest raw value
    auto add = [&](uint64_t p) {
        if (p != 0 && p <= top) out.push_back(p);
    };
    auto add_point = [&](uint64_t p) {   // a single member p: it starts at p, ends before p + 1
        add(p);
        if (p < top) add(p + 1);
    };
    auto add_interval = [&](uint64_t lo, uint64_t hi) {   // members lo..hi, lo <= hi
        add(lo);
        if (hi < top) add(hi + 1);
    };
    switch (in.opc) {
    case OP_RANGE32:
        if (in.b != 0xFFFFFFFFu) {
            add(in.a);
            add((uint32_t)(in.a + in.b + 1u));
        }
        break;
    case OP_RANGE64: {
        const uint64_t lo = rd<uint64_t>(L.pool, 0), sp = rd<uint64_t>(L.pool, 8);
        if (sp != ~0ull) {
            add(lo);
            add(lo + sp + 1);
        }
        break;
    }
    case OP_RANGEF: {
        const float fa = u2f(in.a), fb = u2f(in.b);
        if (fb >= 0.0f)   // members among +0 .. +inf (bit patterns ascend with the value)
            add_interval(fa <= 0.0f ? 0u : f2u(fa), fb == 0.0f ? 0u : f2u(fb));
        if (fa <= 0.0f)   // members among -0 .. -inf (bit patterns ascend as the value falls)
            add_interval(fb >= 0.0f ? 0x80000000u : f2u(fb), fa == 0.0f ? 0x80000000u : f2u(fa));
        break;
    }
    case OP_IN32:
        for (uint32_t k = 0; k < in.a; ++k) add_point(rd<uint32_t>(L.pool, 4 * k));
        break;
    case OP_IN64:
        for (uint32_t k = 0; k < in.a; ++k) add_point(rd<uint64_t>(L.pool, 8 * k));
        break;
    case OP_INF:
        for (uint32_t k = 0; k < in.a; ++k) {
            const float v = u2f(rd<uint32_t>(L.pool, 4 * k));
            if (v == 0.0f) {
                add_point(0u);
                add_point(0x80000000u);
            } else {
                add_point(f2u(v));
            }
        }
        break;
    case OP_BITMAP:
        for (uint32_t d = 0; d < in.b; ++d)
            if ((rd<uint32_t>(L.pool, 4 * (d >> 5)) >> (d & 31u)) & 1u) add_point((uint32_t)(in.a + d));
        break;
    case OP_MASK32:
        for (uint32_t d = 0; d < 32; ++d)
            if ((in.b >> d) & 1u) add_point((uint32_t)(in.a + d));
        break;
    case OP_HASH32: {
        const size_t m = (size_t)1 << (32 - in.b);
        for (size_t s = 0; s < m; ++s) {
            const uint32_t v = rd<uint32_t>(L.pool, 4 * s);
            if (((v * in.a) >> in.b) == s) add_point(v);
        }
        break;
    }
    case OP_HASH64: {
        const size_t m = (size_t)1 << (32 - in.b);
        for (size_t s = 0; s < m; ++s) {
            const uint64_t v = rd<uint64_t>(L.pool, 8 * s);
            const uint32_t k = (uint32_t)v ^ (uint32_t)(v >> 32);
            if (((k * in.a) >> in.b) == s) add_point(v);
        }
        break;
    }
    default: break;
    }
}

// --- disjunctive normal form ------------------------------------------------

bool contradictory(const Group& g) {
    for (size_t i = 1; i < g.size(); ++i)
        if ((g[i] >> 1) == (g[i - 1] >> 1)) return true;   // x and NOT x
    return false;
}

void simplify(Dnf& d) {
    d.erase(std::remove_if(d.begin(), d.end(), contradictory), d.end());
    std::sort(d.begin(), d.end(), [](const Group& a, const Group& b) {
        return a.size() != b.size() ? a.size() < b.size() : a < b;
    });
    d.erase(std::unique(d.begin(), d.end()), d.end());
    Dnf keep;   // absorption: a group that contains a smaller kept group adds nothing
    for (const Group& g : d) {
        bool absorbed = false;
        for (const Group& k : keep)
            if (std::includes(g.begin(), g.end(), k.begin(), k.end())) {
                absorbed = true;
                break;
            }
        if (!absorbed) keep.push_back(g);
    }
    d.swap(keep);
}

bool dnf_and(const Dnf& a, const Dnf& b, Dnf& out) {
    out.clear();
    if (a.size() * b.size() > kMaxDnfGroups) return false;
    for (const Group& x : a)
        for (const Group& y : b) {
            Group g;
            std::set_union(x.begin(), x.end(), y.begin(), y.end(), std::back_inserter(g));
            out.push_back(g);
        }
    simplify(out);
    return true;
}

bool dnf_or(const Dnf& a, const Dnf& b, Dnf& out) {
    if (a.size() + b.size() > kMaxDnfGroups) return false;
    out = a;
    out.insert(out.end(), b.begin(), b.end());
    simplify(out);
    return true;
}

struct Builder {
    std::vector<LeafRec> leaves;
    std::map<std::string, uint32_t> index;

    uint32_t leaf_id(const Instr& in, const std::vector<uint8_t>& pool, uint32_t slot) {
        LeafRec L;
        L.in = in;
        L.in.slot = (uint8_t)slot;
        L.in.neg = 0;
        L.in.comb = 0;
        L.in.off = 0;
        L.slot = slot;
        const size_t nb = leaf_pool_bytes(in);
        if (nb > 0) L.pool.assign(pool.begin() + in.off, pool.begin() + in.off + nb);
        std::string key(reinterpret_cast<const char*>(&L.in), sizeof(Instr));
        key.append(reinterpret_cast<const char*>(L.pool.data()), L.pool.size());
        auto it = index.find(key);
        if (it != index.end()) return it->second;
        const uint32_t id = (uint32_t)leaves.size();
        leaves.push_back(std::move(L));
        index.emplace(key, id);
        return id;
    }

    // The program's DNF; false when it does not fit.
    bool to_dnf(const Program& p, const std::vector<int32_t>& slot_map, Dnf& out) {
        std::vector<Dnf> stk;
        Dnf top;          // the interpreter's top-of-stack register starts as a dummy
        Dnf memo[kMemoSlots];
        auto combine = [&](uint8_t comb, Dnf v) -> bool {
            if (comb == OP_AND) {
                Dnf r;
                if (!dnf_and(top, v, r)) return false;
                top.swap(r);
            } else if (comb == OP_OR) {
                Dnf r;
                if (!dnf_or(top, v, r)) return false;
                top.swap(r);
            } else {
                stk.push_back(top);
                top.swap(v);
            }
            return true;
        };
        for (const Instr& in : p.instrs) {
            if (in.opc == OP_AND || in.opc == OP_OR) {
                if (stk.empty()) return false;
                Dnf r;
                if (!(in.opc == OP_AND ? dnf_and(top, stk.back(), r) : dnf_or(top, stk.back(), r))) return false;
                stk.pop_back();
                top.swap(r);
            } else if (in.opc == OP_SAVE) {
                if (in.a >= (uint32_t)kMemoSlots) return false;
                memo[in.a] = top;
            } else if (in.opc == OP_LOAD) {
                if (in.a >= (uint32_t)kMemoSlots) return false;
                if (!combine(in.comb, memo[in.a])) return false;
            } else if (in.opc == OP_CONST) {
                Dnf v;
                if (!in.neg) v.push_back(Group{});   // TRUE: one empty group
                if (!combine(in.comb, v)) return false;
            } else if (is_leaf(in.opc)) {
                const uint32_t id = leaf_id(in, p.pool, (uint32_t)slot_map[in.slot]);
                Dnf v{Group{(id << 1) | (in.neg ? 1u : 0u)}};
                if (!combine(in.comb, v)) return false;
            } else {
                return false;
            }
        }
        if (p.instrs.empty()) return false;
        out.swap(top);
        return true;
    }
};

template <typename T>
void put_at(std::vector<uint8_t>& b, size_t off, const T& v) {
    std::memcpy(b.data() + off, &v, sizeof(T));
}

size_t append(std::vector<uint8_t>& b, const void* p, size_t n) {
    while (b.size() % 16) b.push_back(0);
    const size_t off = b.size();
    b.insert(b.end(), static_cast<const uint8_t*>(p), static_cast<const uint8_t*>(p) + n);
    return off;
}

}  // namespace

sel_status build_bucket_plan(const std::vector<BkTableIn>& tabs, BucketPlan* out, std::string* why) {
    if (tabs.size() > (size_t)kMaxTables) {
        *why = "more tables than one launch holds";
        return SEL_ERR_UNSUPPORTED;
    }
    std::vector<uint8_t> blob(sizeof(BkHeader), 0);
    BkHeader hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    hdr.n_tables = (uint32_t)tabs.size();
    uint32_t n_out = 0;
    for (size_t ti = 0; ti < tabs.size(); ++ti) {
        const BkTableIn& T = tabs[ti];
        BkTable& bt = hdr.t[ti];
        bt.n_slots = (uint32_t)T.slot_width.size();
        Builder b;
        std::vector<Dnf> dnfs(T.progs.size());
        for (size_t i = 0; i < T.progs.size(); ++i) {
            if (!b.to_dnf(*T.progs[i], T.slot_maps[i], dnfs[i]) || dnfs[i].size() > (size_t)kBkGroups) {
                *why = "a program has more than 4 AND-groups in disjunctive normal form";
                return SEL_ERR_UNSUPPORTED;
            }
        }
        for (uint32_t o : T.outs) n_out = std::max(n_out, o + 1);
        // boundaries per slot
        std::vector<std::vector<uint64_t>> bnd(bt.n_slots);
        for (const LeafRec& L : b.leaves) change_points(L, T.slot_width[L.slot], bnd[L.slot]);
        for (uint32_t s = 0; s < bt.n_slots; ++s) {
            std::sort(bnd[s].begin(), bnd[s].end());
            bnd[s].erase(std::unique(bnd[s].begin(), bnd[s].end()), bnd[s].end());
            if (bnd[s].size() > kMaxBoundaries) {
                *why = "more than 4096 bucket boundaries on one column";
                return SEL_ERR_UNSUPPORTED;
            }
        }
        // membership of every leaf in every bucket of its slot (and the check)
        for (LeafRec& L : b.leaves) {
            const std::vector<uint64_t>& B = bnd[L.slot];
            const uint64_t top = T.slot_width[L.slot] == 8 ? ~0ull : 0xFFFFFFFFull;
            L.member.resize(B.size() + 1);
            for (size_t j = 0; j <= B.size(); ++j) {
                const uint64_t first = j == 0 ? 0 : B[j - 1];
                const uint64_t last = j == B.size() ? top : B[j] - 1;
                const bool m = member(L, first);
                if (member(L, last) != m) {
                    *why = "internal: a leaf changes inside a bucket";
                    return SEL_ERR_UNSUPPORTED;
                }
                L.member[j] = m ? 1 : 0;
            }
        }
        // search data: a linear count for up to 4 boundaries, a direct table
        // when every cell is one value, cells when at most kBkMaxOcc
        // boundaries share a cell, cells and a binary search inside the cell
        // when that takes 2 or more steps fewer than a binary search of all
        // boundaries, else a linear count (up to kBkLinear) or a binary search
        for (uint32_t s = 0; s < bt.n_slots; ++s) {
            const uint32_t w = T.slot_width[s];
            const std::vector<uint64_t>& B = bnd[s];
            BkSlot& sl = bt.slot[s];
            sl.k = (uint32_t)B.size();
            size_t n_entries = sl.k;
            std::vector<uint16_t> cells;
            if (sl.k <= 4) {   // 2 instructions per boundary and row (measured faster than cells up to 4)
                sl.mode = BK_LINEAR;
            } else {
                const uint64_t span = B.back() - B.front();
                uint32_t shift = 0;
                while ((span >> shift) >= (uint64_t)kBkMaxCells) ++shift;
                const uint32_t n_cells = (uint32_t)(span >> shift) + 1;
                std::vector<uint32_t> occ(n_cells, 0);
                for (uint64_t b : B) ++occ[(b - B.front()) >> shift];
                const uint32_t mx = *std::max_element(occ.begin(), occ.end());
                if (shift == 0) {
                    // every cell is one value: the table holds that value's bucket, no compares
                    sl.mode = BK_CELLS;
                    sl.lo = B.front();
                    sl.shift = 0;
                    sl.n_cells = n_cells;
                    sl.occ = 0;
                    cells.resize(n_cells);
                    uint32_t upto = 0;
                    for (uint32_t c = 0; c < n_cells; ++c) {
                        upto += occ[c];
                        cells[c] = (uint16_t)upto;
                    }
                } else {
                    uint32_t steps = 0, cell_steps = 0;   // full binary search; search inside the fullest cell
                    while (((size_t)1 << steps) < (size_t)sl.k + 1) ++steps;
                    while (((size_t)1 << cell_steps) < (size_t)mx + 1) ++cell_steps;
                    if (mx <= (uint32_t)kBkMaxOcc || (sl.k > (uint32_t)kBkLinear && cell_steps + 1 < steps)) {
                        // cells, then up to 3 compares, or a search of cell_steps steps
                        // (a cell lookup costs about one step)
                        const bool bin = mx > (uint32_t)kBkMaxOcc;
                        sl.mode = bin ? BK_CELLS_BIN : BK_CELLS;
                        sl.lo = B.front();
                        sl.shift = shift;
                        sl.n_cells = n_cells;
                        sl.occ = bin ? 0u : mx;
                        sl.half = bin ? 1u << (cell_steps - 1) : 0u;
                        cells.resize(n_cells);
                        uint32_t before = 0;
                        for (uint32_t c = 0; c < n_cells; ++c) {
                            cells[c] = (uint16_t)before;
                            before += occ[c];
                        }
                        n_entries = (size_t)sl.k + (bin ? ((size_t)1 << cell_steps) - 1 : mx);
                    } else if (sl.k <= (uint32_t)kBkLinear) {
                        sl.mode = BK_LINEAR;
                    } else {
                        sl.mode = BK_BINARY;
                        sl.half = 1u << (steps - 1);
                        n_entries = ((size_t)1 << steps) - 1;
                    }
                }
            }
            std::vector<uint8_t> raw(std::max<size_t>(n_entries, 1) * w, 0xFF);
            for (size_t j = 0; j < B.size(); ++j) {
                if (w == 8)
                    std::memcpy(raw.data() + 8 * j, &B[j], 8);
                else {
                    const uint32_t v = (uint32_t)B[j];
                    std::memcpy(raw.data() + 4 * j, &v, 4);
                }
            }
            sl.bnd_off = (uint32_t)append(blob, raw.data(), raw.size());
            if (!cells.empty()) sl.cells_off = (uint32_t)append(blob, cells.data(), cells.size() * 2);
            bt.max_buckets = std::max(bt.max_buckets, sl.k + 1);
        }
        // blocks: for each, its columns, and per column the gm rows of its
        // distinct buckets (local rows) and the global -> local remap
        const size_t np = T.progs.size();
        const uint32_t n_blocks = (uint32_t)((np + kBkBlockProgs - 1) / kBkBlockProgs);
        struct SlotRows {
            std::vector<uint32_t> rows;    // local rows, stride words each
            std::vector<uint16_t> remap;   // global bucket -> local row
            bool identity;                 // local rows are the global buckets
        };
        std::vector<BkBlock> blocks(n_blocks);
        std::vector<std::vector<uint32_t>> block_outs(n_blocks);
        std::vector<std::vector<SlotRows>> block_rows(n_blocks);
        for (uint32_t bi = 0; bi < n_blocks; ++bi) {
            BkBlock& bk = blocks[bi];
            std::memset(&bk, 0, sizeof(bk));
            const size_t p0 = (size_t)bi * kBkBlockProgs, p1 = std::min(np, p0 + kBkBlockProgs);
            bk.n_progs = (uint32_t)(p1 - p0);
            bk.n_words = (bk.n_progs + kBkProgsPerWord - 1) / kBkProgsPerWord;
            bk.nw = bk.n_words <= 1 ? 1 : bk.n_words <= 2 ? 2 : bk.n_words <= 4 ? 4 : 8;
            bk.stride = bk.nw == 8 ? 12 : bk.nw;
            std::vector<uint32_t>& outs = block_outs[bi];
            outs.resize(bk.n_progs);
            for (size_t k = 0; k < bk.n_progs; ++k) {
                outs[k] = T.outs[p0 + k];
                const size_t g = dnfs[p0 + k].size();
                bk.init[k / kBkProgsPerWord] |= ((1u << g) - 1u) << (4 * (k % kBkProgsPerWord));
            }
            std::vector<uint8_t> uses(bt.n_slots, 0);
            for (size_t k = p0; k < p1; ++k)
                for (const Group& g : dnfs[k])
                    for (Lit l : g) uses[b.leaves[l >> 1].slot] = 1;
            for (uint32_t s = 0; s < bt.n_slots; ++s) {
                if (!uses[s]) continue;
                bk.used[bk.n_used++] = s;
                const uint32_t nb = (uint32_t)bnd[s].size() + 1;
                // gm rows per global bucket
                std::vector<uint32_t> rows((size_t)nb * bk.stride, 0xFFFFFFFFu);
                for (size_t k = p0; k < p1; ++k) {
                    const uint32_t word = (uint32_t)((k - p0) / kBkProgsPerWord);
                    const uint32_t field = (uint32_t)((k - p0) % kBkProgsPerWord);
                    for (size_t gi = 0; gi < dnfs[k].size(); ++gi) {
                        const uint32_t bit = 1u << (4 * field + (uint32_t)gi);
                        for (Lit l : dnfs[k][gi]) {
                            const LeafRec& L = b.leaves[l >> 1];
                            if (L.slot != s) continue;
                            for (uint32_t j = 0; j < nb; ++j)
                                if (!(L.member[j] ^ (l & 1u))) rows[(size_t)j * bk.stride + word] &= ~bit;
                        }
                    }
                }
                SlotRows sr;
                sr.identity = true;
                if (n_blocks > 1) {
                    std::map<std::vector<uint32_t>, uint16_t> local;
                    std::vector<uint32_t> gm;
                    sr.remap.resize(nb);
                    for (uint32_t j = 0; j < nb; ++j) {
                        std::vector<uint32_t> r(rows.begin() + (size_t)j * bk.stride,
                                                rows.begin() + (size_t)(j + 1) * bk.stride);
                        auto it = local.find(r);
                        if (it == local.end()) {
                            it = local.emplace(r, (uint16_t)(gm.size() / bk.stride)).first;
                            gm.insert(gm.end(), r.begin(), r.end());
                        }
                        sr.remap[j] = it->second;
                    }
                    if (gm.size() != rows.size()) {
                        sr.identity = false;
                        rows.swap(gm);
                    }
                }
                if (sr.identity) {
                    sr.remap.resize(nb);
                    for (uint32_t j = 0; j < nb; ++j) sr.remap[j] = (uint16_t)j;
                }
                sr.rows.swap(rows);
                block_rows[bi].push_back(std::move(sr));
            }
        }
        // the quad form: at least kBkQuadMinBlocks blocks and 1 to
        // kBkQuadMaxSlots columns
        const bool quad = n_blocks >= (uint32_t)kBkQuadMinBlocks && bt.n_slots >= 1 &&
                          bt.n_slots <= (uint32_t)kBkQuadMaxSlots;
        const uint32_t n_quads = (n_blocks + kBkQuadBlocks - 1) / kBkQuadBlocks;
        if (!quad) {
            for (uint32_t bi = 0; bi < n_blocks; ++bi) {
                BkBlock& bk = blocks[bi];
                bk.out_off = (uint32_t)append(blob, block_outs[bi].data(), block_outs[bi].size() * 4);
                for (uint32_t u = 0; u < bk.n_used; ++u) {
                    const SlotRows& sr = block_rows[bi][u];
                    bk.remap_off[u] =
                        sr.identity ? kBkIdentity : (uint32_t)append(blob, sr.remap.data(), sr.remap.size() * 2);
                    bk.gm_off[u] = (uint32_t)append(blob, sr.rows.data(), sr.rows.size() * 4);
                }
            }
            bt.n_blocks = n_blocks;
            bt.block_off = (uint32_t)append(blob, blocks.data(), blocks.size() * sizeof(BkBlock));
            if (n_blocks > 1) hdr.gb_slots = std::max(hdr.gb_slots, bt.n_slots);
        } else {
            std::vector<BkQuad> quads(n_quads);
            for (uint32_t qi = 0; qi < n_quads; ++qi) {
                BkQuad& Q = quads[qi];
                std::memset(&Q, 0, sizeof(Q));
                const uint32_t b0 = qi * kBkQuadBlocks, nq = std::min<uint32_t>(kBkQuadBlocks, n_blocks - b0);
                std::vector<uint32_t> outs(kBkQuadBlocks * kBkBlockProgs, kBkNoOut);
                for (uint32_t p = 0; p < nq; ++p)
                    for (size_t k = 0; k < block_outs[b0 + p].size(); ++k) outs[p * kBkBlockProgs + k] = block_outs[b0 + p][k];
                Q.out_off = (uint32_t)append(blob, outs.data(), outs.size() * 4);
                // every column of the table, in slot order (the kernel's row
                // records hold the indices in that order; a column no block of
                // the quad reads has only the all-ones and the zero row)
                for (uint32_t s = 0; s < bt.n_slots; ++s) {
                    const uint32_t u = Q.n_used++;
                    Q.used[u] = s;
                    // block p's local rows of column s (none: it has no leaf there)
                    const SlotRows* sr[kBkQuadBlocks] = {nullptr, nullptr, nullptr, nullptr};
                    uint32_t n_local = 0;
                    for (uint32_t p = 0; p < nq; ++p) {
                        const BkBlock& bk = blocks[b0 + p];
                        for (uint32_t v = 0; v < bk.n_used; ++v)
                            if (bk.used[v] == s) sr[p] = &block_rows[b0 + p][v];
                        if (sr[p]) n_local = std::max<uint32_t>(n_local, (uint32_t)(sr[p]->rows.size() / bk.stride));
                    }
                    const uint32_t R = n_local + 2, one = R - 2, zero = R - 1;
                    const uint32_t nb = (uint32_t)bnd[s].size() + 1;
                    std::vector<uint32_t> gm((size_t)R * 32, 0u);
                    for (uint32_t p = 0; p < nq; ++p) {
                        const uint32_t stride = blocks[b0 + p].stride;
                        for (uint32_t r = 0; r < R; ++r)
                            for (uint32_t w = 0; w < (uint32_t)kBkMaxWords; ++w) {
                                uint32_t v = 0;
                                if (r == one) v = 0xFFFFFFFFu;
                                else if (sr[p] && r < sr[p]->rows.size() / stride && w < stride)
                                    v = sr[p]->rows[(size_t)r * stride + w];
                                if (u == 0) v &= blocks[b0 + p].init[w];   // the init mask, once
                                gm[(size_t)r * 32 + 8 * p + w] = v;
                            }
                    }
                    std::vector<uint16_t> remap((size_t)(nb + 1) * kBkQuadBlocks, (uint16_t)zero);
                    for (uint32_t j = 0; j < nb; ++j)
                        for (uint32_t p = 0; p < nq; ++p)
                            remap[(size_t)j * kBkQuadBlocks + p] = sr[p] ? sr[p]->remap[j] : (uint16_t)one;
                    if (R > 65536u) {
                        *why = "internal: more than 65536 local rows";
                        return SEL_ERR_UNSUPPORTED;
                    }
                    Q.remap_off[u] = (uint32_t)append(blob, remap.data(), remap.size() * 2);
                    Q.gm_off[u] = (uint32_t)append(blob, gm.data(), gm.size() * 4);
                }
            }
            bt.n_blocks = n_blocks;   // the blocks themselves are not kept: n_quads > 0 selects the quad form
            bt.n_quads = n_quads;
            bt.quad_off = (uint32_t)append(blob, quads.data(), quads.size() * sizeof(BkQuad));
            hdr.gb_quad = 1;
        }
    }
    hdr.n_out = n_out;
    while (blob.size() % 16) blob.push_back(0);
    put_at(blob, 0, hdr);
    out->blob.swap(blob);
    out->n_out = n_out;
    return SEL_OK;
}

// --- host evaluation (tests) -----------------------------------------------

namespace {

uint32_t host_bucket(const std::vector<uint8_t>& blob, const BkSlot& sl, uint32_t width, uint64_t x) {
    auto bnd = [&](uint32_t j) -> uint64_t {
        if (width == 8) return rd<uint64_t>(blob, sl.bnd_off + 8 * (size_t)j);
        return rd<uint32_t>(blob, sl.bnd_off + 4 * (size_t)j);
    };
    uint32_t idx = 0;
    if (sl.mode == BK_LINEAR) {
        for (uint32_t j = 0; j < sl.k; ++j) idx += x >= bnd(j) ? 1u : 0u;
        return idx;
    }
    if (sl.mode == BK_CELLS || sl.mode == BK_CELLS_BIN) {
        if (x < sl.lo) return 0;
        const uint64_t c = std::min<uint64_t>((x - sl.lo) >> sl.shift, sl.n_cells - 1);
        const uint32_t base = rd<uint16_t>(blob, sl.cells_off + 2 * (size_t)c);
        idx = base;
        if (sl.mode == BK_CELLS) {
            for (uint32_t t = 0; t < sl.occ; ++t) idx += x >= bnd(base + t) ? 1u : 0u;
        } else {
            for (uint32_t h = sl.half; h; h >>= 1)
                if (x >= bnd(idx + h - 1)) idx += h;
        }
        return std::min(idx, sl.k);
    }
    for (uint32_t h = sl.half; h; h >>= 1)
        if (x >= bnd(idx + h - 1)) idx += h;
    return std::min(idx, sl.k);
}

}  // namespace

void bucket_eval_host(const BucketPlan& plan, const std::vector<std::vector<const uint8_t*>>& cols,
                      const std::vector<std::vector<uint32_t>>& widths, const std::vector<int64_t>& n_rows,
                      uint64_t* counts) {
    const std::vector<uint8_t>& blob = plan.blob;
    BkHeader hdr;
    std::memcpy(&hdr, blob.data(), sizeof(hdr));
    for (uint32_t ti = 0; ti < hdr.n_tables; ++ti) {
        const BkTable& bt = hdr.t[ti];
        const bool quad = bt.n_quads > 0;
        std::vector<BkBlock> blocks(quad ? 0 : bt.n_blocks);
        std::memcpy(blocks.data(), blob.data() + bt.block_off, blocks.size() * sizeof(BkBlock));
        std::vector<BkQuad> quads(bt.n_quads);
        std::memcpy(quads.data(), blob.data() + bt.quad_off, quads.size() * sizeof(BkQuad));
        std::vector<uint32_t> gb(bt.n_slots);
        for (int64_t r = 0; r < n_rows[ti]; ++r) {
            for (uint32_t s = 0; s < bt.n_slots; ++s) {
                const uint32_t w = widths[ti][s];
                uint64_t x = 0;
                std::memcpy(&x, cols[ti][s] + (size_t)r * w, w);
                gb[s] = host_bucket(blob, bt.slot[s], w, x);
            }
            // quad form: block p's words of the row are the AND over the
            // quad's columns of its 8 words in the row its remap gives
            for (const BkQuad& Q : quads)
                for (uint32_t p = 0; p < (uint32_t)kBkQuadBlocks; ++p) {
                    uint32_t R[kBkMaxWords];
                    for (uint32_t w = 0; w < kBkMaxWords; ++w) R[w] = 0xFFFFFFFFu;
                    for (uint32_t u = 0; u < Q.n_used; ++u) {
                        const uint32_t s = Q.used[u];
                        const uint32_t lb = rd<uint16_t>(blob, Q.remap_off[u] + 2 * ((size_t)gb[s] * kBkQuadBlocks + p));
                        for (uint32_t w = 0; w < kBkMaxWords; ++w)
                            R[w] &= rd<uint32_t>(blob, Q.gm_off[u] + 4 * ((size_t)lb * 32 + 8 * p + w));
                    }
                    for (uint32_t k = 0; k < (uint32_t)kBkBlockProgs; ++k) {
                        const uint32_t o = rd<uint32_t>(blob, Q.out_off + 4 * ((size_t)p * kBkBlockProgs + k));
                        if (o != kBkNoOut && ((R[k / kBkProgsPerWord] >> (4 * (k % kBkProgsPerWord))) & 0xFu))
                            ++counts[o];
                    }
                }
            for (const BkBlock& bk : blocks) {
                uint32_t R[kBkMaxWords];
                for (uint32_t w = 0; w < kBkMaxWords; ++w) R[w] = bk.init[w];
                for (uint32_t u = 0; u < bk.n_used; ++u) {
                    const uint32_t s = bk.used[u];
                    const uint32_t lb =
                        bk.remap_off[u] == kBkIdentity ? gb[s] : rd<uint16_t>(blob, bk.remap_off[u] + 2 * (size_t)gb[s]);
                    for (uint32_t w = 0; w < bk.n_words; ++w)
                        R[w] &= rd<uint32_t>(blob, bk.gm_off[u] + 4 * ((size_t)lb * bk.stride + w));
                }
                for (uint32_t k = 0; k < bk.n_progs; ++k)
                    if ((R[k / kBkProgsPerWord] >> (4 * (k % kBkProgsPerWord))) & 0xFu)
                        ++counts[rd<uint32_t>(blob, bk.out_off + 4 * (size_t)k)];
            }
        }
    }
}

}  // namespace sel

using namespace sel;

extern "C" sel_status sel_debug_bucket_count_host(const sel_pred* const* preds, int32_t n, const sel_table* table,
                                                  uint64_t* counts, int32_t* n_blocks, int32_t* n_quads) {
    if (!preds || n <= 0 || !table || !counts || table->n_rows < 0 || (table->n_cols > 0 && !table->cols)) {
        set_error("sel_debug_bucket_count_host: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    std::vector<int32_t> cols;
    for (int32_t i = 0; i < n; ++i) {
        if (!preds[i]) {
            set_error("sel_debug_bucket_count_host: predicate %d is NULL", i);
            return SEL_ERR_INVALID_ARG;
        }
        for (int32_t c : preds[i]->prog.slot_col) {
            if (c < 0 || c >= table->n_cols || table->cols[c].type != preds[i]->col_types[c] ||
                (table->n_rows > 0 && !table->cols[c].data)) {
                set_error("sel_debug_bucket_count_host: column %d missing or of another type", c);
                return SEL_ERR_INVALID_ARG;
            }
            cols.push_back(c);
        }
    }
    std::sort(cols.begin(), cols.end());
    cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
    if (cols.size() > (size_t)kMaxSlots) {
        set_error("sel_debug_bucket_count_host: more than 16 columns");
        return SEL_ERR_UNSUPPORTED;
    }
    BkTableIn in;
    std::vector<const uint8_t*> ptrs;
    for (int32_t c : cols) {
        in.slot_width.push_back(table->cols[c].type == SEL_I64 ? 8u : 4u);
        ptrs.push_back(static_cast<const uint8_t*>(table->cols[c].data));
    }
    for (int32_t i = 0; i < n; ++i) {
        std::vector<int32_t> m;
        for (int32_t c : preds[i]->prog.slot_col)
            m.push_back((int32_t)(std::lower_bound(cols.begin(), cols.end(), c) - cols.begin()));
        in.progs.push_back(&preds[i]->prog);
        in.slot_maps.push_back(m);
        in.outs.push_back((uint32_t)i);
    }
    BucketPlan plan;
    std::string why;
    const sel_status s = build_bucket_plan({in}, &plan, &why);
    if (s != SEL_OK) {
        set_error("sel_debug_bucket_count_host: %s", why.c_str());
        return s;
    }
    BkHeader hdr;
    std::memcpy(&hdr, plan.blob.data(), sizeof(hdr));
    if (n_blocks) *n_blocks = (int32_t)hdr.t[0].n_blocks;
    if (n_quads) *n_quads = (int32_t)hdr.t[0].n_quads;
    std::memset(counts, 0, sizeof(uint64_t) * (size_t)n);
    bucket_eval_host(plan, {ptrs}, {in.slot_width}, {table->n_rows}, counts);
    return SEL_OK;
}
