// program.h -- compiled predicate format shared by the host compiler and the
// scan kernels.
//
// A predicate (the WHERE clause of the §3.1 COUNT query) is compiled to a
// postfix program over "slots" (the distinct columns it reads).  Every leaf
// evaluates to an 8-bit row mask for the 8 rows a thread owns in a 256-row
// warp chunk; AND / OR combine the two top masks of a small stack.  NOT has
// been pushed into the leaves (negation normal form), so each leaf carries a
// negate flag instead.
#pragma once
#include <stdint.h>

namespace sel {

enum Opcode : uint8_t {
    OP_AND = 1,
    OP_OR = 2,
    OP_CONST = 3,     // every row true (negated: every row false)
    OP_RANGE32 = 4,   // (uint32)(x - a) <= b              x: int32 / date / dict code
    OP_RANGE64 = 5,   // (uint64)(x - lo) <= span          lo, span: 16 pool bytes at off
    OP_RANGEF = 6,    // fa <= x && x <= fb                binary32 ordered compares
    OP_IN32 = 7,      // x == pool32[k], k < a             pool at off
    OP_IN64 = 8,      // x == pool64[k], k < a
    OP_INF = 9,       // x == poolf[k], k < a
    OP_BITMAP = 10,   // d = (uint32)(x - a); d < b && bit d of the pool words at off
    OP_SAVE = 11,     // memo slot a := top of stack (a leaf that occurs again later)
    OP_LOAD = 12,     // push memo slot a (a repeated leaf, evaluated once)
    OP_MASK32 = 13,   // d = (uint32)(x - a); d < 32 && bit d of b    (a set spanning <= 32 values)
    OP_HASH32 = 14,   // t = pool32 at off; t[(uint32)(x * a) >> b] == x   (perfect multiply-shift hash)
    OP_HASH64 = 15,   // t = pool64 at off; k = lo32(x) ^ hi32(x); t[(uint32)(k * a) >> b] == x
};

constexpr int kMemoSlots = 4;      // 8-bit masks kept in one 32-bit register

// 16 bytes; read uniformly by a whole warp.
struct Instr {
    uint8_t opc;
    uint8_t slot;     // column slot (leaves)
    uint8_t neg;      // 1: complement the leaf's row mask
    uint8_t comb;     // leaves, CONST, LOAD: 0 = push the mask; OP_AND / OP_OR = combine it into the top
    uint32_t off;     // byte offset into the pool (RANGE64, IN*, BITMAP)
    uint32_t a;       // see opcode
    uint32_t b;
};
static_assert(sizeof(Instr) == 16, "Instr layout");

// One program inside a program blob.
struct ProgDesc {
    uint32_t instr_begin;   // index of the first Instr in the blob's instruction array
    uint32_t n_instr;
    uint32_t out;           // index of the program's count in the launch's output array
    uint32_t pad;
};

constexpr int kMaxSlots = 16;
constexpr int kMaxDepth = 8;       // stack entries besides the top-of-stack register
constexpr int kChunkRows = 256;    // rows per warp chunk (8 per lane)

}  // namespace sel
