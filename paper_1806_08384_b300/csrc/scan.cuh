// scan.cuh -- device building blocks of the column scans (sm_103a).
//
//  * bulk (TMA) copies of column tiles global -> shared, completed on an
//    mbarrier (cp.async.bulk ... mbarrier::complete_tx::bytes);
//  * bounded mbarrier waits (a wait gives up after kWaitNs nanoseconds of
//    %globaltimer and the caller reports SEL_ERR_TIMEOUT);
//  * the bit-sliced predicate interpreter: a warp evaluates one compiled
//    program over a 256-row chunk of a staged tile, each lane producing an
//    8-bit mask for its 8 rows.
//
// Row ownership inside a 256-row chunk starting at tile row c0: lane l owns
// rows c0 + 4l + i (mask bit i) and c0 + 128 + 4l + i (mask bit 4 + i),
// i = 0..3.  A 4-byte column is then read with two conflict-free 16-byte
// shared loads per lane; an 8-byte column with four.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "program.h"

namespace sel {



__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// The same for a waiter that is not on the critical path (it would otherwise
// take issue slots from the warps that are): sleeps sleep_ns between tries.
__device__ __forceinline__ bool mbar_wait_bounded_idle(uint64_t* bar, uint32_t parity, uint32_t sleep_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        __nanosleep(sleep_ns);
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

// L2 policy for streamed column data: read once, evict first.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// One bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

// ---------------------------------------------------------------------------
// leaf evaluation over the 8 rows of a lane
// ---------------------------------------------------------------------------

__device__ __forceinline__ void load8x32(uint32_t col_base, uint32_t c0, uint32_t lane, uint32_t (&v)[8]) {
    const uint32_t p = col_base + c0 * 4u + lane * 16u;
    const uint4 a = lds128(p);
    const uint4 b = lds128(p + 512u);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void load8x64(uint32_t col_base, uint32_t c0, uint32_t lane, uint64_t (&v)[8]) {
    const uint32_t p = col_base + c0 * 8u + lane * 32u;
    const uint4 a0 = lds128(p), a1 = lds128(p + 16u);
    const uint4 b0 = lds128(p + 1024u), b1 = lds128(p + 1040u);
    v[0] = (uint64_t)a0.y << 32 | a0.x; v[1] = (uint64_t)a0.w << 32 | a0.z;
    v[2] = (uint64_t)a1.y << 32 | a1.x; v[3] = (uint64_t)a1.w << 32 | a1.z;
    v[4] = (uint64_t)b0.y << 32 | b0.x; v[5] = (uint64_t)b0.w << 32 | b0.z;
    v[6] = (uint64_t)b1.y << 32 | b1.x; v[7] = (uint64_t)b1.w << 32 | b1.z;
}

template <typename Pred>
__device__ __forceinline__ uint32_t mask8(Pred pred) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) m |= (pred(i) ? 1u : 0u) << i;
    return m;
}

// The same from 0/1 values.
template <typename Bit>
__device__ __forceinline__ uint32_t mask8_bits(Bit bit) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) m |= bit(i) << i;
    return m;
}

// Set membership of the lane's 8 rows in blocks of B list values: each block
// is one branch-free OR of B equality tests per row (a short list repeats its
// last value, which changes nothing).
template <int G, int B, typename T, typename Eq>
__device__ __forceinline__ void in_list(const T (&v)[G][8], const T* vals, uint32_t n, Eq eq, uint32_t (&m)[G]) {
    bool hit[G][8];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int i = 0; i < 8; ++i) hit[g][i] = false;
    for (uint32_t k0 = 0; k0 < n; k0 += B) {
        T w[B];
#pragma unroll
        for (int j = 0; j < B; ++j) w[j] = vals[min(k0 + j, n - 1)];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                bool h = hit[g][i];
#pragma unroll
                for (int j = 0; j < B; ++j) h = h | eq(v[g][i], w[j]);
                hit[g][i] = h;
            }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) m[g] = mask8([&](int i) { return hit[g][i]; });
}

// Evaluates one leaf on G chunks (chunk g starts at tile row c0[g]); the pool
// pointer may address shared or global memory.  RANGE32, RANGEF and MASK32
// are evaluated inline by eval_program_g and never come here.
template <int G>
__device__ __forceinline__ void eval_leaf_g(const Instr& in, uint32_t col_base, const uint32_t (&c0)[G], uint32_t lane,
                                            const uint8_t* pool, uint32_t (&m)[G]) {
    switch (in.opc) {
    case OP_RANGE64: {
        uint64_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x64(col_base, c0[g], lane, v[g]);
        const uint64_t lo = *reinterpret_cast<const uint64_t*>(pool + in.off);
        const uint64_t sp = *reinterpret_cast<const uint64_t*>(pool + in.off + 8);
#pragma unroll
        for (int g = 0; g < G; ++g) m[g] = mask8([&](int i) { return v[g][i] - lo <= sp; });
        break;
    }
    case OP_IN32: {
        uint32_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x32(col_base, c0[g], lane, v[g]);
        in_list<G, 8>(v, reinterpret_cast<const uint32_t*>(pool + in.off), in.a,
                      [](uint32_t x, uint32_t w) { return x == w; }, m);
        break;
    }
    case OP_INF: {
        uint32_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x32(col_base, c0[g], lane, v[g]);
        in_list<G, 8>(v, reinterpret_cast<const uint32_t*>(pool + in.off), in.a,
                      [](uint32_t x, uint32_t w) { return __uint_as_float(x) == __uint_as_float(w); }, m);
        break;
    }
    case OP_IN64: {
        uint64_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x64(col_base, c0[g], lane, v[g]);
        in_list<G, (G == 1 ? 8 : G == 2 ? 4 : 2)>(v, reinterpret_cast<const uint64_t*>(pool + in.off), in.a,
                      [](uint64_t x, uint64_t w) { return x == w; }, m);
        break;
    }
    case OP_BITMAP: {
        uint32_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x32(col_base, c0[g], lane, v[g]);
        const uint32_t* words = reinterpret_cast<const uint32_t*>(pool + in.off);
        const uint32_t lo = in.a, nbits = in.b;
#pragma unroll
        for (int g = 0; g < G; ++g)
            m[g] = mask8([&](int i) {
                const uint32_t d = v[g][i] - lo;
                return d < nbits && ((words[d >> 5] >> (d & 31u)) & 1u);
            });
        break;
    }
    case OP_HASH32: {
        uint32_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x32(col_base, c0[g], lane, v[g]);
        const uint32_t* tab = reinterpret_cast<const uint32_t*>(pool + in.off);
        const uint32_t mul = in.a, sh = in.b;
#pragma unroll
        for (int g = 0; g < G; ++g) m[g] = mask8([&](int i) { return tab[(v[g][i] * mul) >> sh] == v[g][i]; });
        break;
    }
    case OP_HASH64: {
        uint64_t v[G][8];
#pragma unroll
        for (int g = 0; g < G; ++g) load8x64(col_base, c0[g], lane, v[g]);
        const uint64_t* tab = reinterpret_cast<const uint64_t*>(pool + in.off);
        const uint32_t mul = in.a, sh = in.b;
#pragma unroll
        for (int g = 0; g < G; ++g)
            m[g] = mask8([&](int i) {
                const uint32_t k = static_cast<uint32_t>(v[g][i]) ^ static_cast<uint32_t>(v[g][i] >> 32);
                return tab[(k * mul) >> sh] == v[g][i];
            });
        break;
    }
    default:  // OP_CONST
#pragma unroll
        for (int g = 0; g < G; ++g) m[g] = 0xFFu;
        break;
    }
    if (in.neg) {
#pragma unroll
        for (int g = 0; g < G; ++g) m[g] ^= 0xFFu;
    }
}

// Runs a compiled program over G 256-row chunks of a staged tile with one
// pass over the instructions; m[g] is the lane's 8-bit row mask of chunk g.
// stage_base: shared address of the staged tile; slot_off: byte offset of
// each slot's column inside the stage.  The next instruction is fetched
// while the current one is evaluated.
template <int G>
__device__ __forceinline__ void eval_program_g(const Instr* __restrict__ prog, uint32_t n_instr,
                                               const uint8_t* __restrict__ pool, uint32_t stage_base,
                                               const uint32_t* slot_off, const uint32_t (&c0)[G], uint32_t lane,
                                               uint32_t (&top)[G]) {
    uint64_t stk[G];     // up to 8 pending 8-bit masks per chunk
    uint32_t memo[G];    // kMemoSlots saved 8-bit masks of repeated leaves
#pragma unroll
    for (int g = 0; g < G; ++g) {
        top[g] = 0;
        stk[g] = 0;
        memo[g] = 0;
    }
    if (n_instr == 0) return;
    Instr nxt = prog[0];
    for (uint32_t pc = 0; pc < n_instr; ++pc) {
        const Instr in = nxt;
        if (pc + 1 < n_instr) nxt = prog[pc + 1];
        if (in.opc == OP_RANGE32 || in.opc == OP_RANGEF || in.opc == OP_MASK32) {
            // the most frequent leaves (ranges over 4-byte columns, small code
            // sets) first and inline: measured 4-13 % fewer instructions per
            // leaf than through the switch; negation as an XOR mask
            // (a clamped funnel shift tests MASK32: offsets >= 32 give 0)
            const uint32_t cb = stage_base + slot_off[in.slot];
            const uint32_t negm = in.neg ? 0xFFu : 0u;
            uint32_t m[G];
            uint32_t v[G][8];
#pragma unroll
            for (int g = 0; g < G; ++g) load8x32(cb, c0[g], lane, v[g]);
            if (in.opc == OP_RANGE32) {
                const uint32_t lo = in.a, sp = in.b;
#pragma unroll
                for (int g = 0; g < G; ++g) m[g] = mask8([&](int i) { return v[g][i] - lo <= sp; }) ^ negm;
            } else if (in.opc == OP_RANGEF) {
                const float lo = __uint_as_float(in.a), hi = __uint_as_float(in.b);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    m[g] = mask8([&](int i) {
                        const float x = __uint_as_float(v[g][i]);
                        return lo <= x && x <= hi;
                    }) ^ negm;
            } else {
                const uint32_t lo = in.a, word = in.b;
#pragma unroll
                for (int g = 0; g < G; ++g)
                    m[g] = mask8_bits([&](int i) { return __funnelshift_rc(word, 0u, v[g][i] - lo) & 1u; }) ^ negm;
            }
            if (in.comb == OP_AND) {
#pragma unroll
                for (int g = 0; g < G; ++g) top[g] &= m[g];
            } else if (in.comb == OP_OR) {
#pragma unroll
                for (int g = 0; g < G; ++g) top[g] |= m[g];
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    stk[g] = (stk[g] << 8) | top[g];
                    top[g] = m[g];
                }
            }
        } else if (in.opc == OP_AND) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                top[g] &= static_cast<uint32_t>(stk[g]) & 0xFFu;
                stk[g] >>= 8;
            }
        } else if (in.opc == OP_OR) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                top[g] |= static_cast<uint32_t>(stk[g]) & 0xFFu;
                stk[g] >>= 8;
            }
        } else if (in.opc == OP_SAVE) {
            const uint32_t sh = 8u * in.a;
#pragma unroll
            for (int g = 0; g < G; ++g) memo[g] = (memo[g] & ~(0xFFu << sh)) | (top[g] << sh);
        } else {
            // a leaf, CONST or LOAD: push its mask, or combine it into the top
            uint32_t m[G];
            if (in.opc == OP_LOAD) {
#pragma unroll
                for (int g = 0; g < G; ++g) m[g] = (memo[g] >> (8u * in.a)) & 0xFFu;
            } else {
                eval_leaf_g<G>(in, stage_base + slot_off[in.slot], c0, lane, pool, m);
            }
            if (in.comb == OP_AND) {
#pragma unroll
                for (int g = 0; g < G; ++g) top[g] &= m[g];
            } else if (in.comb == OP_OR) {
#pragma unroll
                for (int g = 0; g < G; ++g) top[g] |= m[g];
            } else {
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    stk[g] = (stk[g] << 8) | top[g];
                    top[g] = m[g];
                }
            }
        }
    }
}

// One chunk: the lane's 8-bit row mask of the 256-row chunk at tile row c0.
__device__ __forceinline__ uint32_t eval_program(const Instr* __restrict__ prog, uint32_t n_instr,
                                                 const uint8_t* __restrict__ pool, uint32_t stage_base,
                                                 const uint32_t* slot_off, uint32_t c0, uint32_t lane) {
    const uint32_t c[1] = {c0};
    uint32_t m[1];
    eval_program_g<1>(prog, n_instr, pool, stage_base, slot_off, c, lane, m);
    return m[0];
}

// ---------------------------------------------------------------------------
// tiles of a multi-table scan launch (count and bucket kernels)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_table(const ScanArgs& a, int64_t g) {
    int t = 0;
    while (t + 1 < static_cast<int>(a.n_tables) && g >= a.t[t + 1].tile_begin) ++t;
    return t;
}

__device__ __forceinline__ uint32_t tile_valid(const ScanArgs& a, const TableArg& T, int64_t g) {
    const int64_t r0 = (g - T.tile_begin) * static_cast<int64_t>(a.tile_rows);
    const int64_t left = T.n_rows - r0;
    return static_cast<uint32_t>(left < static_cast<int64_t>(a.tile_rows) ? left : a.tile_rows);
}

// Producer warp: fills stage s with tile g (all 32 lanes call this).
__device__ __forceinline__ void produce_tile(const ScanArgs& a, int64_t g, uint32_t s, uint8_t* stages,
                                             uint64_t* full, uint64_t pol, uint32_t lane) {
    const TableArg& T = a.t[find_table(a, g)];
    const int64_t r0 = (g - T.tile_begin) * static_cast<int64_t>(a.tile_rows);
    const uint32_t valid = tile_valid(a, T, g);
    uint8_t* st = stages + static_cast<size_t>(s) * a.stage_bytes;
    if (T.tma && valid == a.tile_rows && T.row_bytes > 0) {
        if (lane == 0) {
            mbar_arrive_expect_tx(&full[s], a.tile_rows * T.row_bytes);
            for (uint32_t j = 0; j < T.n_slots; ++j)
                bulk_g2s(st + T.slot_off[j], T.col[j] + r0 * T.width[j], a.tile_rows * T.width[j], &full[s], pol);
        }
    } else {
        for (uint32_t j = 0; j < T.n_slots; ++j) {
            const uint32_t words = valid * T.width[j] / 4u;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(T.col[j] + r0 * T.width[j]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(st + T.slot_off[j]);
            for (uint32_t i = lane; i < words; i += 32) dst[i] = src[i];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);   // release: the copies above are visible to the waiters
    }
}

// Mask of the lane's rows that lie below `valid` rows of the tile.
__device__ __forceinline__ uint32_t valid_mask(uint32_t c0, uint32_t lane, uint32_t valid) {
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        m |= (c0 + 4u * lane + i < valid ? 1u : 0u) << i;
        m |= (c0 + 128u + 4u * lane + i < valid ? 1u : 0u) << (4 + i);
    }
    return m;
}

// Row (within the tile) of mask bit b for lane l of the chunk at c0.
__device__ __forceinline__ uint32_t bit_row(uint32_t c0, uint32_t lane, uint32_t b) {
    return c0 + (b >> 2) * 128u + 4u * lane + (b & 3u);
}

}  // namespace sel
