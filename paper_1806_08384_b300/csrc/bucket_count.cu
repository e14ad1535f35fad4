// bucket_count.cu -- batched filtered COUNT over the column-bucket form of
// the probes (layout in bucket.h): many selectivity probes of one query
// optimisation (§3.1's COUNT per relation, batched) share one pass over every
// referenced column, and every probe's predicate follows from one bucket
// index per column and row.
//
// Warp roles and the tile pipeline are those of the interpreter's count scan
// (count.cu): a producer warp fills `stages` shared-memory stages with column
// tiles by bulk copies, W consumer warps take the tile's 256-row chunks in
// rotation and release each stage as they finish.  A lane owns 8 rows of a
// chunk (the same row mapping as the interpreter).  For each chunk a consumer
// warp
//   1. finds each row's bucket on every column the table's probes read (a
//      cell table indexed by the value's high bits and at most 3 compares, a
//      branch-free binary search over the sorted boundaries, or a linear count
//      for a few boundaries; all in shared memory); with several blocks of
//      probes on the table the indices go to a per-warp shared buffer and are
//      reused by every block;
//   2. per block, ANDs the gm words of the row's buckets into the row's group
//      words (4 rows x up to 8 words in registers at a time, two halves);
//   3. ORs each program's 4 group bits into the low bit of its field, sums the
//      8 rows' fields (each field stays <= 8), reduces 16-bit fields over the
//      warp and adds each program's chunk count to a per-CTA counter.
// At the end each CTA adds its counters to the launch's counts.
#include <algorithm>

#include "bucket.h"
#include "kernels.h"
#include "scan.cuh"

namespace sel {

namespace {

// Bucket index of each of R values of the lane on one column.
template <typename T, int R>
__device__ __forceinline__ void bucket_rows(const BkSlot& sl, const uint8_t* blob, const T (&v)[R],
                                            uint32_t (&idx)[R]) {
    const T* __restrict__ bnd = reinterpret_cast<const T*>(blob + sl.bnd_off);
    const uint32_t k = sl.k;
    const uint32_t mode = sl.mode;
    if (mode == BK_CELLS || mode == BK_CELLS_BIN) {
        // cell c = (x - lo) >> shift, clamped to the last cell above the
        // boundaries' span; below lo every boundary is above x: bucket 0
        const uint16_t* __restrict__ cells = reinterpret_cast<const uint16_t*>(blob + sl.cells_off);
        const T lo = static_cast<T>(sl.lo);
        const uint32_t shift = sl.shift, last = sl.n_cells - 1u, occ = sl.occ;
        const T* base[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const T c = (v[i] - lo) >> shift;
            const uint32_t cc = v[i] < lo ? 0u : (c > static_cast<T>(last) ? last : static_cast<uint32_t>(c));
            const uint32_t b0 = cells[cc];
            idx[i] = v[i] < lo ? 0u : b0;
            base[i] = bnd + b0;
        }
        if (mode == BK_CELLS_BIN) {
            // boundaries past the cell are above x: the search stays inside it
            for (uint32_t h = sl.half; h; h >>= 1) {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const uint32_t j = idx[i] + h;
                    if (v[i] >= bnd[j - 1]) idx[i] = j;
                }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) idx[i] = min(idx[i], k);
            return;
        }
#pragma unroll
        for (uint32_t t = 0; t < (uint32_t)kBkMaxOcc; ++t) {
            if (t >= occ) break;
#pragma unroll
            for (int i = 0; i < R; ++i) idx[i] += v[i] >= base[i][t] ? 1u : 0u;
        }
        if (occ)
#pragma unroll
            for (int i = 0; i < R; ++i) idx[i] = min(idx[i], k);
        return;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) idx[i] = 0;
    if (mode == BK_LINEAR) {
        for (uint32_t j = 0; j < k; ++j) {
            const T b = bnd[j];
#pragma unroll
            for (int i = 0; i < R; ++i) idx[i] += v[i] >= b ? 1u : 0u;
        }
        return;
    }
    for (uint32_t h = sl.half; h; h >>= 1) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const uint32_t j = idx[i] + h;
            if (v[i] >= bnd[j - 1]) idx[i] = j;
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) idx[i] = min(idx[i], k);
}

// Bucket indices of R of the lane's rows of the chunk at c0 on one slot: all
// 8 (R = 8), or half h (mask bits 4h .. 4h + 3, R = 4; one 16-byte load of a
// 4-byte column).
template <int R>
__device__ __forceinline__ void slot_buckets(const uint8_t* blob, const BkSlot& sl, uint32_t width, uint32_t col_addr,
                                             uint32_t c0, uint32_t lane, uint32_t h, uint32_t (&idx)[R]) {
    if (width == 8) {
        uint64_t v[R];
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint32_t p = col_addr + c0 * 8u + lane * 32u + (h + q) * 1024u;
            const uint4 a = lds128(p), b = lds128(p + 16u);
            v[4 * q + 0] = (uint64_t)a.y << 32 | a.x;
            v[4 * q + 1] = (uint64_t)a.w << 32 | a.z;
            v[4 * q + 2] = (uint64_t)b.y << 32 | b.x;
            v[4 * q + 3] = (uint64_t)b.w << 32 | b.z;
        }
        bucket_rows<uint64_t, R>(sl, blob, v, idx);
    } else {
        uint32_t v[R];
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint4 a = lds128(col_addr + c0 * 4u + lane * 16u + (h + q) * 512u);
            v[4 * q + 0] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
        bucket_rows<uint32_t, R>(sl, blob, v, idx);
    }
}

// Adds each program's row count to its per-CTA counter: N0 (and N1 when two
// chunks were evaluated) hold, per group word, the number of the lane's rows
// where the program holds, in the low bits of its 4-bit field (<= 8 per
// chunk).  The fields are widened to 16 bits, summed over the warp, and lane
// j < 8 adds field j of each word.
template <int NW>
__device__ __forceinline__ void count_fields(const uint8_t* blob, const BkBlock& bk, const uint32_t (&N0)[NW],
                                             const uint32_t (&N1)[NW], uint32_t chunks, uint32_t lane,
                                             uint32_t* cnt) {
    const uint32_t* outs = reinterpret_cast<const uint32_t*>(blob + bk.out_off);
    const uint32_t n_words = bk.n_words, n_progs = bk.n_progs;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        if ((uint32_t)w >= n_words) break;
        const uint32_t a = N0[w], b = chunks > 1 ? N1[w] : 0u;
        const uint32_t f0 = __reduce_add_sync(0xFFFFFFFFu, (a & 0x000F000Fu) + (b & 0x000F000Fu));                 // fields 0, 4
        const uint32_t f1 = __reduce_add_sync(0xFFFFFFFFu, ((a >> 4) & 0x000F000Fu) + ((b >> 4) & 0x000F000Fu));   // 1, 5
        const uint32_t f2 = __reduce_add_sync(0xFFFFFFFFu, ((a >> 8) & 0x000F000Fu) + ((b >> 8) & 0x000F000Fu));   // 2, 6
        const uint32_t f3 = __reduce_add_sync(0xFFFFFFFFu, ((a >> 12) & 0x000F000Fu) + ((b >> 12) & 0x000F000Fu)); // 3, 7
        const uint32_t j = lane & 7u;
        const uint32_t pair = (j & 3u) == 0 ? f0 : (j & 3u) == 1 ? f1 : (j & 3u) == 2 ? f2 : f3;
        const uint32_t c = (pair >> (16u * (j >> 2))) & 0xFFFFu;
        const uint32_t k = 8u * (uint32_t)w + j;
        if (lane < 8 && k < n_progs && c) atomicAdd(&cnt[outs[k]], c);
    }
}

// One block of probes on the lane's 8 rows (vm: the rows that exist), ROWS
// rows at a time (8, or two halves of 4 for 8-word blocks, which keeps the
// group words in registers).  NW: gm words the block reads per row.  gbuf:
// the warp's bucket indices of every slot (null: search here).
template <int NW>
__device__ __forceinline__ void eval_block(const uint8_t* blob, const BkTable& bt, const BkBlock& bk,
                                           const TableArg& T, const uint32_t* s_off, uint32_t st_addr, uint32_t c0,
                                           uint32_t lane, uint32_t vm, const uint16_t* gbuf, uint32_t gstride,
                                           uint32_t* cnt) {
    constexpr int STRIDE = NW == 8 ? 12 : NW;
    constexpr int ROWS = NW == 8 ? 4 : 8;
    uint32_t N[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) N[w] = 0;
    const uint32_t n_used = bk.n_used;
#pragma unroll 1
    for (uint32_t h = 0; h < 8u / ROWS; ++h) {
        uint32_t R[ROWS][NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t init = bk.init[w];
#pragma unroll
            for (int i = 0; i < ROWS; ++i) R[i][w] = ((vm >> (ROWS * h + i)) & 1u) ? init : 0u;
        }
        for (uint32_t u = 0; u < n_used; ++u) {
            const uint32_t s = bk.used[u];
            uint32_t b[ROWS];
            if (gbuf) {
#pragma unroll
                for (int i = 0; i < ROWS; ++i) b[i] = gbuf[(s * gstride + ROWS * h + i) * 32u + lane];
            } else {
                slot_buckets<ROWS>(blob, bt.slot[s], T.width[s], st_addr + s_off[s], c0, lane, h, b);
            }
            const uint32_t ro = bk.remap_off[u];
            if (ro != kBkIdentity) {
                const uint16_t* rm = reinterpret_cast<const uint16_t*>(blob + ro);
#pragma unroll
                for (int i = 0; i < ROWS; ++i) b[i] = rm[b[i]];
            }
            const uint32_t* gm = reinterpret_cast<const uint32_t*>(blob + bk.gm_off[u]);
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                const uint32_t* row = gm + b[i] * STRIDE;
                if (NW == 1) {
                    R[i][0] &= row[0];
                } else if (NW == 2) {
                    const uint2 x = *reinterpret_cast<const uint2*>(row);
                    R[i][0] &= x.x;
                    R[i][NW > 1 ? 1 : 0] &= x.y;
                } else {
#pragma unroll
                    for (int q = 0; q < NW / 4; ++q) {
                        const uint4 x = *reinterpret_cast<const uint4*>(row + 4 * q);
                        R[i][4 * q + 0] &= x.x;
                        R[i][4 * q + 1] &= x.y;
                        R[i][4 * q + 2] &= x.z;
                        R[i][4 * q + 3] &= x.w;
                    }
                }
            }
        }
#pragma unroll
        for (int w = 0; w < NW; ++w)
#pragma unroll
            for (int i = 0; i < ROWS; ++i) {
                uint32_t t = R[i][w] | (R[i][w] >> 1);
                t |= t >> 2;
                N[w] += t & 0x11111111u;   // field k's OR in bit 4k; a field's sum over 8 rows is <= 8
            }
    }
    count_fields<NW>(blob, bk, N, N, 1, lane, cnt);
}

// A block of at most 2 group words on two chunks at once (16 rows of the lane
// per pass: twice the independent work of eval_block for the same loads of
// the block's parameters).
template <int NW>
__device__ __forceinline__ void eval_block2(const uint8_t* blob, const BkTable& bt, const BkBlock& bk,
                                            const TableArg& T, const uint32_t* s_off, uint32_t st_addr,
                                            const uint32_t (&c0)[2], uint32_t lane, const uint32_t (&vm)[2],
                                            const uint16_t* gbuf, uint32_t* cnt) {
    uint32_t R[16][NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t init = bk.init[w];
#pragma unroll
        for (int r = 0; r < 16; ++r) R[r][w] = ((vm[r >> 3] >> (r & 7)) & 1u) ? init : 0u;
    }
    const uint32_t n_used = bk.n_used;
    for (uint32_t u = 0; u < n_used; ++u) {
        const uint32_t s = bk.used[u];
        uint32_t b[16];
        if (gbuf) {
#pragma unroll
            for (int r = 0; r < 16; ++r) b[r] = gbuf[(s * 16u + r) * 32u + lane];
        } else {
            const BkSlot& sl = bt.slot[s];
            const uint32_t col = st_addr + s_off[s];
            if (T.width[s] == 8) {
                uint64_t v[16];
                load8x64(col, c0[0], lane, *reinterpret_cast<uint64_t(*)[8]>(&v[0]));
                load8x64(col, c0[1], lane, *reinterpret_cast<uint64_t(*)[8]>(&v[8]));
                bucket_rows<uint64_t, 16>(sl, blob, v, b);
            } else {
                uint32_t v[16];
                load8x32(col, c0[0], lane, *reinterpret_cast<uint32_t(*)[8]>(&v[0]));
                load8x32(col, c0[1], lane, *reinterpret_cast<uint32_t(*)[8]>(&v[8]));
                bucket_rows<uint32_t, 16>(sl, blob, v, b);
            }
        }
        const uint32_t ro = bk.remap_off[u];
        if (ro != kBkIdentity) {
            const uint16_t* rm = reinterpret_cast<const uint16_t*>(blob + ro);
#pragma unroll
            for (int r = 0; r < 16; ++r) b[r] = rm[b[r]];
        }
        const uint32_t* gm = reinterpret_cast<const uint32_t*>(blob + bk.gm_off[u]);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const uint32_t* row = gm + b[r] * NW;
            if (NW == 1) {
                R[r][0] &= row[0];
            } else {
                const uint2 x = *reinterpret_cast<const uint2*>(row);
                R[r][0] &= x.x;
                R[r][NW > 1 ? 1 : 0] &= x.y;
            }
        }
    }
    uint32_t N0[NW], N1[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        N0[w] = 0;
        N1[w] = 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            uint32_t t = R[r][w] | (R[r][w] >> 1);
            t |= t >> 2;
            if (r < 8)
                N0[w] += t & 0x11111111u;
            else
                N1[w] += t & 0x11111111u;
        }
    }
    count_fields<NW>(blob, bk, N0, N1, 2, lane, cnt);
}

__device__ __forceinline__ uint32_t lds_u16(uint32_t addr) {
    uint32_t v;
    asm("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// The bucket record of every row of the chunk at c0 (quad form): entry
// e = 32 i + lane (the lane's row i) holds the bucket index of slot s at
// uint16 s of its 16 bytes; rows past the table's end (vm bit clear) get
// index k + 1, whose remap entry reads the all-zero row.
__device__ __forceinline__ void fill_records(const uint8_t* blob, const BkTable& bt, const TableArg& T,
                                             const uint32_t* s_off, uint32_t st_addr, uint32_t c0, uint32_t lane,
                                             uint32_t vm, uint32_t rec_addr) {
    for (uint32_t sl = 0; sl < bt.n_slots; ++sl) {
        uint32_t b[8];
        slot_buckets<8>(blob, bt.slot[sl], T.width[sl], st_addr + s_off[sl], c0, lane, 0u, b);
        if (vm != 0xFFu) {
            const uint32_t past = bt.slot[sl].k + 1u;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (!((vm >> i) & 1u)) b[i] = past;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t a = rec_addr + ((32u * i + lane) * 8u + sl) * 2u;
            asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"(static_cast<unsigned short>(b[i])) : "memory");
        }
    }
}

// The 4-bit fields of w, each OR-ed into its low bit (bit 4k).
__device__ __forceinline__ uint32_t field_any(uint32_t w) {
    uint32_t t = w | (w >> 1);
    t |= t >> 2;
    return t & 0x11111111u;
}

// One quad on one chunk whose row records are at rec_addr (NS slots): quarter
// qq takes rows e = 4t + qq; in it lane pair p ANDs block p's group words
// (lane h of the pair words 4h .. 4h + 3) over the slots, ORs each program's
// group bits and counts them in 4-bit fields (flushed every 8 rows into
// 8-bit fields).  At the end the 4 quarters' counts are summed and each
// program's count is added to the per-CTA counters.
template <int NS>
__device__ __forceinline__ void eval_quad(const uint8_t* blob, const BkQuad& Q, uint32_t blob_addr, uint32_t rec_addr,
                                          uint32_t lane, uint32_t* cnt) {
    const uint32_t qq = lane >> 3, p = (lane >> 1) & 3u, h = lane & 1u;
    uint32_t rmb[NS], gmb[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        rmb[u] = blob_addr + Q.remap_off[u] + 2u * p;
        gmb[u] = blob_addr + Q.gm_off[u] + 32u * p + 16u * h;
    }
    uint32_t N[4] = {0u, 0u, 0u, 0u}, C[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    const uint32_t rec0 = rec_addr + qq * 16u;
#pragma unroll 1
    for (uint32_t t8 = 0; t8 < 64u; t8 += 8u) {
#pragma unroll 2
        for (uint32_t t = t8; t < t8 + 8u; ++t) {
            const uint4 r = lds128(rec0 + t * 64u);
            const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
            uint32_t R[4];
#pragma unroll
            for (int u = 0; u < NS; ++u) {
                const uint32_t b = (u & 1) ? (rw[u >> 1] >> 16) : (rw[u >> 1] & 0xFFFFu);
                const uint32_t l = lds_u16(rmb[u] + b * 8u);
                const uint4 x = lds128(gmb[u] + l * 128u);
                if (u == 0) {
                    R[0] = x.x;
                    R[1] = x.y;
                    R[2] = x.z;
                    R[3] = x.w;
                } else {
                    R[0] &= x.x;
                    R[1] &= x.y;
                    R[2] &= x.z;
                    R[3] &= x.w;
                }
            }
#pragma unroll
            for (int w = 0; w < 4; ++w) N[w] += field_any(R[w]);   // a field stays <= 8
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {   // fields 0, 2, 4, 6 and 1, 3, 5, 7 into bytes (<= 64 a chunk)
            C[2 * w] += N[w] & 0x0F0F0F0Fu;
            C[2 * w + 1] += (N[w] >> 4) & 0x0F0F0F0Fu;
            N[w] = 0u;
        }
    }
    // bytes to 16-bit halves (field f of word w: C[2w + (f & 1)], byte f / 2),
    // summed over the quarters (<= 256)
    uint32_t H[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        H[2 * j] = C[j] & 0x00FF00FFu;             // bytes 0, 2
        H[2 * j + 1] = (C[j] >> 8) & 0x00FF00FFu;  // bytes 1, 3
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        H[j] += __shfl_xor_sync(0xFFFFFFFFu, H[j], 8);
        H[j] += __shfl_xor_sync(0xFFFFFFFFu, H[j], 16);
    }
    // quarter qq adds word w = qq of the lane's 4: fields f = 0..7 of block
    // p's word 4h + qq, i.e. program 8 (4h + qq) + f
    uint32_t cf[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) {
        cf[f] = 0u;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            // C[2w + (f & 1)] byte f / 2: byte 0 or 2 -> H[2j] low/high half, byte 1 or 3 -> H[2j + 1]
            const int j = 2 * w + (f & 1), byte = f >> 1;
            const uint32_t hv = H[2 * j + (byte & 1)];
            if ((uint32_t)w == qq) cf[f] = (byte >> 1) ? (hv >> 16) : (hv & 0xFFFFu);
        }
    }
    // lane (p, h) of a quarter takes its fields in the order rot, rot + 1, ...
    // (rot = 2p + h): the 32 lanes of one add then hit 32 different banks
    // (program 8 (4h + qq) + f of block p sits in bank 8 qq + f when the
    // probes' counters are in order); cf is rotated by rot in 3 select steps
    const uint32_t rot = 2u * p + h;
#pragma unroll
    for (int st = 1; st < 8; st <<= 1) {
        const bool take = (rot & (uint32_t)st) != 0u;
        uint32_t nx[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) nx[f] = take ? cf[(f + st) & 7] : cf[f];
#pragma unroll
        for (int f = 0; f < 8; ++f) cf[f] = nx[f];
    }
    const uint32_t* outs = reinterpret_cast<const uint32_t*>(blob + Q.out_off) + 64u * p + 8u * (4u * h + qq);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t o = outs[(i + rot) & 7u];
        if (cf[i] && o != kBkNoOut) atomicAdd(&cnt[o], cf[i]);
    }
}

// Every quad of a quad table on the chunk at c0 (the warp's records at
// rec_addr are rewritten for each chunk).
__device__ __forceinline__ void eval_quads(const uint8_t* blob, const BkTable& bt, const TableArg& T,
                                           const uint32_t* s_off, uint32_t st_addr, uint32_t c0, uint32_t lane,
                                           uint32_t vm, uint32_t rec_addr, uint32_t* cnt) {
    fill_records(blob, bt, T, s_off, st_addr, c0, lane, vm, rec_addr);
    __syncwarp();
    const BkQuad* quads = reinterpret_cast<const BkQuad*>(blob + bt.quad_off);
    const uint32_t blob_addr = smem_u32(blob);
    for (uint32_t qi = 0; qi < bt.n_quads; ++qi) {
        const BkQuad& Q = quads[qi];
        switch (Q.n_used) {
        case 1: eval_quad<1>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 2: eval_quad<2>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 3: eval_quad<3>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 4: eval_quad<4>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 5: eval_quad<5>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 6: eval_quad<6>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        case 7: eval_quad<7>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        default: eval_quad<8>(blob, Q, blob_addr, rec_addr, lane, cnt); break;
        }
    }
    __syncwarp();   // the records are rewritten for the next chunk
}

// All blocks of a table on G chunks (c0[q], valid rows vm[q]; vm 0: no chunk).
template <int G>
__device__ __forceinline__ void eval_chunks(const uint8_t* blob, const BkTable& bt, const TableArg& T,
                                            const uint32_t* s_off, uint32_t st_addr, const uint32_t (&c0)[G],
                                            uint32_t lane, const uint32_t (&vm)[G], uint32_t n_have, uint16_t* gbuf,
                                            uint32_t* cnt) {
    if (bt.n_quads > 0) {
        const uint32_t rec_addr = smem_u32(gbuf);
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if ((uint32_t)q >= n_have) break;   // the group's missing chunk (the same on every lane)
            eval_quads(blob, bt, T, s_off, st_addr, c0[q], lane, vm[q], rec_addr, cnt);
        }
        return;
    }
    const BkBlock* blocks = reinterpret_cast<const BkBlock*>(blob + bt.block_off);
    const uint32_t n_blocks = bt.n_blocks;
    const uint16_t* gb = nullptr;
    if (n_blocks > 1) {   // every slot's bucket indices once, for all blocks
        for (uint32_t sl = 0; sl < bt.n_slots; ++sl)
#pragma unroll
            for (int q = 0; q < G; ++q) {
                uint32_t b[8];
                slot_buckets<8>(blob, bt.slot[sl], T.width[sl], st_addr + s_off[sl], c0[q], lane, 0u, b);
#pragma unroll
                for (int i = 0; i < 8; ++i) gbuf[(sl * 8u * G + 8u * q + i) * 32u + lane] = (uint16_t)b[i];
            }
        gb = gbuf;
    }
    for (uint32_t bi = 0; bi < n_blocks; ++bi) {
        const BkBlock& bk = blocks[bi];
        const uint32_t nw = bk.nw;
        if (G == 2 && nw <= 2) {
            const uint32_t (&c2)[2] = *reinterpret_cast<const uint32_t(*)[2]>(&c0[0]);
            const uint32_t (&v2)[2] = *reinterpret_cast<const uint32_t(*)[2]>(&vm[0]);
            if (nw == 1)
                eval_block2<1>(blob, bt, bk, T, s_off, st_addr, c2, lane, v2, gb, cnt);
            else
                eval_block2<2>(blob, bt, bk, T, s_off, st_addr, c2, lane, v2, gb, cnt);
            continue;
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if ((uint32_t)q >= n_have) break;   // the group's missing chunk (the same on every lane)
            const uint16_t* g = gb ? gb + 8u * q * 32u : nullptr;
            const uint32_t gs = 8u * G;
            switch (nw) {
            case 1: eval_block<1>(blob, bt, bk, T, s_off, st_addr, c0[q], lane, vm[q], g, gs, cnt); break;
            case 2: eval_block<2>(blob, bt, bk, T, s_off, st_addr, c0[q], lane, vm[q], g, gs, cnt); break;
            case 4: eval_block<4>(blob, bt, bk, T, s_off, st_addr, c0[q], lane, vm[q], g, gs, cnt); break;
            default: eval_block<8>(blob, bt, bk, T, s_off, st_addr, c0[q], lane, vm[q], g, gs, cnt); break;
            }
        }
    }
}

template <int W, int G>
__device__ __forceinline__ void consume_buckets(const ScanArgs& a, const uint8_t* blob, uint64_t* full, uint64_t* empty,
                                                uint32_t* cnt, uint8_t* stages, uint16_t* gbuf_all,
                                                const uint32_t (&s_off)[kMaxTables][kMaxSlots], uint32_t* s_fail,
                                                uint32_t warp, uint32_t lane) {
    const BkHeader* hdr = reinterpret_cast<const BkHeader*>(blob);
    const int64_t NB = gridDim.x;
    const uint32_t S = a.stages;
    uint16_t* gbuf = gbuf_all + (size_t)warp * (bk_gb_bytes_per_warp(hdr->gb_slots, hdr->gb_quad, G) / 2u);
    uint32_t rot = 0;   // running chunk-group count: group c of a tile belongs to warp (rot + c) % W
    uint32_t s = 0, parity = 0;
    for (int64_t k = 0;; ++k) {
        const int64_t g = blockIdx.x + k * NB;
        if (g >= a.total_tiles) break;
        const int ti = find_table(a, g);
        const TableArg& T = a.t[ti];
        const BkTable& bt = hdr->t[ti];
        const uint32_t valid = tile_valid(a, T, g);
        const uint32_t n_chunks = (valid + kChunkRows - 1) / kChunkRows;
        const uint32_t n_groups = (n_chunks + G - 1) / G;
        const uint32_t first = (warp + W - rot % W) % W;
        const bool okw = __all_sync(0xFFFFFFFFu, mbar_wait_bounded(&full[s], parity));
        if (!okw) {
            if (lane == 0) {
                atomicOr(a.err, 1u);
                atomicOr(s_fail, 1u);
                mbar_wait_bounded(&full[s], parity);
            }
            break;
        }
        if (*reinterpret_cast<volatile uint32_t*>(s_fail)) break;
        const uint32_t st_addr = smem_u32(stages + static_cast<size_t>(s) * a.stage_bytes);
        for (uint32_t grp = first; grp < n_groups; grp += W) {
            uint32_t c0[G], vm[G];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                const uint32_t ch = grp * G + q;
                // a missing chunk of the last group re-reads the group's first chunk, with no rows
                c0[q] = (ch < n_chunks ? ch : grp * G) * kChunkRows;
                vm[q] = ch >= n_chunks ? 0u
                        : (c0[q] + kChunkRows <= valid) ? 0xFFu
                                                          : valid_mask(c0[q], lane, valid);
            }
            eval_chunks<G>(blob, bt, T, s_off[ti], st_addr, c0, lane, vm, min((uint32_t)G, n_chunks - grp * G),
                           gbuf, cnt);
        }
        rot += n_groups;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (++s == S) {
            s = 0;
            parity ^= 1u;
        }
    }
}

}  // namespace

template <int W, int G>
__global__ void __launch_bounds__((W + 1) * 32, 1) bucket_count_kernel(const __grid_constant__ ScanArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ uint32_t s_off[kMaxTables][kMaxSlots];
    __shared__ uint32_t s_fail;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t S = a.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + S;
    // per-CTA counts: 32 bits (a CTA scans fewer than 2^32 rows: checked on the host)
    uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + a.cnt_off);
    uint8_t* stages = smem + a.stage_off;

    if (tid == 0) {
        for (uint32_t s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], W);
        }
        fence_mbar_init();
        s_fail = 0;
    }
    for (uint32_t i = tid; i < kMaxTables * kMaxSlots; i += blockDim.x)
        s_off[i / kMaxSlots][i % kMaxSlots] = a.t[i / kMaxSlots].slot_off[i % kMaxSlots];
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x) cnt[p] = 0u;
    {
        uint4* dst = reinterpret_cast<uint4*>(smem + a.prog_off);
        const uint4* src = reinterpret_cast<const uint4*>(a.blob);
        for (uint32_t i = tid; i < a.blob_bytes / 16u; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int64_t NB = gridDim.x;

    if (warp == W) {
        const uint64_t pol = policy_evict_first();
        uint32_t s = 0, phase = 0;
        for (int64_t k = 0;; ++k) {
            const int64_t g = blockIdx.x + k * NB;
            if (g >= a.total_tiles) break;
            if (k >= S) {
                const bool ok = mbar_wait_bounded(&empty[s], phase ^ 1u);
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    if (lane == 0) {
                        atomicOr(a.err, 1u);
                        atomicOr(&s_fail, 1u);
                    }
                    break;
                }
            }
            produce_tile(a, g, s, stages, full, pol, lane);
            if (++s == S) {
                s = 0;
                phase ^= 1u;
            }
        }
    } else {
        consume_buckets<W, G>(a, smem + a.prog_off, full, empty, cnt, stages,
                           reinterpret_cast<uint16_t*>(smem + a.aux_off), s_off, &s_fail, warp, lane);
    }
    __syncthreads();
    if (s_fail) return;
    for (uint32_t p = tid; p < a.n_progs; p += blockDim.x)
        if (cnt[p]) atomicAdd(&a.counts[p], static_cast<unsigned long long>(cnt[p]));
}

static inline uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

size_t bucket_layout(ScanArgs& a, int warps, uint32_t gb_bytes_per_warp) {
    a.prog_in_smem = 1;
    a.cnt_off = align_up(16u * a.stages, 16u);
    a.prog_off = align_up(a.cnt_off + 4u * a.n_progs, 16u);
    a.aux_off = align_up(a.prog_off + align_up(a.blob_bytes, 16u), 16u);
    a.stage_off = align_up(a.aux_off + (uint32_t)warps * gb_bytes_per_warp, 128u);
    return static_cast<size_t>(a.stage_off) + static_cast<size_t>(a.stages) * a.stage_bytes;
}

// 15 and 11 consumer warps (16 and 12 warps in all: 4 and 3 per scheduler's
// register file) get 128 and 168 registers a thread; 16 consumer warps put 5
// warps on one scheduler and get 96.
bool bucket_variant_ok(int warps, int group) {
    return (warps == 8 || warps == 11 || warps == 15 || warps == 16) && (group == 1 || group == 2);
}

template <int W, int G>
static cudaError_t bucket_smem_limit(int optin, int* dyn_max) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, bucket_count_kernel<W, G>);
    if (e != cudaSuccess) return e;
    const int lim = optin - static_cast<int>(fa.sharedSizeBytes);
    *dyn_max = *dyn_max < 0 ? lim : std::min(*dyn_max, lim);
    return cudaFuncSetAttribute(bucket_count_kernel<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

cudaError_t bucket_kernel_max_smem(int optin, int* dyn_max) {
    *dyn_max = -1;
    cudaError_t e = bucket_smem_limit<8, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<16, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<8, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<16, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<15, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<15, 2>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<11, 1>(optin, dyn_max);
    if (e == cudaSuccess) e = bucket_smem_limit<11, 2>(optin, dyn_max);
    return e;
}

cudaError_t launch_bucket_count(const ScanArgs& a, int grid, size_t smem, cudaStream_t st, int warps, int group) {
    if (warps == 8 && group == 1)
        bucket_count_kernel<8, 1><<<grid, 9 * 32, smem, st>>>(a);
    else if (warps == 16 && group == 1)
        bucket_count_kernel<16, 1><<<grid, 17 * 32, smem, st>>>(a);
    else if (warps == 8 && group == 2)
        bucket_count_kernel<8, 2><<<grid, 9 * 32, smem, st>>>(a);
    else if (warps == 16 && group == 2)
        bucket_count_kernel<16, 2><<<grid, 17 * 32, smem, st>>>(a);
    else if (warps == 15 && group == 1)
        bucket_count_kernel<15, 1><<<grid, 16 * 32, smem, st>>>(a);
    else if (warps == 15 && group == 2)
        bucket_count_kernel<15, 2><<<grid, 16 * 32, smem, st>>>(a);
    else if (warps == 11 && group == 1)
        bucket_count_kernel<11, 1><<<grid, 12 * 32, smem, st>>>(a);
    else if (warps == 11 && group == 2)
        bucket_count_kernel<11, 2><<<grid, 12 * 32, smem, st>>>(a);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace sel
