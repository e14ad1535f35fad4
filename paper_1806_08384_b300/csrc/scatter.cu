// scatter.cu -- the second pass of the two-pass selection push-down (§3.3
// "Materialization"; Algorithm 1, Execute with isSPD = true).
//
// The first pass is the COUNT scan itself (count.cu with a mask output): it
// evaluates the predicate once and leaves, for every 256-row chunk with
// selected rows, its 32 lane bytes (rowmask.cuh), and for every segment of
// kSegChunks chunks its number of selected rows and the bitmap of its chunks
// that have some.
//
// seg_scan_kernel          one CTA: the output offset of each group of
//                          kGrpSegs segments (an exclusive prefix sum).
// pushdown_scatter_kernel  one warp per segment.  Its offset is its group's
//                          plus the segments before it in the group.  Lane l
//                          reads the masks of chunks l and 32 + l (if they
//                          have rows), counts them, and turns them into
//                          row-order words in shared memory; a warp scan of
//                          the counts gives the chunk prefixes.  Then lane l writes the segment's selected
//                          rows of rank l, l + 32, ...: it finds the rank's
//                          chunk (galloping from its previous rank's chunk)
//                          and row, reads the row's projected values and
//                          stores them and the row id at the segment's offset
//                          plus the rank, so a warp's stores are contiguous.
// No wait on another CTA anywhere: the order of the output is fixed by the
// counts the first pass left.  Positions >= max_rows are not written.
#include "kernels.h"
#include "rowmask.cuh"

namespace sel {

namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kScatterWarps = 4;   // segments per CTA

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    return x;
}

// Row (in the table) of rank r among the selected rows of a segment.  pre:
// the exclusive prefixes of the segment's chunks (pre[kSegChunks] = the
// segment's count); words: their row-order masks.  c: on entry a chunk whose
// prefix is <= r (0 always is), on return r's chunk, the last one whose
// prefix is <= r (it has selected rows).  The search gallops forward from c
// and then halves: a lane's ranks increase by 32 at a time.
__device__ __forceinline__ int64_t seg_rank_row(const uint32_t* pre, const uint32_t* words, int64_t c_first,
                                                uint32_t r, uint32_t& c) {
    uint32_t step = 1u;
    while (c + step < kSegChunks && pre[c + step] <= r) {
        c += step;
        step <<= 1;
    }
    uint32_t hi = c + step < kSegChunks ? c + step : kSegChunks;   // pre[hi] > r
    while (hi - c > 1u) {
        const uint32_t mid = (c + hi) >> 1;
        if (pre[mid] <= r) c = mid;
        else hi = mid;
    }
    uint32_t o = r - pre[c];
    const uint32_t* w = words + c * 8u;
    uint32_t k = 0, wd = w[0], pc = __popc(wd);
    while (o >= pc && k < 7u) {   // o < the chunk's count: at most 7 steps
        o -= pc;
        wd = w[++k];
        pc = __popc(wd);
    }
    return (c_first + c) * kChunkRows + 32 * k + select_bit(wd, o);
}

// Up to 4 projected columns from j0 on: R ranks a lane, every load first
// (the stores cannot alias them as far as the compiler knows), then the stores.
template <int R>
__device__ __forceinline__ void scatter_columns(const ScatterArgs& a, uint32_t j0, const int64_t (&row)[R], uint32_t r0,
                                                uint32_t n_out, uint32_t lane, unsigned long long base) {
    unsigned long long v[4][R];
#pragma unroll
    for (uint32_t jj = 0; jj < 4; ++jj) {
        const uint32_t j = j0 + jj;
        if (j < a.n_proj) {
            const bool wide = a.width[j] == 8;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (r0 + 32u * k + lane < n_out)
                    v[jj][k] = wide ? __ldg(reinterpret_cast<const unsigned long long*>(a.src[j]) + row[k])
                                    : __ldg(reinterpret_cast<const uint32_t*>(a.src[j]) + row[k]);
            }
        }
    }
#pragma unroll
    for (uint32_t jj = 0; jj < 4; ++jj) {
        const uint32_t j = j0 + jj;
        if (j < a.n_proj) {
            const bool wide = a.width[j] == 8;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const uint32_t r = r0 + 32u * k + lane;
                if (r < n_out) {
                    if (wide) reinterpret_cast<unsigned long long*>(a.dst[j])[base + r] = v[jj][k];
                    else reinterpret_cast<uint32_t*>(a.dst[j])[base + r] = static_cast<uint32_t>(v[jj][k]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(1024) seg_scan_kernel(const uint32_t* __restrict__ seg_cnt,
                                                        unsigned long long* __restrict__ grp_off, int64_t n_grp) {
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int64_t g0 = 0; g0 < n_grp; g0 += 1024) {
        const int64_t g = g0 + tid;
        uint32_t v = 0;   // at most kGrpSegs * kSegChunks * 256 = 2^20 rows
        if (g < n_grp) {
            const uint4* p = reinterpret_cast<const uint4*>(seg_cnt + g * kGrpSegs);
            uint4 q[kGrpSegs / 4];
#pragma unroll
            for (uint32_t i = 0; i < kGrpSegs / 4; ++i) q[i] = p[i];
#pragma unroll
            for (uint32_t i = 0; i < kGrpSegs / 4; ++i) v += q[i].x + q[i].y + q[i].z + q[i].w;
        }
        const uint32_t x = warp_incl_scan(v, lane);
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(kFull, w, o);
                if (lane >= static_cast<uint32_t>(o)) w += y;
            }
            s_w[lane] = w;
        }
        __syncthreads();
        const unsigned long long carry = s_carry;
        if (g < n_grp) grp_off[g] = carry + (warp ? s_w[warp - 1] : 0ull) + (x - v);
        __syncthreads();
        if (tid == 0) s_carry = carry + s_w[31];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScatterWarps * 32, 8) pushdown_scatter_kernel(const __grid_constant__ ScatterArgs a) {
    __shared__ __align__(16) uint32_t s_words[kScatterWarps][kSegChunks * 8];
    __shared__ uint32_t s_pre[kScatterWarps][kSegChunks + 1];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const int64_t seg = static_cast<int64_t>(blockIdx.x) * kScatterWarps + warp;
    if (seg >= a.n_seg) return;
    const int64_t grp = seg / kGrpSegs, s0 = grp * kGrpSegs;
    const uint32_t js = static_cast<uint32_t>(seg - s0);
    const int64_t c_first = seg * kSegChunks;
    // independent loads: the segment's count and chunk bitmap, the counts of
    // the group's segments before it and the group's offset
    const uint32_t sc = a.seg_cnt[seg];
    const unsigned long long nz = a.seg_nz[seg];
    const uint32_t b0 = lane < js ? a.seg_cnt[s0 + lane] : 0u;
    const uint32_t b1 = lane + 32u < js ? a.seg_cnt[s0 + 32 + lane] : 0u;
    const unsigned long long goff = a.grp_off[grp];
    if (sc == 0) return;   // warp-uniform; the kernel has no block-wide barrier
    const unsigned long long base = goff + __reduce_add_sync(kFull, b0 + b1);
    if (base >= a.max_rows) return;
    const uint32_t n_out = a.max_rows - base < sc ? static_cast<uint32_t>(a.max_rows - base) : sc;
    // the masks of the lane's chunks (lane, 32 + lane), their counts, and
    // their row-order words; a chunk without rows has no mask and is never ranked
    uint32_t* words = s_words[warp];
    uint32_t* pre = s_pre[warp];
    const bool hlo = (nz >> lane) & 1ull, hhi = (nz >> (32u + lane)) & 1ull;
    uint4 x0 = make_uint4(0, 0, 0, 0), y0 = x0, x1 = x0, y1 = x0;
    if (hlo) {
        const uint4* mp = reinterpret_cast<const uint4*>(a.mask + (c_first + lane) * 32);
        x0 = mp[0];
        y0 = mp[1];
    }
    if (hhi) {
        const uint4* mp = reinterpret_cast<const uint4*>(a.mask + (c_first + 32 + lane) * 32);
        x1 = mp[0];
        y1 = mp[1];
    }
    const uint32_t clo = __popc(x0.x) + __popc(x0.y) + __popc(x0.z) + __popc(x0.w) + __popc(y0.x) + __popc(y0.y) +
                         __popc(y0.z) + __popc(y0.w);
    const uint32_t chi = __popc(x1.x) + __popc(x1.y) + __popc(x1.z) + __popc(x1.w) + __popc(y1.x) + __popc(y1.y) +
                         __popc(y1.z) + __popc(y1.w);
    const uint32_t xlo = warp_incl_scan(clo, lane);
    const uint32_t tlo = __shfl_sync(kFull, xlo, 31);
    pre[lane] = xlo - clo;
    pre[32 + lane] = tlo + warp_incl_scan(chi, lane) - chi;
    if (lane == 0) pre[kSegChunks] = sc;
    if (hlo) lane_bytes_to_rows(reinterpret_cast<uint4*>(words + lane * 8u), x0, y0);
    if (hhi) lane_bytes_to_rows(reinterpret_cast<uint4*>(words + (32u + lane) * 8u), x1, y1);
    __syncwarp();
    constexpr int R = 4;   // ranks a lane has in flight
    uint32_t c = 0;
    for (uint32_t r0 = 0; r0 < n_out; r0 += 32u * R) {
        int64_t row[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t r = r0 + 32u * k + lane;
            row[k] = r < n_out ? seg_rank_row(pre, words, c_first, r, c) : 0;
        }
        for (uint32_t j0 = 0; j0 < a.n_proj; j0 += 4) scatter_columns<R>(a, j0, row, r0, n_out, lane, base);
        if (a.rowids) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const uint32_t r = r0 + 32u * k + lane;
                if (r < n_out) a.rowids[base + r] = row[k];
            }
        }
    }
}

}  // namespace

cudaError_t launch_seg_scan(const uint32_t* seg_cnt, unsigned long long* grp_off, int64_t n_grp, cudaStream_t st) {
    if (n_grp <= 0) return cudaSuccess;
    seg_scan_kernel<<<1, 1024, 0, st>>>(seg_cnt, grp_off, n_grp);
    return cudaGetLastError();
}

cudaError_t launch_pushdown_scatter(const ScatterArgs& a, cudaStream_t st) {
    if (a.n_seg <= 0) return cudaSuccess;
    for (uint32_t j = 0; j < a.n_proj; ++j)
        if (a.width[j] != 4 && a.width[j] != 8) return cudaErrorInvalidValue;
    const int64_t grid = (a.n_seg + kScatterWarps - 1) / kScatterWarps;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    pushdown_scatter_kernel<<<static_cast<unsigned>(grid), kScatterWarps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace sel
