// scatter.cu -- the second pass of the two-pass selection push-down (§3.3
// "Materialization"; Algorithm 1, Execute with isSPD = true).
//
// The first pass is the COUNT scan itself (count.cu with a mask output): it
// evaluates the predicate once and leaves, for every 256-row chunk, its
// number of selected rows and, if it has some, its 32 lane bytes
// (rowmask.cuh).
//
// seg_sum_kernel           a warp per segment of kSegChunks chunks: its
//                          number of selected rows.
// seg_scan_kernel          one CTA: the output offset of each group of
//                          kGrpSegs segments (an exclusive prefix sum), and
//                          the total: the exact count.
// pushdown_scatter_kernel  one warp per segment.  Its offset is its group's
//                          plus the segments before it in the group; a warp
//                          scan of its chunk counts gives the chunk prefixes.
//                          Lane l turns the masks of chunks l and 32 + l (if
//                          they have rows) into row-order words in shared
//                          memory.  Then lane l writes the segment's selected
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

// Up to 4 projected columns from j0 on: R ranks a lane (row[k] < 0: no rank),
// every load first (the stores cannot alias them as far as the compiler
// knows), then the stores at base + the rank.
template <int R>
__device__ __forceinline__ void scatter_columns(const ScatterArgs& a, uint32_t j0, const int64_t (&row)[R], uint32_t r0,
                                                uint32_t lane, unsigned long long base) {
    unsigned long long v[4][R];
#pragma unroll
    for (uint32_t jj = 0; jj < 4; ++jj) {
        const uint32_t j = j0 + jj;
        if (j < a.n_proj) {
            const bool wide = a.width[j] == 8;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                if (row[k] >= 0)
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
                if (row[k] >= 0) {
                    if (wide) reinterpret_cast<unsigned long long*>(a.dst[j])[base + r] = v[jj][k];
                    else reinterpret_cast<uint32_t*>(a.dst[j])[base + r] = static_cast<uint32_t>(v[jj][k]);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) seg_sum_kernel(const uint16_t* __restrict__ ccnt, int64_t n_chunks,
                                                      uint32_t* __restrict__ seg_cnt, int64_t n_seg_all) {
    const uint32_t lane = threadIdx.x & 31u;
    const int64_t seg = static_cast<int64_t>(blockIdx.x) * 8 + (threadIdx.x >> 5);
    if (seg >= n_seg_all) return;
    const int64_t c0 = seg * kSegChunks + lane;
    const uint32_t v = (c0 < n_chunks ? ccnt[c0] : 0u) + (c0 + 32 < n_chunks ? ccnt[c0 + 32] : 0u);
    const uint32_t t = __reduce_add_sync(kFull, v);
    if (lane == 0) seg_cnt[seg] = t;
}

// The group sums are built in shared memory a block of kScanGroups groups at
// a time: 16 threads read a group's 64 segment counts as 16 consecutive
// 16-byte words (a warp reads 512 contiguous bytes), then the block scans them.
constexpr uint32_t kScanGroups = 4096;

__global__ void __launch_bounds__(1024) seg_scan_kernel(const uint32_t* __restrict__ seg_cnt,
                                                        unsigned long long* __restrict__ grp_off, int64_t n_grp,
                                                        unsigned long long* __restrict__ total) {
    __shared__ uint32_t s_sum[kScanGroups];
    __shared__ unsigned long long s_w[32];
    __shared__ unsigned long long s_carry;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    const uint4* q = reinterpret_cast<const uint4*>(seg_cnt);
    for (int64_t g0 = 0; g0 < n_grp; g0 += kScanGroups) {
        const uint32_t ng = static_cast<uint32_t>(n_grp - g0 < kScanGroups ? n_grp - g0 : kScanGroups);
        for (uint32_t i0 = 0; i0 < ng * (kGrpSegs / 4); i0 += 1024) {   // every lane takes part in the shuffles
            const uint32_t i = i0 + tid;
            uint32_t x = 0;
            if (i < ng * (kGrpSegs / 4)) {
                const uint4 v = q[g0 * (kGrpSegs / 4) + i];
                x = v.x + v.y + v.z + v.w;
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);   // 16 threads a group
            if ((i & 15u) == 0 && i < ng * (kGrpSegs / 4)) s_sum[i >> 4] = x;
        }
        __syncthreads();
        // each thread scans 4 consecutive groups; the block scans the threads' sums
        uint32_t v[4], tsum = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t gi = tid * 4 + k;
            v[k] = gi < ng ? s_sum[gi] : 0u;
            tsum += v[k];   // at most 4 groups of 2^20 rows
        }
        const uint32_t x = warp_incl_scan(tsum, lane);
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
        unsigned long long run = carry + (warp ? s_w[warp - 1] : 0ull) + (x - tsum);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t gi = tid * 4 + k;
            if (gi < ng) grp_off[g0 + gi] = run;
            run += v[k];
        }
        __syncthreads();
        if (tid == 0) s_carry = carry + s_w[31];
        __syncthreads();
    }
    if (tid == 0) *total = s_carry;
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
    // independent loads: the segment's count, its chunks' counts, the counts
    // of the group's segments before it and the group's offset
    const int64_t n_chunks = (a.n_rows + kChunkRows - 1) / kChunkRows;
    const uint32_t sc = a.seg_cnt[seg];
    const uint32_t clo = c_first + lane < n_chunks ? a.ccnt[c_first + lane] : 0u;
    const uint32_t chi = c_first + 32 + lane < n_chunks ? a.ccnt[c_first + 32 + lane] : 0u;
    const uint32_t b0 = lane < js ? a.seg_cnt[s0 + lane] : 0u;
    const uint32_t b1 = lane + 32u < js ? a.seg_cnt[s0 + 32 + lane] : 0u;
    const unsigned long long goff = a.grp_off[grp];
    if (sc == 0) return;   // warp-uniform; the kernel has no block-wide barrier
    const unsigned long long base = goff + __reduce_add_sync(kFull, b0 + b1);
    if (base >= a.max_rows) return;
    const uint32_t n_out = a.max_rows - base < sc ? static_cast<uint32_t>(a.max_rows - base) : sc;
    // the masks of the lane's chunks (lane, 32 + lane) as row-order words; a
    // chunk without rows is never ranked
    uint32_t* words = s_words[warp];
    uint32_t* pre = s_pre[warp];
    const bool hlo = clo != 0, hhi = chi != 0;
    uint4 x0, y0, x1, y1;
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
            row[k] = r < n_out ? seg_rank_row(pre, words, c_first, r, c) : -1;
            // a row past the table only comes from masks a failed first pass left behind
            if (row[k] >= a.n_rows) row[k] = -1;
        }
        for (uint32_t j0 = 0; j0 < a.n_proj; j0 += 4) scatter_columns<R>(a, j0, row, r0, lane, base);
        if (a.rowids) {
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const uint32_t r = r0 + 32u * k + lane;
                if (row[k] >= 0) a.rowids[base + r] = row[k];
            }
        }
    }
}

}  // namespace

cudaError_t launch_seg_sum(const uint16_t* ccnt, int64_t n_chunks, uint32_t* seg_cnt, int64_t n_grp, cudaStream_t st) {
    const int64_t n_seg_all = n_grp * kGrpSegs;
    if (n_seg_all <= 0) return cudaSuccess;
    const int64_t grid = (n_seg_all + 7) / 8;
    if (grid > 0x7FFFFFFF) return cudaErrorInvalidValue;
    seg_sum_kernel<<<static_cast<unsigned>(grid), 256, 0, st>>>(ccnt, n_chunks, seg_cnt, n_seg_all);
    return cudaGetLastError();
}

cudaError_t launch_seg_scan(const uint32_t* seg_cnt, unsigned long long* grp_off, int64_t n_grp,
                            unsigned long long* total, cudaStream_t st) {
    if (n_grp <= 0) return cudaSuccess;
    seg_scan_kernel<<<1, 1024, 0, st>>>(seg_cnt, grp_off, n_grp, total);
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
