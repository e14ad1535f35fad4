// lookback.cuh -- tile status words of the push-down's decoupled look-back
// (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016): one 64-bit word per tile, flag in bits 62-63 (0: not
// published, 1: aggregate of the tile, 2: inclusive prefix up to the tile),
// value below.  A word is written once per state with a relaxed store and
// read with relaxed loads; the flag and the value travel in the same word.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "scan.cuh"

namespace sel {

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Windows of 32 predecessors read per round trip.  With one tile in flight
// per CTA, the nearest inclusive prefix is usually about one CTA count (148)
// back: eight windows reach it with one round trip of independent loads.
constexpr int kLookbackWindows = 8;

// Exclusive prefix of tile t (t >= 1), computed by one warp; false if a wait
// timed out.  Lane l reads the status of tile base - 32 m - l for the
// kLookbackWindows windows m at once.  A window is resolved as soon as every
// tile from its first back to the nearest inclusive prefix has published
// (tiles further back are not waited for); with no inclusive prefix in the
// window, its 32 aggregates are summed and the walk moves to the next window.
__device__ __forceinline__ bool look_back(const PushdownArgs& a, long long t, uint32_t lane,
                                          unsigned long long* excl_out) {
    constexpr int M = kLookbackWindows;
    unsigned long long excl = 0;
    long long base = t - 1;
    // the start time and every timeout decision are the same for all lanes, so
    // the warp leaves together (a lane left behind in a ballot would wait forever)
    __syncwarp();
    const unsigned long long t0 = __shfl_sync(0xFFFFFFFFu, global_ns(), 0);
    while (true) {
        unsigned long long vw[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {   // independent loads: one round trip for all windows
            const long long idx = base - 32ll * m - static_cast<long long>(lane);
            vw[m] = (idx >= 0) ? ld_relaxed(&a.status[idx]) : kFlagInc;
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const long long idx = base - 32ll * m - static_cast<long long>(lane);
            unsigned long long v = vw[m];
            uint32_t take;   // lanes whose values are summed in this window
            bool done;
            while (true) {
                const uint32_t pub = __ballot_sync(0xFFFFFFFFu, (v >> 62) != 0);
                const uint32_t inc = __ballot_sync(0xFFFFFFFFu, (v >> 62) == 2);
                const uint32_t upto = inc ? (inc & (0u - inc)) * 2u - 1u : 0xFFFFFFFFu;   // lanes 0..nearest inclusive
                if ((pub & upto) == upto) {
                    take = upto;
                    done = inc != 0;
                    break;
                }
                const unsigned long long now = __shfl_sync(0xFFFFFFFFu, global_ns(), 0);
                if (now - t0 > a.wait_ns) {
                    *excl_out = excl;
                    return false;
                }
                __nanosleep(100);   // a predecessor is still evaluating: leave the issue slots to other warps
                if ((v >> 62) == 0) v = ld_relaxed(&a.status[idx]);
            }
            unsigned long long x = ((take >> lane) & 1u) ? (v & kValMask) : 0ull;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
            excl += x;
            if (done) {
                *excl_out = excl;
                return true;
            }
        }
        base -= 32ll * M;
    }
}

}  // namespace sel
