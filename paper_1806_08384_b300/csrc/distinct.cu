// distinct.cu -- V(R, A): the number of distinct values of a column, optionally
// over the rows of a pushed-down selection only (V(sigma_P(R), A)), the input
// of the join-size estimate |R join S| = |R||S| / max(V(R,A), V(S,A)) (§1.1,
// §3.2).  With a predicate, the selected values are first compacted by the
// push-down kernel; the distinct count is then one pass of inserts into an
// open-addressing hash set in device memory.
//
// The set holds 64-bit keys (int32/date/dict codes sign-extended, int64 as
// is, float32 by bits with -0.0 folded into +0.0); all-ones marks an empty
// slot, and a value equal to it is counted through a separate flag.  A thread
// probes linearly from hash(key) & (cap - 1) with atomicCAS: a CAS that finds
// the slot empty inserts the key (one new distinct value), one that finds the
// key stops.  The capacity is a power of two of at least twice the values, so
// a probe sequence always meets an empty slot or its key; a probe count above
// the capacity (impossible by construction) sets the error flag and stops.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"

namespace sel {

namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long key_of(const uint8_t* col, int type, int64_t i) {
    if (type == 1) return static_cast<unsigned long long>(reinterpret_cast<const int64_t*>(col)[i]);
    if (type == 2) {
        uint32_t b = reinterpret_cast<const uint32_t*>(col)[i];
        if (b == 0x80000000u) b = 0u;   // -0.0 == +0.0
        return b;
    }
    return static_cast<unsigned long long>(static_cast<int64_t>(reinterpret_cast<const int32_t*>(col)[i]));
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {   // SplitMix64 output function
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

// type: 0 = 4-byte integer (int32, date, dictionary code), 1 = int64, 2 = float32.
__global__ void __launch_bounds__(256) distinct_insert_kernel(const uint8_t* col, int type, int64_t n,
                                                              unsigned long long* table, unsigned long long cap,
                                                              unsigned long long* n_new, unsigned int* flags) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        bool fresh = false;
        if (i < n) {
            const unsigned long long k = key_of(col, type, i);
            if (k == kEmpty) {
                atomicOr(flags, 2u);   // the all-ones value occurs: counted once at the end
            } else {
                unsigned long long h = mix64(k) & (cap - 1);
                for (unsigned long long probes = 0;; ++probes) {
                    if (probes > cap) {
                        atomicOr(flags, 1u);
                        break;
                    }
                    const unsigned long long prev = atomicCAS(&table[h], kEmpty, k);
                    if (prev == kEmpty) {
                        fresh = true;
                        break;
                    }
                    if (prev == k) break;
                    h = (h + 1) & (cap - 1);
                }
            }
        }
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, fresh);
        if (lane == 0 && b) atomicAdd(n_new, static_cast<unsigned long long>(__popc(b)));
    }
}

cudaError_t launch_distinct(const uint8_t* col, int type, int64_t n, unsigned long long* table, unsigned long long cap,
                            unsigned long long* n_new, unsigned int* flags, int n_sm, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks_needed = (n + 255) / 256;
    const int grid = static_cast<int>(blocks_needed < (int64_t)n_sm * 8 ? blocks_needed : (int64_t)n_sm * 8);
    distinct_insert_kernel<<<grid, 256, 0, st>>>(col, type, n, table, cap, n_new, flags);
    return cudaGetLastError();
}

}  // namespace sel

// ---------------------------------------------------------------------------
// COUNT(*) over a key join of two (selected) relations: the build side's keys
// go into an open-addressing map key -> multiplicity (same hashing, empty
// marker and -0.0 folding as above), then every key of the probe side adds
// the multiplicity of its key.  Build-side keys equal to the empty marker are
// counted apart and matched by probe keys equal to it.
// ---------------------------------------------------------------------------

namespace sel {

__global__ void __launch_bounds__(256) join_build_kernel(const uint8_t* col, int type, int64_t n,
                                                         unsigned long long* keys, unsigned long long* mult,
                                                         unsigned long long cap, unsigned long long* marker_mult,
                                                         unsigned int* flags) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long k = key_of(col, type, i);
        if (k == kEmpty) {
            atomicAdd(marker_mult, 1ull);
            continue;
        }
        unsigned long long h = mix64(k) & (cap - 1);
        for (unsigned long long probes = 0;; ++probes) {
            if (probes > cap) {
                atomicOr(flags, 1u);
                break;
            }
            const unsigned long long prev = atomicCAS(&keys[h], kEmpty, k);
            if (prev == kEmpty || prev == k) {
                atomicAdd(&mult[h], 1ull);
                break;
            }
            h = (h + 1) & (cap - 1);
        }
    }
}

__global__ void __launch_bounds__(256) join_probe_kernel(const uint8_t* col, int type, int64_t n,
                                                         const unsigned long long* keys,
                                                         const unsigned long long* mult, unsigned long long cap,
                                                         const unsigned long long* marker_mult,
                                                         unsigned long long* total, unsigned int* flags) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned long long acc = 0;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        if (i < n) {
            const unsigned long long k = key_of(col, type, i);
            if (k == kEmpty) {
                acc += *marker_mult;
            } else {
                unsigned long long h = mix64(k) & (cap - 1);
                for (unsigned long long probes = 0;; ++probes) {
                    if (probes > cap) {
                        atomicOr(flags, 1u);
                        break;
                    }
                    const unsigned long long kk = keys[h];
                    if (kk == k) {
                        acc += mult[h];
                        break;
                    }
                    if (kk == kEmpty) break;   // not on the build side
                    h = (h + 1) & (cap - 1);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0 && acc) atomicAdd(total, acc);
}

cudaError_t launch_join_count(const uint8_t* build, int64_t n_build, const uint8_t* probe, int64_t n_probe, int type,
                              unsigned long long* keys, unsigned long long* mult, unsigned long long cap,
                              unsigned long long* counters, unsigned int* flags, int n_sm, cudaStream_t st) {
    // counters[0]: the join count; counters[1]: build-side keys equal to the empty marker
    auto grid_for = [&](int64_t n) {
        const int64_t b = (n + 255) / 256;
        return static_cast<int>(b < (int64_t)n_sm * 8 ? (b > 0 ? b : 1) : (int64_t)n_sm * 8);
    };
    if (n_build > 0) {
        join_build_kernel<<<grid_for(n_build), 256, 0, st>>>(build, type, n_build, keys, mult, cap, counters + 1, flags);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_probe > 0 && n_build > 0) {
        join_probe_kernel<<<grid_for(n_probe), 256, 0, st>>>(probe, type, n_probe, keys, mult, cap, counters + 1,
                                                             counters, flags);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace sel
