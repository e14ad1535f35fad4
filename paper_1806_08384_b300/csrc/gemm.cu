// gemm.cu -- BF16 x BF16 -> FP32 matrix product on the 5th-generation tensor
// cores (tcgen05.mma, accumulator in TMEM), with the fused epilogues the
// learned estimator's forward and backward passes need:
//   C[M x N] = A[M x K] * B[N x K]^T      (A and B row-major, K contiguous)
// One CTA (4 warps) computes a 128 x 256 tile.  K is walked in 64-column
// blocks: all 128 threads copy the next A and B blocks into the other of two
// shared-memory stages (16-byte cp.async into the 128-byte-swizzled K-major
// layout, zero-filled past M, N or K) while thread 0 has the tensor core
// multiply the current stage (4 MMAs of K = 16) and commits their completion
// to that stage's mbarrier.  The epilogue reads the tile back from TMEM, one
// row per thread, 32 columns at a time.  Split-K (gridDim.z > 1) adds partial
// tiles with FP32 atomics.
#include <cuda_bf16.h>

#include "gemm.h"
#include "tc.cuh"

namespace sel {

namespace {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr uint32_t kStageA = BM * BK * 2;   // 16 KiB
constexpr uint32_t kStageB = BN * BK * 2;   // 32 KiB
constexpr uint32_t kStage = kStageA + kStageB;

__device__ __forceinline__ void load_stage(const GemmArgs& g, uint32_t sA, uint32_t sB, int m0, int n0, int k0,
                                           uint32_t tid) {
    // A: 128 rows x 8 chunks; B: 256 rows x 8 chunks of 16 bytes
    for (uint32_t i = tid; i < BM * 8; i += 128) {
        const uint32_t r = i >> 3, c = i & 7u;
        const int row = m0 + (int)r, col = k0 + (int)c * 8;
        const bool ok = row < g.M && col < g.K;
        const __nv_bfloat16* src = ok ? g.A + (size_t)row * g.lda + col : g.A;
        cp_async16(sA + sw128_offset(r, c), src, ok ? 16u : 0u);
    }
    for (uint32_t i = tid; i < BN * 8; i += 128) {
        const uint32_t r = i >> 3, c = i & 7u;
        const int row = n0 + (int)r, col = k0 + (int)c * 8;
        const bool ok = row < g.N && col < g.K;
        const __nv_bfloat16* src = ok ? g.B + (size_t)row * g.ldb + col : g.B;
        cp_async16(sB + sw128_offset(r, c), src, ok ? 16u : 0u);
    }
    cp_async_commit();
}

}  // namespace

__global__ void __launch_bounds__(128) tc_gemm_kernel(const __grid_constant__ GemmArgs g) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ uint64_t mma_done[2];
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_fail;
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    // stage s: A tile at base + s * kStage, B tile kStageA bytes after it
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int nkb_total = (g.K + BK - 1) / BK;
    const int per = (nkb_total + (int)gridDim.z - 1) / (int)gridDim.z;
    const int kb0 = (int)blockIdx.z * per;
    const int kb1 = min(nkb_total, kb0 + per);
    const int nkb = kb1 - kb0;

    if (warp == 0) tc_alloc(&tmem_base, 256);
    if (tid == 0) {
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(BM, BN);

    if (nkb > 0) {
        load_stage(g, base, base + kStageA, m0, n0, kb0 * BK, tid);
        for (int i = 0; i < nkb; ++i) {
            const int s = i & 1;
            if (i + 1 < nkb) {
                if (i >= 1) {   // the MMAs of iteration i-1 read the other stage
                    const bool ok = mbar_wait_bounded(&mma_done[s ^ 1], static_cast<uint32_t>(((i - 1) >> 1) & 1));
                    if (!ok) atomicOr(&s_fail, 1u);
                }
                load_stage(g, base + (s ^ 1) * kStage, base + (s ^ 1) * kStage + kStageA, m0, n0, (kb0 + i + 1) * BK, tid);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            fence_proxy_async();   // make the copied tiles visible to the tensor core
            __syncthreads();
            if (s_fail) break;
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc_mma(tmem, sw128_desc(base + s * kStage + 32u * kk),
                           sw128_desc(base + s * kStage + kStageA + 32u * kk), idesc,
                           (i > 0 || kk > 0) ? 1u : 0u);
                tc_commit(&mma_done[s]);
            }
        }
        // all MMAs of this thread are complete when the last commit arrives
        const int last = nkb - 1;
        if (!mbar_wait_bounded(&mma_done[last & 1], static_cast<uint32_t>((last >> 1) & 1))) atomicOr(&s_fail, 1u);
    }
    __syncthreads();
    tc_fence_after();
    if (s_fail) {
        if (tid == 0) atomicOr(g.err, 1u);
    } else {
        // Each warp owns 32 accumulator rows; 32 columns at a time go through a
        // padded shared tile so that global stores run along rows (coalesced)
        // and column sums are one add per lane.  The stage buffers are free:
        // every MMA has completed.
        float* tile = reinterpret_cast<float*>(smem_raw + (base - smem_u32(smem_raw))) + warp * (32 * 33);
        const int rbase = m0 + (int)(warp * 32);
        const int row = rbase + (int)lane;
        const bool row_ok = row < g.M;
#pragma unroll 1
        for (int cc = 0; cc < BN / 32; ++cc) {
            float f[32];
            if (nkb > 0) {
                tc_ld32(tmem + ((warp * 32u) << 16) + (uint32_t)cc * 32u, f);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) f[j] = 0.f;
            }
            const int c0 = n0 + cc * 32;
            const int col = c0 + (int)lane;   // this lane's column in the row-wise phase
            if (g.epi == EPI_DRELU) {   // the 32 x 32 mask block, read along rows, into the tile
                for (int r = 0; r < 32; ++r)
                    tile[r * 33 + lane] = (rbase + r < g.M && col < g.N)
                        ? __bfloat162float(g.mask[(size_t)(rbase + r) * g.ldm + col]) : 0.f;
                __syncwarp();
            }
            if (g.epi != EPI_F32) {
                // EPI_BIAS_RELU: relu(acc + bias); EPI_DRELU: acc where mask > 0
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int cj = c0 + j;
                    float v = f[j];
                    if (g.epi == EPI_BIAS_RELU) v = fmaxf(v + (cj < g.N ? g.bias[cj] : 0.f), 0.f);
                    else v = tile[lane * 33 + j] > 0.f ? v : 0.f;
                    if (!row_ok) v = 0.f;
                    f[j] = v;
                }
                __syncwarp();
                if (row_ok && g.outT)   // lanes write consecutive rows of the transposed matrix: coalesced
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < g.N) g.outT[(size_t)(c0 + j) * g.ldoT + row] = __float2bfloat16_rn(f[j]);
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = f[j];
            __syncwarp();
            // row-wise phase: lane = column
            if (g.epi == EPI_F32) {
                if (col < g.N)
                    for (int r = 0; r < 32 && rbase + r < g.M; ++r) {
                        float* dst = g.C + (size_t)(rbase + r) * g.ldc + col;
                        if (gridDim.z > 1) atomicAdd(dst, tile[r * 33 + lane]);
                        else *dst = tile[r * 33 + lane];
                    }
            } else {
                if (g.out && col < g.N)
                    for (int r = 0; r < 32 && rbase + r < g.M; ++r)
                        g.out[(size_t)(rbase + r) * g.ldo + col] = __float2bfloat16_rn(tile[r * 33 + lane]);
                if (g.epi == EPI_DRELU && g.colsum && col < g.N) {
                    float sum = 0.f;
#pragma unroll 8
                    for (int r = 0; r < 32; ++r) sum += tile[r * 33 + lane];   // rows past M hold 0
                    atomicAdd(&g.colsum[col], sum);
                }
            }
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// The estimator's inference pass fused into one kernel (a7).  One CTA of 4
// warps owns 128 rows.  Their activations stay in one 64 KiB shared buffer H
// (4 K blocks of 128 rows x 64 bf16 in the swizzled layout the MMA reads),
// which is the A operand of every layer: the features are copied into it
// first (144 columns, zero-filled to 192), and each layer's epilogue writes
// relu(acc + b) back over it once that layer's MMAs have completed.  The
// weights stream through two 32 KiB stages, one 64-column K block of all 256
// rows at a time, the next block loading while the tensor core multiplies
// the current one.  The accumulator (128 x 256 FP32) lives in TMEM; thread t
// reads row t's columns back.  After the third layer each thread finishes
// its row's two outputs with the 256 -> 2 head in FP32, in the same order
// and roundings as the layer-by-layer path.
namespace {

constexpr int kMlpIn = 144, kMlpHid = 256;
constexpr uint32_t kHBlock = BM * BK * 2;           // 16 KiB: one K block of H
constexpr uint32_t kHBytes = 4 * kHBlock;           // 64 KiB
constexpr uint32_t kWStage = kMlpHid * BK * 2;      // 32 KiB: one K block of a weight matrix

__device__ __forceinline__ void mlp_load_x(const MlpFwdArgs& a, uint32_t H, int m0, uint32_t tid) {
    for (uint32_t kb = 0; kb < 3; ++kb)
        for (uint32_t i = tid; i < BM * 8; i += 128) {
            const uint32_t r = i >> 3, c = i & 7u;
            const int row = m0 + (int)r, col = (int)(kb * BK + c * 8);
            const bool ok = row < a.n && col < kMlpIn;
            const __nv_bfloat16* src = ok ? a.x + (size_t)row * kMlpIn + col : a.x;
            cp_async16(H + kb * kHBlock + sw128_offset(r, c), src, ok ? 16u : 0u);
        }
}

// K block k0 .. k0 + 63 of W (256 rows, row stride and width K) into a stage; commits.
__device__ __forceinline__ void mlp_load_w(const __nv_bfloat16* W, int K, uint32_t dst, int k0, uint32_t tid) {
    for (uint32_t i = tid; i < kMlpHid * 8; i += 128) {
        const uint32_t r = i >> 3, c = i & 7u;
        const int col = k0 + (int)c * 8;
        const bool ok = col < K;
        const __nv_bfloat16* src = ok ? W + (size_t)r * K + col : W;
        cp_async16(dst + sw128_offset(r, c), src, ok ? 16u : 0u);
    }
    cp_async_commit();
}

}  // namespace

__global__ void __launch_bounds__(128) mlp_forward_kernel(const __grid_constant__ MlpFwdArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ uint64_t mma_done[2];
    __shared__ uint32_t tmem_base;
    __shared__ uint32_t s_fail;
    __shared__ float s_b[3][kMlpHid];
    __shared__ float s_w4[2][kMlpHid];
    const uint32_t tid = threadIdx.x, warp = tid >> 5;
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t* const hgen = smem_raw + (base - smem_u32(smem_raw));   // H through a generic pointer
    const uint32_t H = base, S0 = base + kHBytes;                    // stage s at S0 + s * kWStage
    const int m0 = blockIdx.x * BM;

    if (warp == 0) tc_alloc(&tmem_base, 256);
    if (tid == 0) {
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        fence_mbar_init();
        s_fail = 0;
    }
    for (uint32_t k = tid; k < (uint32_t)kMlpHid; k += 128) {
        s_b[0][k] = a.b[0][k];
        s_b[1][k] = a.b[1][k];
        s_b[2][k] = a.b[2][k];
        s_w4[0][k] = __bfloat162float(a.w4[k]);
        s_w4[1][k] = __bfloat162float(a.w4[kMlpHid + k]);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(BM, kMlpHid);

    mlp_load_x(a, H, m0, tid);                    // joins the commit group of W1's first K block
    mlp_load_w(a.w[0], kMlpIn, S0, 0, tid);
    uint32_t it = 0;   // K blocks multiplied so far: block `it` uses stage it & 1 and commits phase (it >> 1) & 1
    float o0 = 0.f, o1 = 0.f;
    for (int L = 0; L < 3; ++L) {
        const int K = L == 0 ? kMlpIn : kMlpHid;
        const int nkb = L == 0 ? 3 : 4;
        const __nv_bfloat16* W = a.w[L];
        // the first K block's stage was last read two blocks ago, before the last layer's epilogue
        if (L > 0) mlp_load_w(W, K, S0 + (it & 1u) * kWStage, 0, tid);
        for (int kb = 0; kb < nkb; ++kb) {
            const uint32_t i = it + (uint32_t)kb, s = i & 1u;
            if (kb + 1 < nkb) {
                if (kb >= 1) {   // the other stage was read by block i - 1 of this layer
                    const bool ok = mbar_wait_bounded(&mma_done[s ^ 1u], ((i - 1u) >> 1) & 1u);
                    if (!ok) atomicOr(&s_fail, 1u);
                }
                mlp_load_w(W, K, S0 + (s ^ 1u) * kWStage, (kb + 1) * BK, tid);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            fence_proxy_async();   // the copied tiles (and H) visible to the tensor core
            __syncthreads();
            if (s_fail) break;
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    tc_mma(tmem, sw128_desc(H + (uint32_t)kb * kHBlock + 32u * kk),
                           sw128_desc(S0 + s * kWStage + 32u * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                tc_commit(&mma_done[s]);
            }
        }
        if (s_fail) break;
        const uint32_t last = it + (uint32_t)nkb - 1u;
        if (!mbar_wait_bounded(&mma_done[last & 1u], (last >> 1) & 1u)) atomicOr(&s_fail, 1u);
        it += (uint32_t)nkb;
        __syncthreads();
        if (s_fail) break;
        tc_fence_after();
        // epilogue: row tid of the tile, 32 columns at a time
#pragma unroll 1
        for (int cc = 0; cc < kMlpHid / 32; ++cc) {
            float f[32];
            tc_ld32(tmem + ((warp * 32u) << 16) + (uint32_t)cc * 32u, f);
#pragma unroll
            for (int j = 0; j < 32; ++j) f[j] = fmaxf(f[j] + s_b[L][cc * 32 + j], 0.f);
            if (L < 2) {   // the next layer's input, over this layer's (all its MMAs have completed)
                uint8_t* hb = hgen + (uint32_t)(cc >> 1) * kHBlock;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t w[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(f[8 * q + 2 * e], f[8 * q + 2 * e + 1]);
                        w[e] = *reinterpret_cast<const uint32_t*>(&h2);
                    }
                    *reinterpret_cast<uint4*>(hb + sw128_offset(tid, (uint32_t)((cc & 1) * 4 + q))) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            } else {       // the head, on the BF16-rounded activations
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float h = __bfloat162float(__float2bfloat16_rn(f[j]));
                    o0 = fmaf(h, s_w4[0][cc * 32 + j], o0);
                    o1 = fmaf(h, s_w4[1][cc * 32 + j], o1);
                }
            }
        }
        tc_fence_before();
        fence_proxy_async();   // H's new contents visible to the next layer's MMAs
        __syncthreads();
        tc_fence_after();
    }
    cp_async_wait<0>();   // nothing of ours lands after the exit (a failed wait can leave copies in flight)
    if (s_fail) {
        if (tid == 0) atomicOr(a.err, 1u);
    } else {
        const int row = m0 + (int)tid;
        if (row < a.n) {
            a.out[2 * (size_t)row] = o0 + a.b4[0];
            a.out[2 * (size_t)row + 1] = o1 + a.b4[1];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, 256);
}

size_t mlp_forward_smem_bytes() { return (size_t)kHBytes + 2 * (size_t)kWStage + 1024; }

cudaError_t launch_mlp_forward(const MlpFwdArgs& a, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)mlp_forward_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (a.n <= 0) return cudaSuccess;
    mlp_forward_kernel<<<(a.n + BM - 1) / BM, 128, mlp_forward_smem_bytes(), st>>>(a);
    return cudaGetLastError();
}

size_t gemm_smem_bytes() { return 2 * (size_t)kStage + 1024; }

cudaError_t launch_gemm(const GemmArgs& g, int k_splits, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gemm_smem_bytes());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, k_splits < 1 ? 1 : k_splits);
    tc_gemm_kernel<<<grid, 128, gemm_smem_bytes(), st>>>(g);
    return cudaGetLastError();
}

}  // namespace sel
