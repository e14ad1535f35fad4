// gemm_api.cpp -- C entry point of the tcgen05 GEMM for tests (include/sel.h).
#include "gemm.h"
#include "internal.h"

using namespace sel;

extern "C" sel_status sel_debug_gemm_bf16(void* cuda_stream, const void* A, const void* B, int32_t M, int32_t N,
                                          int32_t K, float* C, int32_t k_splits, uint32_t* dev_err) {
    if (!A || !B || !C || !dev_err || M <= 0 || N <= 0 || K <= 0 || K % 8 || k_splits < 1 || k_splits > 64 ||
        reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(B) % 16) {
        set_error("sel_debug_gemm_bf16: bad arguments");
        return SEL_ERR_INVALID_ARG;
    }
    GemmArgs g{};
    g.A = static_cast<const __nv_bfloat16*>(A);
    g.B = static_cast<const __nv_bfloat16*>(B);
    g.lda = K;
    g.ldb = K;
    g.M = M;
    g.N = N;
    g.K = K;
    g.epi = EPI_F32;
    g.C = C;
    g.ldc = N;
    g.err = reinterpret_cast<unsigned int*>(dev_err);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSuccess;
    if (k_splits > 1) e = cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(float), st);
    if (e == cudaSuccess) e = launch_gemm(g, k_splits, st);
    if (e != cudaSuccess) {
        set_error("sel_debug_gemm_bf16: %s", cudaGetErrorString(e));
        return SEL_ERR_CUDA;
    }
    return SEL_OK;
}
