// gemm_probe.cu -- the fold-in encoder's tensor-core GEMM on its own (test-only
// entry point; the kernel is the product's, compiled from csrc/k_gemm_tc.cu into
// this probe library).
#include "nef_internal.h"
#include "nef_probe.h"

extern "C" int nef_tc_gemm(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int M,
                           int N, int K, int* err, void* stream) {
    const cudaError_t e =
        nef::launch_gemm_nt(A, lda, B, ldb, C, ldc, M, N, K, 0, err, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? 0 : 5;
}

extern "C" int nef_tc_gemm_split(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                                 int M, int N, int K, int n_split, float* ws, int64_t ws_floats, int* err,
                                 void* stream) {
    const cudaError_t e = nef::launch_gemm_nt(A, lda, B, ldb, C, ldc, M, N, K, 0, err,
                                              static_cast<cudaStream_t>(stream), ws, ws_floats, n_split);
    return e == cudaSuccess ? 0 : 5;
}
