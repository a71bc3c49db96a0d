/*
 * nef_probe.h -- test-only probes of the tensor-core building blocks (built into
 * tests/tc_probe/_build/libnef_probe.so, not into the product library).
 */
#ifndef NEF_PROBE_H
#define NEF_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * nef_tc_probe -- run the two tensor-core products of the fused pass once on
 * caller-given BF16 tiles, with exactly the shared-memory layouts, descriptors
 * and instruction descriptors the pass uses (Eq. 2.1 tile product and the
 * Eq. 3.6-3.8 contraction):
 *   D1[128 x 64]  = P[128 x bp] . Q[64 x bp]^T
 *   D2[128 x bp]  = W[128 x 64] . Q[64 x bp]
 * with the A operands P and W in shared memory (a_in_tmem = 0) or in tensor
 * memory (a_in_tmem != 0).
 * All pointers are device pointers to row-major arrays; BF16 values are raw
 * 16-bit patterns.  bond_pad is 16, 32 or 64.  err (device int) receives a
 * nonzero code if the bounded completion wait gave up.  Enqueued on `stream`
 * (a cudaStream_t).  Returns 0 on a successful launch, 1 for a bad bond_pad,
 * 5 for a CUDA error.
 */
int nef_tc_probe(int bond_pad, int a_in_tmem, const uint16_t* P, const uint16_t* Q, const uint16_t* W,
                 float* D1, float* D2, int* err, void* stream);

/*
 * nef_tc_gemm -- the tensor-core GEMM of the fold-in encoder on its own:
 * C[M x N] = A[M x K] . B[N x K]^T.  A, B: device row-major BF16 (raw 16-bit
 * patterns) with row pitches lda, ldb (elements, multiples of 8) and 16-byte
 * aligned bases; C: device row-major FP32, pitch ldc.  err (device int)
 * receives a nonzero code if a bounded wait gave up.  Enqueued on `stream`.
 * Returns 0 on a successful launch, 5 for a CUDA error (including bad pitches).
 */
int nef_tc_gemm(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int M, int N,
                int K, int* err, void* stream);

/*
 * nef_tc_gemm_split -- the same product with K split over n_split CTAs per tile,
 * their partial tiles in ws (device, ws_floats FP32 values, at least
 * n_split * M * ldc) summed in split order.  Returns as nef_tc_gemm.
 */
int nef_tc_gemm_split(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int M,
                      int N, int K, int n_split, float* ws, int64_t ws_floats, int* err, void* stream);


#ifdef __cplusplus
}
#endif

#endif /* NEF_PROBE_H */
