/*
 * nef_debug.h -- diagnostic entry points of the engine (not part of the sweep).
 */
#ifndef NEF_DEBUG_H
#define NEF_DEBUG_H

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
 * nef_tc_trace -- wait-cycle counters of the tensor-core fused pass, summed over
 * every CTA of every launch on `plan` since the last reset (plans created with
 * nef_options.profile = 2, in a library built with -DNEF_TC_TRACE=1; other builds
 * compile the counters out and leave them zero.  The counters add shared-memory
 * atomics to every tile, so timings taken with them are not representative).  out (host) receives 32 values: out[0] = summed
 * CTA lifetimes in SM cycles; out[k], k = 1..12 = cycles spent in bounded waits
 * at site k: 1 producer waits for a free Y stage, 3 MMA waits for the P tile,
 * 4 MMA waits for a Q tile, 5 MMA waits for a free yhat buffer, 6 MMA waits for
 * a W tile, 8 operand warps wait for a free Q stage, 9 epilogue waits for yhat,
 * 10 epilogue waits for Y, 11 epilogue waits for a free W buffer, 12 epilogue
 * waits for the final S, 13 operand warps wait for staged source rows, 14
 * producer waits for a free row stage; busy
 * phases: 16 operand look-ahead, 17 operand build, 18 operand fence and
 * arrival, 20 epilogue TMEM load, 21 epilogue Y read, 22 epilogue weights,
 * 23 epilogue W store, 24 epilogue fence and arrival (waits and phases of the
 * operand and epilogue warps are counted once per warp).  reset != 0 clears the counters afterwards.  Returns 0, 1 for
 * a plan without counters, 5 for a CUDA error.  Synchronises the plan's stream.
 */
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

typedef struct nef_plan_s* nef_plan_handle;
int nef_tc_trace(nef_plan_handle plan, unsigned long long* out, int reset);

#ifdef __cplusplus
}
#endif

#endif /* NEF_DEBUG_H */
