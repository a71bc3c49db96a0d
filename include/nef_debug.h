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
 * All pointers are device pointers to row-major arrays; BF16 values are raw
 * 16-bit patterns.  bond_pad is 16, 32 or 64.  err (device int) receives a
 * nonzero code if the bounded completion wait gave up.  Enqueued on `stream`
 * (a cudaStream_t).  Returns 0 on a successful launch, 1 for a bad bond_pad,
 * 5 for a CUDA error.
 */
int nef_tc_probe(int bond_pad, const uint16_t* P, const uint16_t* Q, const uint16_t* W, float* D1,
                 float* D2, int* err, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NEF_DEBUG_H */
