// k_view_tc_persist.cu -- the persistent batched fit: one launch of one CTA per SM
// for every sweep of every (problem, restart) unit (k_batched_persistent).
#include <algorithm>

#include "k_view_tc.cuh"
#include "nef_batched.h"

namespace nef {

cudaError_t launch_batched_persistent(const PersistDesc& d, const WeightSpec& w, int n_sm, cudaStream_t st) {
    if (d.n_items <= 0 || d.n_sweeps <= 0) return cudaSuccess;
    const bool kl = w.lik == LIK_NONE && !w.log_case && w.y_code == POW_ID && w.a_code == POW_RCP &&
                    w.b_code == POW_ONE;
    if (d.bp != 16 && d.bp != 32) return cudaErrorInvalidValue;
    auto kern = d.bp == 16 ? (kl ? tc::k_batched_persistent<16, tc::WK_KL> : tc::k_batched_persistent<16, tc::WK_GEN>)
                           : (kl ? tc::k_batched_persistent<32, tc::WK_KL> : tc::k_batched_persistent<32, tc::WK_GEN>);
    const int smem = d.bp == 16 ? tc::Layout<16, true>::kAlloc : tc::Layout<32, true>::kAlloc;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // One CTA per SM.  No CTA waits for an item that no running CTA holds: a stage's
    // items precede (in queue order) every item that waits for the stage, and they
    // were taken by CTAs that are running, so the launch makes progress whether or
    // not all CTAs are resident at once.
    kern<<<std::max(1, n_sm), tc::kThreads, smem, st>>>(d);
    return cudaGetLastError();
}

}  // namespace nef
