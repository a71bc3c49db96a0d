// k_view_tc_inst.cuh -- instantiation helper: one translation unit per bond width.
#pragma once
#include "k_view_tc.cuh"

namespace nef {
namespace tc {

template <int BP, bool DEN, int WK, bool LOSS, int QM, int CFG = 0>
cudaError_t launch_one(const CUtensorMap& map, const CUtensorMap& vmap, const CUtensorMap& cmap, const Params& p, int grid,
                       cudaStream_t st) {
    auto kern = k_view_tc<BP, DEN, WK, LOSS, QM, CFG>;
    const int sm = Layout<BP, DEN, CFG>::kAlloc;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    launch_pdl(kern, grid, kThreads, sm, st, map, vmap, cmap, p);
    return cudaGetLastError();
}

template <int BP, bool LOSS, int QM, int CFG = 0>
cudaError_t launch_bp(const CUtensorMap& map, const CUtensorMap& vmap, const CUtensorMap& cmap, const Params& p, int den,
                      int wk, int grid, cudaStream_t st) {
    if (den) {
        switch (wk) {
            case WK_KL: return launch_one<BP, true, WK_KL, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
            case WK_B05: return launch_one<BP, true, WK_B05, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
            case WK_HEL: return launch_one<BP, true, WK_HEL, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
            default: return launch_one<BP, true, WK_GEN, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
        }
    }
    switch (wk) {
        case WK_KL: return launch_one<BP, false, WK_KL, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
        case WK_HEL: return launch_one<BP, false, WK_HEL, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
        default: return launch_one<BP, false, WK_GEN, LOSS, QM, CFG>(map, vmap, cmap, p, grid, st);
    }
}

// The weight kinds of the other loss families: reverse KL (0,1) and the
// likelihood families (negative binomial and binomial always contract the
// denominator; Jensen-Shannon and reverse KL have b == 1 and take the closed form
// when there is no mask).
template <int BP, bool LOSS, int QM>
cudaError_t launch_bp_lik(const CUtensorMap& map, const CUtensorMap& vmap, const CUtensorMap& cmap, const Params& p,
                          int den, int wk, int grid, cudaStream_t st) {
    if (!den) {
        switch (wk) {
            case WK_JS: return launch_one<BP, false, WK_JS, LOSS, QM>(map, vmap, cmap, p, grid, st);
            case WK_RKL: return launch_one<BP, false, WK_RKL, LOSS, QM>(map, vmap, cmap, p, grid, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (wk) {
        case WK_NB: return launch_one<BP, true, WK_NB, LOSS, QM>(map, vmap, cmap, p, grid, st);
        case WK_BIN: return launch_one<BP, true, WK_BIN, LOSS, QM>(map, vmap, cmap, p, grid, st);
        case WK_JS: return launch_one<BP, true, WK_JS, LOSS, QM>(map, vmap, cmap, p, grid, st);
        case WK_RKL: return launch_one<BP, true, WK_RKL, LOSS, QM>(map, vmap, cmap, p, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
}  // namespace nef

// SUFFIX names the instance set: plain or loss-summing (LOSS), with the Q operand
// built from TMA-staged rows (QM 1) or gathered rows (QM 0, suffix _g)
#define NEF_TC_INSTANCE_X(BP, SUFFIX, LOSS, QM)                                               \
    namespace nef {                                                                          \
    namespace tc {                                                                           \
    cudaError_t launch_bp##BP##SUFFIX(const CUtensorMap& map, const CUtensorMap& vmap,        \
                                      const CUtensorMap& cmap, const Params& p, int den, int wk, \
                                      int grid, cudaStream_t st) {                           \
        return launch_bp<BP, LOSS, QM>(map, vmap, cmap, p, den, wk, grid, st);               \
    }                                                                                        \
    }                                                                                        \
    }
#define NEF_TC_LIK_INSTANCE_X(BP, SUFFIX, LOSS)                                               \
    namespace nef {                                                                          \
    namespace tc {                                                                           \
    cudaError_t launch_bp##BP##SUFFIX(const CUtensorMap& map, const CUtensorMap& vmap,        \
                                      const CUtensorMap& cmap, const Params& p, int den, int wk, \
                                      int grid, cudaStream_t st) {                           \
        return launch_bp_lik<BP, LOSS, 1>(map, vmap, cmap, p, den, wk, grid, st);            \
    }                                                                                        \
    }                                                                                        \
    }
#define NEF_TC_LIK_INSTANCE(BP) NEF_TC_LIK_INSTANCE_X(BP, _lik, false)
#define NEF_TC_LIK_LOSS_INSTANCE(BP) NEF_TC_LIK_INSTANCE_X(BP, _lik_loss, true)
#define NEF_TC_RING1_INSTANCE(BP)                                                            \
    namespace nef {                                                                          \
    namespace tc {                                                                           \
    cudaError_t launch_bp##BP##_r1(const CUtensorMap& map, const CUtensorMap& vmap,           \
                                   const CUtensorMap& cmap, const Params& p, int den, int wk, \
                                   int grid, cudaStream_t st) {                              \
        return launch_bp<BP, false, 1, 1>(map, vmap, cmap, p, den, wk, grid, st);            \
    }                                                                                        \
    }                                                                                        \
    }
#define NEF_TC_INSTANCE(BP) NEF_TC_INSTANCE_X(BP, , false, 1)
#define NEF_TC_LOSS_INSTANCE(BP) NEF_TC_INSTANCE_X(BP, _loss, true, 1)
#define NEF_TC_GATHER_INSTANCE(BP) NEF_TC_INSTANCE_X(BP, _g, false, 0)
#define NEF_TC_GATHER_LOSS_INSTANCE(BP) NEF_TC_INSTANCE_X(BP, _g_loss, true, 0)
