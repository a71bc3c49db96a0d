// k_view_simt.cu -- dispatch of the CUDA-core fused pass over (element type, bond_pad).
#include "nef_internal.h"

namespace nef {

#define NEF_SIMT_DECL(NAME, T)                                                                  \
    cudaError_t NAME(const T* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, \
                     int need_den, int n_split, T* s_num, T* s_den, const LossSpec* loss,       \
                     double* loss_part, cudaStream_t st, int* n_ctas);
NEF_SIMT_DECL(view_simt_f32_b16, float)
NEF_SIMT_DECL(view_simt_f32_b32, float)
NEF_SIMT_DECL(view_simt_f32_b64, float)
NEF_SIMT_DECL(view_simt_f64_b32, double)
NEF_SIMT_DECL(view_simt_f64_b64, double)

template <>
cudaError_t launch_view_simt<float>(const float* y, const uint32_t* mbits, const ViewDesc& v,
                                    const WeightSpec& w, int need_den, int n_split, float* s_num,
                                    float* s_den, const LossSpec* loss, double* loss_part,
                                    cudaStream_t st, int* n_ctas) {
    switch (v.bond_pad) {
        case 16: return view_simt_f32_b16(y, mbits, v, w, need_den, n_split, s_num, s_den, loss, loss_part, st, n_ctas);
        case 32: return view_simt_f32_b32(y, mbits, v, w, need_den, n_split, s_num, s_den, loss, loss_part, st, n_ctas);
        case 64: return view_simt_f32_b64(y, mbits, v, w, need_den, n_split, s_num, s_den, loss, loss_part, st, n_ctas);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_view_simt<double>(const double* y, const uint32_t* mbits, const ViewDesc& v,
                                     const WeightSpec& w, int need_den, int n_split, double* s_num,
                                     double* s_den, const LossSpec* loss, double* loss_part,
                                     cudaStream_t st, int* n_ctas) {
    switch (v.bond_pad) {
        case 32: return view_simt_f64_b32(y, mbits, v, w, need_den, n_split, s_num, s_den, loss, loss_part, st, n_ctas);
        case 64: return view_simt_f64_b64(y, mbits, v, w, need_den, n_split, s_num, s_den, loss, loss_part, st, n_ctas);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace nef
