// k_view_simt_f32_b16.cu -- one instantiation of the CUDA-core fused pass (float, bond_pad 16).
#include "k_view_simt.cuh"

namespace nef {
NEF_SIMT_INSTANCE(view_simt_f32_b16, float, 64, 16)
}  // namespace nef
