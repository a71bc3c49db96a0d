// k_view_simt_f32_b32.cu -- one instantiation of the CUDA-core fused pass (float, bond_pad 32).
#include "k_view_simt.cuh"

namespace nef {
NEF_SIMT_INSTANCE(view_simt_f32_b32, float, 64, 32)
}  // namespace nef
