// k_view_simt_f32_b64.cu -- one instantiation of the CUDA-core fused pass (float, bond_pad 64).
#include "k_view_simt.cuh"

namespace nef {
NEF_SIMT_INSTANCE(view_simt_f32_b64, float, 64, 64)
}  // namespace nef
