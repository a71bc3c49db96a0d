// k_view_simt_f64_b32.cu -- one instantiation of the CUDA-core fused pass (double, bond_pad 32).
#include "k_view_simt.cuh"

namespace nef {
NEF_SIMT_INSTANCE(view_simt_f64_b32, double, 32, 32)
}  // namespace nef
