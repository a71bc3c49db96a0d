// k_view_simt_f64_b64.cu -- one instantiation of the CUDA-core fused pass (double, bond_pad 64).
#include "k_view_simt.cuh"

namespace nef {
NEF_SIMT_INSTANCE(view_simt_f64_b64, double, 32, 64)
}  // namespace nef
