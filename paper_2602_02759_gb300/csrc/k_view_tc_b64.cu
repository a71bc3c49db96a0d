// k_view_tc_b64.cu -- tcgen05 fused pass instantiated for bond_pad 64.
#include "k_view_tc_inst.cuh"

NEF_TC_INSTANCE(64)
