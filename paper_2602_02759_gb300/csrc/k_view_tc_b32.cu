// k_view_tc_b32.cu -- tcgen05 fused pass instantiated for bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_INSTANCE(32)
