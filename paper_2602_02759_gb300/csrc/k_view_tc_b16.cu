// k_view_tc_b16.cu -- tcgen05 fused pass instantiated for bond_pad 16.
#include "k_view_tc_inst.cuh"

NEF_TC_INSTANCE(16)
