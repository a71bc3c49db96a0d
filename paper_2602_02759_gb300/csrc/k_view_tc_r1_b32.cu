// k_view_tc_r1_b32.cu -- tcgen05 fused pass with staged Q rows in the alternative
// ring-depth configuration (chosen per view by the autotuner), bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_RING1_INSTANCE(32)
