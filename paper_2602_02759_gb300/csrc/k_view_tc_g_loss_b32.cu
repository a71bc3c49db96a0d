// k_view_tc_g_loss_b32.cu -- loss-summing tcgen05 fused pass with gathered Q rows, bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_GATHER_LOSS_INSTANCE(32)
