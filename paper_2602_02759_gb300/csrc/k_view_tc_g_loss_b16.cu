// k_view_tc_g_loss_b16.cu -- loss-summing tcgen05 fused pass with gathered Q rows, bond_pad 16.
#include "k_view_tc_inst.cuh"

NEF_TC_GATHER_LOSS_INSTANCE(16)
