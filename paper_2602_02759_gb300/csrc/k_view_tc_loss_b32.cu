// k_view_tc_loss_b32.cu -- loss-summing tcgen05 fused pass for bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_LOSS_INSTANCE(32)
