// k_view_tc_lik_loss_b32.cu -- loss-summing tcgen05 fused pass for the likelihood
// families of App. B, bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_LIK_LOSS_INSTANCE(32)
