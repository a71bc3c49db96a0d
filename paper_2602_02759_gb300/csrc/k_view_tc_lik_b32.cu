// k_view_tc_lik_b32.cu -- tcgen05 fused pass for the likelihood families of App. B
// (negative binomial, binomial on the odds, Jensen-Shannon), bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_LIK_INSTANCE(32)
