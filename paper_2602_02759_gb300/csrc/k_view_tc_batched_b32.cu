// k_view_tc_batched_b32.cu -- batched tensor-core pass instantiated for bond_pad 32.
#include "k_view_tc_inst.cuh"

NEF_TC_BATCHED_INSTANCE(32)
