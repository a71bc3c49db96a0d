"""GB300-native (sm_103a) multiplicative-update engine for nonnegative einsum
factorizations (NNEinFact).

    import paper_2602_02759_gb300 as nef
    plan = nef.Plan("ir,jr,kr->ijk", dict(i=512, j=512, k=512, r=64), precision="bf16")
    plan.fit(Y, None, [A, B, C], alpha=1.0, beta=0.0, iters=100)   # Algorithm 1
    total, count = plan.loss(Y, None, [A, B, C], 1.0, 0.0)         # Eq. 3.1

The work runs in libnef.so (C ABI in include/nef.h); this package only marshals
arguments.
"""
from ._nef import (  # noqa: F401
    EXPORTS,
    LIB_PATH,
    FoldIn,
    NEF_BF16,
    NEF_FP32,
    NEF_FP64,
    NefError,
    Plan,
    cp3_update_static,
    fit_batched,
    fit_batched_tune,
    load,
    pack_params,
    split_model,
)
from .slab import SlabFit, slab_bounds, slab_sweeps  # noqa: F401
