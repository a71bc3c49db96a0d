"""The bounded-wait failure path of the tensor-core pass, without faulting the GPU.

Every wait inside the pass gives up after nef_options.wait_cycles SM cycles; the
kernel then raises its error flag, waits (under the fixed long limit) for its own
copies and products already in flight, frees its tensor memory and returns.  A
plan with a limit of a few cycles makes its first waits run out: nef_check must
report NEF_ETIMEOUT, and afterwards the same context must run a normal fit that
still matches the FP64 oracle.  No trap, no fault and no endless loop is
involved: the host reads the status between calls.
"""
import numpy as np
import pytest

from oracle import OracleModel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_wait_limit_runs_out_and_context_stays_usable():
    import paper_2602_02759_gb300 as nef
    from paper_2602_02759_gb300._nef import NefError
    model_str, dims = "ir,jr,kr->ijk", dict(i=128, j=96, k=160, r=32)
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(31)
    truth = [rng.gamma(0.3, 1.0, m.factor_shape(l)) for l in range(3)]
    y = rng.poisson(np.einsum(model_str, *truth)).astype(np.float32)
    init = [rng.uniform(0.5, 1.5, m.factor_shape(l)) for l in range(3)]
    Y = torch.from_numpy(y).cuda()

    tiny = nef.Plan(model_str, dims, precision="bf16", wait_cycles=16, eager=True)
    fs = [torch.from_numpy(f.astype(np.float32)).cuda() for f in init]
    tiny.fit(Y, None, fs, 1.0, 0.0, 2)
    with pytest.raises(NefError) as ei:
        tiny.check()
    assert ei.value.status == 7, ei.value  # NEF_ETIMEOUT
    tiny.check()  # the flag was cleared
    del tiny
    torch.cuda.synchronize()

    iters = 5
    _, trace = m.fit(y, None, init, 1.0, 0.0, iters, trace=True)
    plan = nef.Plan(model_str, dims, precision="bf16")
    fs = [torch.from_numpy(f.astype(np.float32)).cuda() for f in init]
    plan.fit(Y, None, fs, 1.0, 0.0, iters)
    plan.check()
    lo, _ = plan.loss(Y, None, fs, 1.0, 0.0)
    assert lo == pytest.approx(trace[-1], rel=1e-3)
