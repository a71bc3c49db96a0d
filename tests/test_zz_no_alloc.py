"""nef_cp3_update_static, the factor update that allocates no device memory,
through the C ABI.

Callers that cannot allocate device memory (a framework's caching allocator
owns it, or their loop forbids allocation after start-up) use the static entry
point.  It must give the factor update of Algorithm 1 (Eq. 3.4 with App. B's
weights) that the FP64 oracle gives, within the FP32 tolerance the other parity
tests use (1e-5 relative, Frobenius), call after call, and agree with the planned
NEF_FP32 update nef_update.  This file is collected last so that a run that
stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from oracle import OracleModel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.0, -0.5)])
def test_static_update_matches_oracle_two_calls(R, ab):
    import paper_2602_02759_gb300 as nef
    a, b = ab
    I, J, K = 160, 96, 192
    rng = np.random.default_rng(5 + R)
    truth = [rng.gamma(0.3, 1.0, (n, R)) for n in (I, J, K)]
    y = rng.poisson(np.einsum("ir,jr,kr->ijk", *truth)).astype(np.float32)
    init = [rng.uniform(0.5, 1.5, (n, R)).astype(np.float32) for n in (I, J, K)]
    m = OracleModel("ir,jr,kr->ijk", dict(i=I, j=J, k=K, r=R))
    Y = torch.from_numpy(y).cuda()
    plan = nef.Plan("ir,jr,kr->ijk", dict(i=I, j=J, k=K, r=R), precision="fp32")
    for l in range(3):
        ref = [f.astype(np.float64) for f in init]
        planned = [torch.from_numpy(f).cuda() for f in init]
        got = [torch.from_numpy(f).cuda() for f in init]
        for call in range(2):  # two calls in a row on the same factors
            ref = m.update_factor(l, y, None, ref, a, b)[0]
            plan.update(l, Y, None, planned, a, b)
            nef.cp3_update_static(Y, got, l, a, b)
            torch.cuda.synchronize()
            g = got[l].cpu().numpy()
            assert _rel(g, ref[l]) < 1e-5, (l, call, _rel(g, ref[l]))
            assert _rel(g, planned[l].cpu().numpy()) < 1e-5
            for q in range(3):
                if q != l:
                    assert np.array_equal(got[q].cpu().numpy(), init[q])


def test_static_update_at_the_scratch_limit():
    """rows x R = 1,048,576 exactly (I = 16384, R = 64): the scratch then holds one
    column split and the reduced num/den; checked against the oracle."""
    import paper_2602_02759_gb300 as nef
    I, J, K, R = 16384, 8, 12, 64
    rng = np.random.default_rng(6)
    truth = [rng.gamma(0.3, 1.0, (n, R)) for n in (I, J, K)]
    y = rng.poisson(np.einsum("ir,jr,kr->ijk", *truth)).astype(np.float32)
    init = [rng.uniform(0.5, 1.5, (n, R)).astype(np.float32) for n in (I, J, K)]
    m = OracleModel("ir,jr,kr->ijk", dict(i=I, j=J, k=K, r=R))
    ref = m.update_factor(0, y, None, [f.astype(np.float64) for f in init], 1.0, 0.0)[0]
    got = [torch.from_numpy(f).cuda() for f in init]
    nef.cp3_update_static(torch.from_numpy(y).cuda(), got, 0, 1.0, 0.0)
    torch.cuda.synchronize()
    assert _rel(got[0].cpu().numpy(), ref[0]) < 1e-5


def test_static_update_rejects_bad_arguments_before_launch():
    import paper_2602_02759_gb300 as nef
    from paper_2602_02759_gb300._nef import NefError
    Y = torch.ones(4, 4, 4, device="cuda")
    with pytest.raises(NefError, match="rank"):
        nef.cp3_update_static(Y, [torch.ones(4, 8, device="cuda") for _ in range(3)], 0, 1.0, 0.0)
    # a factor with too few rows, a rank mismatch, a wrong dtype: caught by the binding
    with pytest.raises(NefError, match="factor 1"):
        nef.cp3_update_static(Y, [torch.ones(4, 16, device="cuda"), torch.ones(3, 16, device="cuda"),
                                  torch.ones(4, 16, device="cuda")], 0, 1.0, 0.0)
    with pytest.raises(NefError, match="factor 2"):
        nef.cp3_update_static(Y, [torch.ones(4, 16, device="cuda")] * 2 + [torch.ones(4, 32, device="cuda")],
                              0, 1.0, 0.0)
    with pytest.raises(NefError, match="factor 0"):
        nef.cp3_update_static(Y, [torch.ones(4, 16, device="cuda", dtype=torch.float64)] +
                              [torch.ones(4, 16, device="cuda")] * 2, 0, 1.0, 0.0)
    with pytest.raises(NefError, match="Y must"):
        nef.cp3_update_static(Y.double(), [torch.ones(4, 16, device="cuda")] * 3, 0, 1.0, 0.0)
    good = [torch.ones(4, 16, device="cuda") for _ in range(3)]
    before = [g.clone() for g in good]
    for a, b, eps in ((float("nan"), 0.0, 1e-10), (1.0, float("inf"), 1e-10), (1.0, 0.0, float("inf")),
                      (1.0, 0.0, -1.0)):
        with pytest.raises(NefError) as ei:
            nef.cp3_update_static(Y, good, 0, a, b, eps=eps)
        assert ei.value.status == 1
    with pytest.raises(NefError) as ei:
        nef.cp3_update_static(Y, good, 0, 0.0, 0.5)
    assert ei.value.status == 3
    torch.cuda.synchronize()
    assert all(torch.equal(g, h) for g, h in zip(good, before))
    # rows x rank beyond the fixed scratch: only the shape is checked, nothing is launched
    lib = nef.load()
    Yb = torch.ones(1, 1, 1, device="cuda")
    shape_facs = [torch.ones(1, 64, device="cuda")] * 3
    shape = (ctypes.c_int64 * 3)(1 << 15, 1, 1)
    arr = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in shape_facs])
    rc = lib.nef_cp3_update_static(ctypes.c_void_p(Yb.data_ptr()), shape, 64, arr, 0, 1.0, 0.0, 1e-10,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1 and b"static scratch" in lib.nef_last_error()
