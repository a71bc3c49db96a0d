"""nef_cp3_update_static (the factor update that allocates no device memory)
against the planned update nef_update, through the C ABI.

Callers that cannot allocate device memory (a framework's caching allocator
owns it, or their loop forbids allocation) use the static entry point; it must
give the same factors as a planned NEF_FP32 update, within the FP32 tolerance
the other parity tests use (1e-5 relative), call after call.  This file is
collected last so that a run that stops at the first failure has already run
every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu()
    b = b.double().cpu()
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.0, -0.5)])
def test_static_update_matches_planned_update_two_calls(ab):
    import paper_2602_02759_gb300 as nef
    a, b = ab
    I, J, K, R = 160, 96, 192, 32
    rng = np.random.default_rng(5)
    truth = [rng.gamma(0.3, 1.0, (n, R)) for n in (I, J, K)]
    y = rng.poisson(np.einsum("ir,jr,kr->ijk", *truth)).astype(np.float32)
    init = [rng.uniform(0.5, 1.5, (n, R)).astype(np.float32) for n in (I, J, K)]
    Y = torch.from_numpy(y).cuda()
    plan = nef.Plan("ir,jr,kr->ijk", dict(i=I, j=J, k=K, r=R), precision="fp32")
    for l in range(3):
        ref = [torch.from_numpy(f).cuda() for f in init]
        got = [torch.from_numpy(f).cuda() for f in init]
        for call in range(2):  # two calls in a row on the same factors
            plan.update(l, Y, None, ref, a, b)
            nef.cp3_update_static(Y, got, l, a, b)
            torch.cuda.synchronize()
            assert _rel(got[l], ref[l]) < 1e-5, (l, call, _rel(got[l], ref[l]))
            for q in range(3):
                if q != l:
                    assert torch.equal(got[q], ref[q])


def test_static_update_rejects_oversized_and_bad_rank():
    import paper_2602_02759_gb300 as nef
    from paper_2602_02759_gb300._nef import NefError
    Y = torch.ones(4, 4, 4, device="cuda")
    bad_rank = [torch.ones(4, 8, device="cuda") for _ in range(3)]
    with pytest.raises(NefError, match="rank"):
        nef.cp3_update_static(Y, bad_rank, 0, 1.0, 0.0)
    # rows x rank beyond the fixed scratch: only the shape is checked, nothing is launched
    big_rows = 1 << 15
    Yb = torch.ones(1, 1, 1, device="cuda")
    shape_facs = [torch.ones(1, 64, device="cuda")] * 3
    import ctypes
    lib = nef.load()
    shape = (ctypes.c_int64 * 3)(big_rows, 1, 1)
    arr = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in shape_facs])
    rc = lib.nef_cp3_update_static(ctypes.c_void_p(Yb.data_ptr()), shape, 64, arr, 0, 1.0, 0.0, 1e-10,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1 and b"static scratch" in lib.nef_last_error()
