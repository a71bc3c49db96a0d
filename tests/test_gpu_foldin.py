"""GPU: the fold-in encoder (nef_foldin_*) and its tensor-core GEMM.

Tolerances: the GEMM is compared with the FP64 product of the same BF16
values (FP32 accumulation: 1e-5 relative).  The encoder computes its products
in BF16 (inputs, weights, activations and backward signals rounded to BF16,
FP32 accumulation), so its loss is compared with the FP64 oracle run on the
same parameters within 2e-3 relative, and each parameter's gradient within
3e-2 relative (Frobenius).  One Adam step moves every parameter by at most lr
(Adam's first step); the GPU and oracle steps agree elementwise within 2 lr and
on average within 0.05 lr.
"""
import numpy as np
import pytest

import synth
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu



def _probe():
    """The test-only probe library (tests/tc_probe): layout probe and GEMM alone."""
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tc_probe", "build.py")
    spec = importlib.util.spec_from_file_location("nef_probe_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.load()

def _nef():
    import paper_2602_02759_gb300 as nef
    return nef


def bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 72, 96), (64, 32, 32), (1536, 512, 1024), (96, 512, 1536)])
def test_tc_gemm(M, N, K):
    nef = _nef()
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K)).astype(np.float32)
    tA = torch.as_tensor(A).cuda().to(torch.bfloat16).contiguous()
    tB = torch.as_tensor(B).cuda().to(torch.bfloat16).contiguous()
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _probe().nef_tc_gemm(tA.data_ptr(), K, tB.data_ptr(), K, C.data_ptr(), N, M, N, K, err.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    ref = bf16(A) @ bf16(B).T
    got = C.cpu().numpy()
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("M,N,K,ldc", [(200, 72, 96, 80), (50, 30, 64, 30), (50, 30, 64, 33), (300, 40, 128, 44)])
def test_tc_gemm_row_pitch(M, N, K, ldc):
    """C with a row pitch wider than N: the tile stores (TMA stores where the pitch is a
    whole number of 16-byte units, per-element stores otherwise) write the M x N block
    and leave the columns between N and the pitch untouched."""
    nef = _nef()
    rng = np.random.default_rng(M + 3 * N + K + ldc)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K)).astype(np.float32)
    tA = torch.as_tensor(A).cuda().to(torch.bfloat16).contiguous()
    tB = torch.as_tensor(B).cuda().to(torch.bfloat16).contiguous()
    C = torch.full((M, ldc), -7.0, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _probe().nef_tc_gemm(tA.data_ptr(), K, tB.data_ptr(), K, C.data_ptr(), ldc, M, N, K, err.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    got = C.cpu().numpy()
    ref = bf16(A) @ bf16(B).T
    np.testing.assert_allclose(got[:, :N], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    assert np.all(got[:, N:] == -7.0)


@pytest.mark.parametrize("M,N,K,splits", [(256, 256, 4096, 8), (200, 72, 1000, 3), (1536, 512, 2048, 3)])
def test_tc_gemm_split_k(M, N, K, splits):
    """Split-K: the K blocks of each tile spread over `splits` CTAs, partial tiles
    summed in split order: the BF16 product within FP32 rounding of the FP64
    product of the same BF16 values, and bit-identical on a second call."""
    rng = np.random.default_rng(M + N + K)
    A = rng.uniform(-1, 1, (M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (N, K)).astype(np.float32)
    tA = torch.as_tensor(A).cuda().to(torch.bfloat16).contiguous()
    tB = torch.as_tensor(B).cuda().to(torch.bfloat16).contiguous()
    ws = torch.empty(splits * M * N, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = []
    for _ in range(2):
        C = torch.full((M, N), float("nan"), device="cuda")
        rc = _probe().nef_tc_gemm_split(tA.data_ptr(), K, tB.data_ptr(), K, C.data_ptr(), N, M, N, K, splits,
                                        ws.data_ptr(), ws.numel(), err.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0 and int(err.item()) == 0
        outs.append(C.cpu().numpy())
    ref = bf16(A) @ bf16(B).T
    np.testing.assert_allclose(outs[0], ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    np.testing.assert_array_equal(outs[0], outs[1])


def _setup(d=256, h=64, o=16, n=48, seed=0):
    rng = np.random.default_rng(seed)
    params = synth.mlp_params((d, h, h, o), seed=seed)
    params = [p + rng.uniform(-0.05, 0.05, p.shape) for p in params]   # nonzero biases
    slices = rng.poisson(rng.gamma(0.5, 2.0, (n, d))).astype(np.float32)
    targets = rng.gamma(0.5, 1.0, (n, o)).astype(np.float32)
    return params, slices, targets


def test_foldin_grad_matches_oracle():
    nef = _nef()
    d, h, o, n = 256, 64, 16, 48
    params, slices, targets = _setup(d, h, o, n)
    flat = torch.as_tensor(nef.pack_params(params)).cuda()
    enc = nef.FoldIn(d, h, o, n, flat)
    g, loss = enc.grad(torch.as_tensor(slices).cuda(), torch.as_tensor(targets).cuda())
    torch.cuda.synchronize()
    # oracle at the parameters the GPU computes with (BF16 inputs and weights)
    p_bf = [bf16(p) if p.ndim == 2 else p for p in params]
    out, cache = mlp.forward(p_bf, bf16(np.log1p(slices.astype(np.float64))))
    ref_loss = mlp.loss(out, targets.astype(np.float64))
    ref_g = mlp.backward(p_bf, cache, targets.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=2e-3)
    got = g.cpu().numpy().astype(np.float64)
    off = 0
    for k, rg in enumerate(ref_g):
        gk = got[off:off + rg.size].reshape(rg.shape)
        off += rg.size
        rel = np.linalg.norm(gk - rg) / max(np.linalg.norm(rg), 1e-30)
        assert rel < 3e-2, (k, rel)
    assert off == got.size


def test_foldin_adam_step_matches_oracle():
    nef = _nef()
    d, h, o, n = 256, 64, 16, 48
    params, slices, targets = _setup(d, h, o, n, seed=1)
    flat = torch.as_tensor(nef.pack_params(params)).cuda()
    enc = nef.FoldIn(d, h, o, n, flat)
    lr = 1e-3
    enc.train_step(torch.as_tensor(slices).cuda(), torch.as_tensor(targets).cuda(), lr)
    got = enc.params().cpu().numpy().astype(np.float64)
    p_ref = [p.astype(np.float64).copy() for p in params]
    p_bf = [bf16(p) if p.ndim == 2 else p for p in params]
    out, cache = mlp.forward(p_bf, bf16(np.log1p(slices.astype(np.float64))))
    grads = mlp.backward(p_bf, cache, targets.astype(np.float64))
    mlp.adam_step(p_ref, grads, mlp.adam_state(p_ref), lr, 1)
    ref = np.concatenate([p.reshape(-1) for p in p_ref])
    start = np.concatenate([np.asarray(p, np.float32).reshape(-1) for p in params]).astype(np.float64)
    assert np.max(np.abs(got - start)) <= lr * 1.001 + 1e-7
    diff = np.abs(got - ref)
    assert diff.max() <= 2 * lr * 1.001 + 1e-7
    assert diff.mean() < 0.05 * lr


def test_foldin_gain_over_plain_foldin():
    """The trained encoder's loadings, refined by k MU passes on mode 0 with B, C
    fixed, reach a lower held-out loss than the plain MU fold-in from the usual
    initialisation after the same k passes (k = 0, 1, 2).  The encoder is trained
    on each component's expected count in the slice, A[i, r] * sum_j B[j, r] *
    sum_k C[k, r] (the scale of the data, where log1p separates small loadings),
    and its output is divided by the same factor."""
    nef = _nef()
    n_tr, n_te, J, K, R = 256, 128, 16, 16, 8
    p = synth.make_problem("ir,jr,kr->ijk", {"i": n_tr + n_te, "j": J, "k": K, "r": R}, seed=5,
                           gamma=(0.3, 1.0), missing=0.0, alpha=1.0, beta=0.0)
    y = torch.as_tensor(p.y).cuda()
    ytr, yte = y[:n_tr].contiguous(), y[n_tr:].contiguous()
    # 1. MU fit on the training slices: B, C and the training loadings
    A0, B0, C0 = (torch.as_tensor(f).cuda() for f in p.inits[0])
    fs = [A0[:n_tr].contiguous(), B0.clone(), C0.clone()]
    fit = nef.Plan("ir,jr,kr->ijk", dict(i=n_tr, j=J, k=K, r=R), precision="fp32")
    fit.fit(ytr, None, fs, 1.0, 0.0, 300)
    A_tr, B, C = fs
    # 2. train the encoder on (slice, loading) pairs
    d = J * K
    params = synth.mlp_params((d, 64, 64, R), seed=3)
    enc = nef.FoldIn(d, 64, R, n_tr, torch.as_tensor(nef.pack_params(params)).cuda())
    xs = ytr.reshape(n_tr, d).contiguous()
    mass = (B.sum(0) * C.sum(0))[None, :]
    targets = (A_tr * mass).contiguous()
    first = last = None
    for step in range(400):
        l = enc.train_step(xs, targets, 2e-3, want_loss=(step % 50 == 0 or step == 399))
        if l is not None:
            first = l if first is None else first
            last = l
    assert last < 0.5 * first
    # 3. fold in the held-out slices: encoder + k passes vs plain init + k passes
    ref = nef.Plan("ir,jr,kr->ijk", dict(i=n_te, j=J, k=K, r=R), precision="fp32")
    A_enc = (enc.predict(yte.reshape(n_te, d).contiguous()) / mass).contiguous()
    A_plain = A0[n_tr:].contiguous()

    def held_out_loss(A, k):
        fs2 = [A.clone(), B, C]
        for _ in range(k):
            ref.update(0, yte, None, fs2, 1.0, 0.0)
        return ref.loss(yte, None, fs2, 1.0, 0.0)[0]

    full = held_out_loss(A_plain, 200)
    for k in (0, 1, 2):
        le, lp = held_out_loss(A_enc, k), held_out_loss(A_plain, k)
        # the gap to the converged fold-in shrinks by at least 2x
        assert (le - full) < 0.5 * (lp - full), (k, le, lp, full)
    assert held_out_loss(A_enc, 20) == pytest.approx(full, rel=1e-2)


def test_foldin_gain_at_benchmark_size():
    """The fold-in workload at its full size: CP 'ir,jr,kr->ijk' 2048 x 128 x 128,
    R = 32, KL; B, C from a BF16 MU fit of the 1536 training slices; the encoder
    16384 -> 512 -> 512 -> 32 trained by 200 Adam steps on (slice, component count
    mass) pairs; the 512 held-out slices folded in from the encoder's loadings and
    from the plain initialisation, each refined by k MU passes on mode 0 with B, C
    fixed.  The encoder's gap to the converged fold-in (500 passes) is below the
    plain initialisation's after k = 0, 1, 2 and 5 passes."""
    nef = _nef()
    p = synth.config5()
    n, J, K = p.y.shape
    R, n_tr = p.dims["r"], 1536
    n_te, d = n - n_tr, J * K
    y = torch.from_numpy(p.y).cuda()
    ytr, yte = y[:n_tr].contiguous(), y[n_tr:].contiguous()
    A0, B0, C0 = (torch.from_numpy(f).cuda() for f in p.inits[0])
    fs = [A0[:n_tr].contiguous(), B0.clone(), C0.clone()]
    nef.Plan(p.model_str, dict(i=n_tr, j=J, k=K, r=R), precision="bf16").fit(ytr, None, fs, 1.0, 0.0, 100)
    A_tr, B, C = fs
    mass = (B.sum(0) * C.sum(0))[None, :]
    enc = nef.FoldIn(d, 512, R, n_tr,
                     torch.from_numpy(nef.pack_params(synth.mlp_params((d, 512, 512, R), 3))).cuda())
    xs = ytr.reshape(n_tr, d).contiguous()
    targets = (A_tr * mass).contiguous()
    first = enc.train_step(xs, targets, 1e-3)
    for _ in range(198):
        enc.train_step(xs, targets, 1e-3, want_loss=False)
    last = enc.train_step(xs, targets, 1e-3)
    assert last < 0.5 * first, (first, last)
    ref = nef.Plan(p.model_str, dict(i=n_te, j=J, k=K, r=R), precision="fp32")
    A_enc = (enc.predict(yte.reshape(n_te, d).contiguous()) / mass).contiguous()
    A_plain = A0[n_tr:].contiguous()

    def held_out_loss(A, k):
        fs2 = [A.clone(), B, C]
        for _ in range(k):
            ref.update(0, yte, None, fs2, 1.0, 0.0)
        return ref.loss(yte, None, fs2, 1.0, 0.0)[0]

    full = held_out_loss(A_plain, 500)
    gaps = {}
    for k in (0, 1, 2, 5):
        le, lp = held_out_loss(A_enc, k), held_out_loss(A_plain, k)
        gaps[k] = ((le - full) / full, (lp - full) / full)
        assert le - full < lp - full, (k, gaps)
    print("fold-in gaps (encoder, plain) by passes:", gaps)


def test_foldin_kept_batch_steps_equal_passed_batch():
    """Full-batch training on the GPU: five Adam steps on a batch kept by
    nef_foldin_load_batch give bit for bit the parameters of five steps that pass
    the slices each time (the same features, products and reductions)."""
    nef = _nef()
    d, h, o, n = 1024, 256, 32, 384
    rng = np.random.default_rng(11)
    xs = torch.as_tensor(rng.poisson(0.4, (n, d)).astype(np.float32)).cuda()
    tg = torch.as_tensor(rng.gamma(0.5, 1.0, (n, o)).astype(np.float32)).cuda()
    flat = torch.as_tensor(nef.pack_params(synth.mlp_params((d, h, h, o), 4))).cuda()
    a = nef.FoldIn(d, h, o, n, flat.clone())
    b = nef.FoldIn(d, h, o, n, flat.clone())
    b.load_batch(xs)
    for _ in range(5):
        a.train_step(xs, tg, 1e-3, want_loss=False)
        b.train_step(None, tg, 1e-3, want_loss=False)
    torch.cuda.synchronize()
    assert torch.equal(a.params(), b.params())
