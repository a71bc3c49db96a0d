"""Host logic of the fold-in encoder (foldin.cpp: parameter packing, buffer
layout, the forward and backward orchestration with its transposed BF16
copies, Adam, the loss read-back and the argument checks) against the FP64
oracle MLP.

foldin.cpp is compiled with g++ into the host test double (tests/hostcheck),
where plain-loop launchers follow each kernel's documented meaning (BF16
copies rounded to nearest even, FP32 accumulation); the kernels themselves are
checked on the GPU (test_gpu_foldin.py).  Tolerances as there: loss 2e-3,
gradients 3e-2 relative, one Adam step within 2 lr elementwise.
"""
import ctypes
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "hostcheck"))
import build as hostcheck_build  # noqa: E402

import synth  # noqa: E402
from oracle import mlp  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    lib = ctypes.CDLL(hostcheck_build.build())
    vp = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.nef_foldin_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                      ctypes.POINTER(vp)]
    lib.nef_foldin_destroy.argtypes = [vp]
    lib.nef_foldin_grad.argtypes = [vp, vp, vp, ctypes.c_int, vp, dp]
    lib.nef_foldin_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, dp]
    lib.nef_foldin_predict.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.nef_foldin_load_batch.argtypes = [vp, vp, ctypes.c_int]
    lib.nef_foldin_params.argtypes = [vp, vp]
    lib.nef_foldin_num_params.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.nef_foldin_num_params.restype = ctypes.c_int64
    lib.nef_last_error.restype = ctypes.c_char_p
    return lib


def bf16(x):
    a = np.ascontiguousarray(np.asarray(x, np.float32)).view(np.uint32)
    r = ((a + np.uint32(0x7FFF) + ((a >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def setup(d=64, h=32, o=8, n=12, seed=0):
    rng = np.random.default_rng(seed)
    params = synth.mlp_params((d, h, h, o), seed=seed)
    params = [p + rng.uniform(-0.05, 0.05, p.shape) for p in params]
    slices = rng.poisson(rng.gamma(0.5, 2.0, (n, d))).astype(np.float32)
    targets = rng.gamma(0.5, 1.0, (n, o)).astype(np.float32)
    flat = np.concatenate([np.asarray(p, np.float32).reshape(-1) for p in params])
    return params, slices, targets, flat


def create(lib, d, h, o, n, flat):
    handle = ctypes.c_void_p()
    rc = lib.nef_foldin_create(d, h, o, n, flat.ctypes.data, None, ctypes.byref(handle))
    assert rc == 0, lib.nef_last_error()
    return handle


def oracle_grads(params, slices, targets):
    p_bf = [bf16(p) if p.ndim == 2 else p for p in params]
    out, cache = mlp.forward(p_bf, bf16(np.log1p(slices.astype(np.float64))))
    return mlp.loss(out, targets.astype(np.float64)), mlp.backward(p_bf, cache, targets.astype(np.float64)), out


def test_foldin_grad_and_predict_match_oracle(lib):
    d, h, o, n = 64, 32, 8, 12
    params, slices, targets, flat = setup(d, h, o, n)
    assert lib.nef_foldin_num_params(d, h, o) == flat.size
    f = create(lib, d, h, o, n, flat)
    try:
        g = np.zeros(flat.size, np.float32)
        loss = ctypes.c_double()
        assert lib.nef_foldin_grad(f, slices.ctypes.data, targets.ctypes.data, n, g.ctypes.data,
                                   ctypes.byref(loss)) == 0
        ref_loss, ref_g, ref_out = oracle_grads(params, slices, targets)
        assert loss.value == pytest.approx(ref_loss, rel=2e-3)
        off = 0
        for k, rg in enumerate(ref_g):
            gk = g[off:off + rg.size].reshape(rg.shape).astype(np.float64)
            off += rg.size
            assert np.linalg.norm(gk - rg) / max(np.linalg.norm(rg), 1e-30) < 3e-2, k
        assert off == g.size
        out = np.zeros((n - 3, o), np.float32)
        assert lib.nef_foldin_predict(f, slices.ctypes.data, n - 3, out.ctypes.data) == 0
        np.testing.assert_allclose(out, ref_out[: n - 3], rtol=2e-2, atol=1e-3)
    finally:
        lib.nef_foldin_destroy(f)


def test_foldin_adam_step_matches_oracle(lib):
    d, h, o, n = 64, 32, 8, 12
    params, slices, targets, flat = setup(d, h, o, n, seed=1)
    f = create(lib, d, h, o, n, flat)
    try:
        lr = 1e-3
        loss = ctypes.c_double()
        assert lib.nef_foldin_train_step(f, slices.ctypes.data, targets.ctypes.data, n, lr, 0.9, 0.999, 1e-8,
                                         ctypes.byref(loss)) == 0
        got = np.zeros(flat.size, np.float32)
        assert lib.nef_foldin_params(f, got.ctypes.data) == 0
        p_ref = [p.astype(np.float64).copy() for p in params]
        _, grads, _ = oracle_grads(params, slices, targets)
        mlp.adam_step(p_ref, grads, mlp.adam_state(p_ref), lr, 1)
        ref = np.concatenate([p.reshape(-1) for p in p_ref])
        got = got.astype(np.float64)
        assert np.max(np.abs(got - flat.astype(np.float64))) <= lr * 1.001 + 1e-7
        diff = np.abs(got - ref)
        assert diff.max() <= 2 * lr * 1.001 + 1e-7
        assert diff.mean() < 0.05 * lr
    finally:
        lib.nef_foldin_destroy(f)


def test_foldin_argument_errors(lib):
    d, h, o, n = 64, 32, 8, 12
    _, slices, targets, flat = setup(d, h, o, n)
    handle = ctypes.c_void_p()
    assert lib.nef_foldin_create(60, h, o, n, flat.ctypes.data, None, ctypes.byref(handle)) != 0
    assert b"multiples of 8" in lib.nef_last_error()
    assert lib.nef_foldin_create(d, h, o, 0, flat.ctypes.data, None, ctypes.byref(handle)) != 0
    f = create(lib, d, h, o, n, flat)
    try:
        out = np.zeros((n + 1, o), np.float32)
        assert lib.nef_foldin_predict(f, slices.ctypes.data, n + 1, out.ctypes.data) != 0
        assert b"batch" in lib.nef_last_error()
        assert lib.nef_foldin_train_step(f, slices.ctypes.data, targets.ctypes.data, n, -1.0, 0.9, 0.999, 1e-8,
                                         None) != 0
    finally:
        lib.nef_foldin_destroy(f)


def test_foldin_kept_batch_steps_equal_passed_batch(lib):
    """Three Adam steps on a batch kept by nef_foldin_load_batch give exactly the
    parameters of three steps that pass the slices each time; a call that passes
    slices drops the kept batch, after which slices == NULL is rejected."""
    d, h, o, n = 64, 32, 8, 12
    _, slices, targets, flat = setup(d, h, o, n, seed=2)
    a = create(lib, d, h, o, n, flat)
    b = create(lib, d, h, o, n, flat)
    try:
        assert lib.nef_foldin_load_batch(b, slices.ctypes.data, n) == 0
        for _ in range(3):
            assert lib.nef_foldin_train_step(a, slices.ctypes.data, targets.ctypes.data, n, 1e-3, 0.9, 0.999,
                                             1e-8, None) == 0
            assert lib.nef_foldin_train_step(b, None, targets.ctypes.data, n, 1e-3, 0.9, 0.999, 1e-8, None) == 0
        pa = np.zeros(flat.size, np.float32)
        pb = np.zeros(flat.size, np.float32)
        assert lib.nef_foldin_params(a, pa.ctypes.data) == 0 and lib.nef_foldin_params(b, pb.ctypes.data) == 0
        assert np.array_equal(pa, pb)
        assert lib.nef_foldin_train_step(b, None, targets.ctypes.data, n - 1, 1e-3, 0.9, 0.999, 1e-8, None) != 0
        out = np.zeros((n, o), np.float32)
        assert lib.nef_foldin_predict(b, slices.ctypes.data, n, out.ctypes.data) == 0
        assert lib.nef_foldin_train_step(b, None, targets.ctypes.data, n, 1e-3, 0.9, 0.999, 1e-8, None) != 0
        assert b"kept" in lib.nef_last_error()
    finally:
        lib.nef_foldin_destroy(a)
        lib.nef_foldin_destroy(b)
