"""Host logic of the batched engine (batched.cpp: padded layouts, units, work
tables, per-split partial offsets, the graph-captured sweep loop and the
per-restart losses) against the oracle.

batched.cpp is compiled with g++ into the host test double (tests/hostcheck),
where plain-loop launchers follow each kernel descriptor's documented meaning
and round operands to BF16 where the tensor-core pass does; the kernels
themselves are checked on the GPU (test_gpu_batched.py).
"""
import ctypes
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "hostcheck"))
import build as hostcheck_build  # noqa: E402

from oracle import OracleModel  # noqa: E402
from test_host_plan import NEF_BF16, NEF_FP32, Opt  # noqa: E402

MODEL = "ir,jr,kr->ijk"


@pytest.fixture(scope="module")
def lib():
    lib = ctypes.CDLL(hostcheck_build.build())
    vp = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.nef_fit_batched.argtypes = [ctypes.c_int, i64p, i64p, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.POINTER(Opt), ctypes.POINTER(ctypes.c_double)]
    lib.nef_fit_batched_tune.argtypes = [ctypes.c_int, i64p, i64p, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(Opt), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]
    lib.nef_default_options.argtypes = [ctypes.POINTER(Opt)]
    lib.nef_last_error.restype = ctypes.c_char_p
    return lib


def problems(seed, shapes, ranks, restarts, missing):
    rng = np.random.default_rng(seed)
    out = []
    for (I, J, K), R in zip(shapes, ranks):
        truth = [rng.gamma(0.3, 1.0, (n, R)) for n in (I, J, K)]
        y = rng.poisson(np.einsum(MODEL, *truth)).astype(np.float32)
        mask = (rng.random(y.shape) >= missing).astype(np.uint8)
        inits = [[rng.uniform(0.5, 1.5, (n, R)).astype(np.float32) for n in (I, J, K)] for _ in range(restarts)]
        out.append((y, mask, inits))
    return out


def call(lib, shapes, ranks, probs, restarts, a, b, iters, prec=NEF_BF16, tiles=0):
    n = len(shapes)
    sh = (ctypes.c_int64 * (3 * n))(*[d for s in shapes for d in s])
    rk = (ctypes.c_int64 * n)(*ranks)
    ys = (ctypes.c_void_p * n)(*[p[0].ctypes.data for p in probs])
    ms = (ctypes.c_void_p * n)(*[p[1].ctypes.data for p in probs])
    work = [[f.copy() for f in p[2][k % len(p[2])]] for p in probs for k in range(restarts)]
    fs = (ctypes.c_void_p * (3 * n * restarts))(*[f.ctypes.data for u in work for f in u])
    losses = (ctypes.c_double * (n * restarts))()
    o = Opt()
    lib.nef_default_options(ctypes.byref(o))
    o.precision = prec
    o.batch_tiles = tiles
    rc = lib.nef_fit_batched(n, sh, rk, ys, ms, fs, restarts, a, b, iters, ctypes.byref(o), losses)
    return rc, work, list(losses)


@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.0, -0.5)])
def test_batched_fit_matches_oracle(lib, ab):
    """Uneven shapes (not multiples of 4: padded), ranks on both bond widths
    (16 and 32), two restarts, 10 % missing: every unit's factors after two
    sweeps and its loss against the FP64 oracle started from the same point."""
    a, b = ab
    shapes = [(5, 7, 9), (12, 3, 6), (70, 9, 66)]
    ranks = [3, 17, 8]
    restarts = 2
    probs = problems(3, shapes, ranks, restarts, 0.1)
    rc, work, losses = call(lib, shapes, ranks, probs, restarts, a, b, 2)
    assert rc == 0, lib.nef_last_error()
    for p, ((I, J, K), R) in enumerate(zip(shapes, ranks)):
        m = OracleModel(MODEL, dict(i=I, j=J, k=K, r=R))
        y, mask, inits = probs[p]
        for k in range(restarts):
            ref = m.fit(y.astype(np.float64), mask, [f.astype(np.float64) for f in inits[k]], a, b, 2)
            got = work[p * restarts + k]
            for q in range(3):
                rel = np.linalg.norm(got[q] - ref[q]) / np.linalg.norm(ref[q])
                assert rel < 1e-2, (p, k, q, rel)
            lref, _ = m.loss(y.astype(np.float64), mask, [g.astype(np.float64) for g in got], a, b)
            assert losses[p * restarts + k] == pytest.approx(lref, rel=1e-5)


def test_batched_argument_errors(lib):
    shapes = [(5, 7, 9)]
    probs = problems(4, shapes, [3], 1, 0.0)
    rc, _, _ = call(lib, shapes, [3], probs, 1, 1.0, 0.0, 1, prec=NEF_FP32)
    assert rc != 0 and b"tensor cores" in lib.nef_last_error()
    rc, _, _ = call(lib, shapes, [33], probs, 1, 1.0, 0.0, 1)
    assert rc != 0 and b"ranks" in lib.nef_last_error()
    rc, _, _ = call(lib, shapes, [3], probs, 17, 1.0, 0.0, 1)
    assert rc != 0 and b"restarts" in lib.nef_last_error()
    rc, _, _ = call(lib, shapes, [3], probs, 1, 0.0, 0.5, 1)
    assert rc != 0
    rc, _, _ = call(lib, shapes, [3], probs, 1, 1.0, 0.0, 1, tiles=-1)
    assert rc != 0 and b"batch_tiles" in lib.nef_last_error()


@pytest.mark.parametrize("tiles", [1, 3, 4096])
def test_batched_tiles_per_item(lib, tiles):
    """Work items of 1 and 3 column tiles (views of up to 66 tiles then split into
    many partials) and of 4096 (one item per row block): the fit still matches the
    FP64 oracle."""
    shapes = [(5, 7, 9), (70, 9, 66)]
    ranks = [3, 17]
    probs = problems(5, shapes, ranks, 1, 0.1)
    rc, work, _ = call(lib, shapes, ranks, probs, 1, 1.0, 0.0, 2, tiles=tiles)
    assert rc == 0, lib.nef_last_error()
    for p, ((I, J, K), R) in enumerate(zip(shapes, ranks)):
        m = OracleModel(MODEL, dict(i=I, j=J, k=K, r=R))
        y, mask, inits = probs[p]
        ref = m.fit(y.astype(np.float64), mask, [f.astype(np.float64) for f in inits[0]], 1.0, 0.0, 2)
        for q in range(3):
            assert np.linalg.norm(work[p][q] - ref[q]) / np.linalg.norm(ref[q]) < 1e-2, (tiles, p, q)


def test_batched_tune_leaves_factors(lib):
    """nef_fit_batched_tune returns one of its candidates, reports a time for each,
    and leaves the caller's factors as they were."""
    shapes = [(6, 10, 13), (30, 8, 20)]
    ranks = [4, 20]
    restarts = 2
    probs = problems(6, shapes, ranks, restarts, 0.1)
    n = len(shapes)
    sh = (ctypes.c_int64 * (3 * n))(*[d for t in shapes for d in t])
    rk = (ctypes.c_int64 * n)(*ranks)
    ys = (ctypes.c_void_p * n)(*[p[0].ctypes.data for p in probs])
    ms = (ctypes.c_void_p * n)(*[p[1].ctypes.data for p in probs])
    work = [[f.copy() for f in p[2][k]] for p in probs for k in range(restarts)]
    before = [[f.copy() for f in u] for u in work]
    fs = (ctypes.c_void_p * (3 * n * restarts))(*[f.ctypes.data for u in work for f in u])
    o = Opt()
    lib.nef_default_options(ctypes.byref(o))
    o.precision = NEF_BF16
    best = ctypes.c_int()
    times = (ctypes.c_double * 5)()
    rc = lib.nef_fit_batched_tune(n, sh, rk, ys, ms, fs, restarts, 1.0, 0.0, ctypes.byref(o), ctypes.byref(best),
                                  times)
    assert rc == 0, lib.nef_last_error()
    assert best.value in (16, 32, 64, 128, 256)
    assert all(t > 0 for t in times)
    for u, v in zip(work, before):
        for f, g in zip(u, v):
            assert np.array_equal(f, g)
