"""Host logic of the C ABI (parser, planner, sweep driver) against the oracle.

plan.cpp is compiled with g++ against a fake CUDA runtime whose "device"
memory is host memory, with plain-loop launchers that implement each kernel
descriptor's documented meaning (tests/hostcheck).  This checks the planner's
views, strides, epilogue einsums, closed-form denominators and the generic
fallback on a CPU-only host; the kernels themselves are checked on the GPU.
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

NEF_FP32, NEF_BF16, NEF_FP64 = 0, 1, 2


# the options struct of include/nef.h, as the binding declares it (one layout for both)
from paper_2602_02759_gb300._nef import FitControl, Options as Opt  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    lib = ctypes.CDLL(hostcheck_build.build())
    vp = ctypes.c_void_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.nef_plan.argtypes = [ctypes.c_char_p, i64p, ctypes.c_int, i64p, ctypes.c_int,
                             ctypes.POINTER(Opt), ctypes.POINTER(vp)]
    lib.nef_fit.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                            ctypes.c_int]
    lib.nef_update.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(vp), ctypes.c_double,
                               ctypes.c_double]
    lib.nef_loss.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                             ctypes.POINTER(ctypes.c_double)]
    lib.nef_plan_destroy.argtypes = [vp]
    lib.nef_plan_info.argtypes = [vp, ctypes.c_char_p, ctypes.c_int]
    lib.nef_last_error.restype = ctypes.c_char_p
    lib.nef_default_options.argtypes = [ctypes.POINTER(Opt)]
    lib.nef_fit_ex.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_int)]
    lib.nef_fit_ctl.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, ctypes.POINTER(FitControl), ctypes.POINTER(ctypes.c_int)]
    lib.nef_plan_sweeps.argtypes = [vp]
    return lib


def split(model_str):
    lhs, rhs = model_str.split("->")
    lat = []
    for ch in lhs.replace(",", ""):
        if ch not in rhs and ch not in lat:
            lat.append(ch)
    return list(rhs), lat, lhs.split(",")


def make_plan(lib, model_str, dims, prec, force_generic=False, eps=1e-10, eager=False):
    obs, lat, _ = split(model_str)
    shapes = (ctypes.c_int64 * max(1, len(obs)))(*[dims[c] for c in obs])
    ranks = (ctypes.c_int64 * max(1, len(lat)))(*[dims[c] for c in lat])
    o = Opt()
    lib.nef_default_options(ctypes.byref(o))
    o.precision = prec
    o.eps = eps
    o.force_generic = int(force_generic)
    o.eager = int(eager)
    h = ctypes.c_void_p()
    rc = lib.nef_plan(model_str.encode(), shapes, len(obs), ranks, len(lat), ctypes.byref(o),
                      ctypes.byref(h))
    return rc, h


def info(lib, h):
    buf = ctypes.create_string_buffer(8192)
    lib.nef_plan_info(h, buf, 8192)
    return buf.value.decode()


def facs_arr(fs):
    arr = (ctypes.c_void_p * len(fs))()
    for k, f in enumerate(fs):
        arr[k] = f.ctypes.data
    return arr


MODELS = [
    ("ir,jr,kr->ijk", dict(i=5, j=6, k=7, r=3)),
    ("ir,jr->ij", dict(i=7, j=5, r=2)),
    ("ir,js,kt,rst->ijk", dict(i=4, j=3, k=5, r=2, s=3, t=2)),
    ("iab,jbc,kca->ijk", dict(i=3, j=4, k=3, a=2, b=2, c=3)),
    ("ia,ja,ab,kb,lb->ijkl", dict(i=4, j=3, k=5, l=3, a=3, b=2)),
    ("ij,jk,ik->ijk", dict(i=3, j=4, k=5)),
    ("i,jr,kr->ijk", dict(i=4, j=3, k=5, r=2)),
    ("ir,jkr->ijk", dict(i=4, j=3, k=5, r=3)),
    ("ir,jr,ak,kr,tr->ijat", dict(i=3, j=4, a=3, t=2, k=2, r=3)),
    ("wr,dr,hr,irk,jrk->wdhij", dict(w=2, d=3, h=2, i=3, j=4, r=2, k=2)),
    ("ri,jr,kr->ijk", dict(i=4, j=3, k=5, r=3)),
    ("ir,js,rs->ij", dict(i=5, j=4, r=2, s=3)),
    # large enough that the ia / ja passes take one-letter views whose Q operand
    # includes the contracted group sum_b C K L (an operand source of three factors)
    ("ia,ja,ab,kb,lb->ijkl", dict(i=12, j=12, k=8, l=8, a=3, b=2)),
]


@pytest.mark.parametrize("model_str,dims", MODELS)
@pytest.mark.parametrize("prec", [NEF_FP64, NEF_FP32])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.5, 0.5), (1.0, -0.5), (0.0, 1.0)])
@pytest.mark.parametrize("masked", [False, True])
def test_fit_matches_oracle(lib, model_str, dims, prec, ab, masked):
    a, b = ab
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(hash((model_str, a, b, masked)) % 2**32)
    dt = np.float64 if prec == NEF_FP64 else np.float32
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)).astype(dt) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape).astype(dt)
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8) if masked else None
    rc, h = make_plan(lib, model_str, dims, prec)
    assert rc == 0, lib.nef_last_error()
    try:
        ref = m.fit(y, mask, [f.astype(np.float64) for f in fs], a, b, 2)
        work = [f.copy() for f in fs]
        rc = lib.nef_fit(h, y.ctypes.data, None if mask is None else mask.ctypes.data,
                         facs_arr(work), a, b, 2)
        assert rc == 0, lib.nef_last_error()
        tol = 1e-10 if prec == NEF_FP64 else 2e-5
        for l in range(m.n_factors):
            rel = np.linalg.norm(work[l] - ref[l]) / np.linalg.norm(ref[l])
            assert rel < tol, (l, rel, info(lib, h))
        out = (ctypes.c_double * 2)()
        rc = lib.nef_loss(h, y.ctypes.data, None if mask is None else mask.ctypes.data,
                          facs_arr(work), a, b, out)
        assert rc == 0, lib.nef_last_error()
        lref, cnt = m.loss(y, mask, [w.astype(np.float64) for w in work], a, b)
        assert out[1] == cnt
        assert out[0] == pytest.approx(lref, rel=1e-9 if prec == NEF_FP64 else 1e-5)
    finally:
        lib.nef_plan_destroy(h)


@pytest.mark.parametrize("model_str,dims", MODELS[:5])
def test_generic_path_matches_oracle(lib, model_str, dims):
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(3)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape)
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8)
    rc, h = make_plan(lib, model_str, dims, NEF_FP64, force_generic=True)
    assert rc == 0
    try:
        assert "generic" in info(lib, h)
        ref = m.fit(y, mask, fs, 1.0, 0.0, 1)
        work = [f.copy() for f in fs]
        assert lib.nef_fit(h, y.ctypes.data, mask.ctypes.data, facs_arr(work), 1.0, 0.0, 1) == 0
        for l in range(m.n_factors):
            np.testing.assert_allclose(work[l], ref[l], rtol=1e-11)
    finally:
        lib.nef_plan_destroy(h)


def test_update_single_factor(lib):
    model_str, dims = "ia,ja,ab,kb,lb->ijkl", dict(i=4, j=3, k=5, l=3, a=3, b=2)
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(4)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape)
    rc, h = make_plan(lib, model_str, dims, NEF_FP64)
    try:
        for l in range(m.n_factors):
            ref, _, _ = m.update_factor(l, y, None, fs, 0.5, 0.5)
            work = [f.copy() for f in fs]
            assert lib.nef_update(h, l, y.ctypes.data, None, facs_arr(work), 0.5, 0.5) == 0
            for q in range(m.n_factors):
                np.testing.assert_allclose(work[q], ref[q], rtol=1e-12)
    finally:
        lib.nef_plan_destroy(h)


def test_planner_views(lib):
    """The chosen views for the benchmark shapes: CP uses one row letter per
    factor with gathered columns; the LR-core custom model uses bond b."""
    rc, h = make_plan(lib, "ir,jr,kr->ijk", dict(i=16, j=16, k=16, r=8), NEF_FP32)
    txt = info(lib, h)
    lib.nef_plan_destroy(h)
    assert txt.count("gather") == 3 and "generic" not in txt, txt
    rc, h = make_plan(lib, "ia,ja,ab,kb,lb->ijkl", dict(i=16, j=16, k=8, l=4, a=4, b=2), NEF_FP32)
    txt = info(lib, h)
    lib.nef_plan_destroy(h)
    assert "generic" not in txt, txt
    rc, h = make_plan(lib, "ij,jk,ik->ijk", dict(i=3, j=4, k=5), NEF_FP32)
    txt = info(lib, h)
    lib.nef_plan_destroy(h)
    assert txt.count("generic") == 3, txt


def test_planner_groups_and_row_padding(lib):
    """Column factors that share a letter outside the bond become one operand
    source (custom 4-way model: the ia pass runs on the 256-row view 'i' with
    Q = B o (sum_b C K L), not on the 65536-row view 'ij'), and views whose rows
    fill a small part of a tile lose to wider views (Uber shape: the dr pass runs
    on the 4536-row view 'wdh', not on the 7-row view 'd')."""
    rc, h = make_plan(lib, "ia,ja,ab,kb,lb->ijkl", dict(i=256, j=256, k=64, l=32, a=16, b=8), NEF_BF16)
    assert rc == 0, lib.nef_last_error()
    lines = info(lib, h).splitlines()
    lib.nef_plan_destroy(h)
    assert "rows='i' (256)" in lines[0] and "Q=gather(2)" in lines[0], lines
    assert "rows='j' (256)" in lines[1], lines
    rc, h = make_plan(lib, "wr,dr,hr,irk,jrk->wdhij", dict(w=27, d=7, h=24, i=100, j=100, r=10, k=6), NEF_BF16)
    assert rc == 0, lib.nef_last_error()
    lines = info(lib, h).splitlines()
    lib.nef_plan_destroy(h)
    assert all("rows='wdh' (4536)" in lines[q] for q in range(3)), lines
    # small problems keep the one-letter views (extra kernels would cost more than the padding)
    rc, h = make_plan(lib, "ir,jr,kr->ijk", dict(i=30, j=40, k=50, r=5), NEF_BF16)
    lines = info(lib, h).splitlines()
    lib.nef_plan_destroy(h)
    assert [ln.split("rows='")[1][0] for ln in lines] == ["i", "j", "k"], lines


def _random_model(rng):
    """A random valid model string: 2-3 observed letters, 1-3 latent letters,
    2-5 factors; every observed letter in one factor, every latent letter in
    1-3 factors (some factors get extra latent letters)."""
    obs = list("ijkl")[: rng.integers(2, 4)]
    lat = list("rstu")[: rng.integers(1, 4)]
    n_fac = int(rng.integers(2, 6))
    terms = [[] for _ in range(n_fac)]
    for x in obs:
        terms[int(rng.integers(n_fac))].append(x)
    for x in lat:
        for f in rng.choice(n_fac, size=int(rng.integers(1, min(3, n_fac) + 1)), replace=False):
            terms[int(f)].append(x)
    for f in range(n_fac):
        if lat and rng.random() < 0.3:
            x = lat[int(rng.integers(len(lat)))]
            if x not in terms[f]:
                terms[f].append(x)
        rng.shuffle(terms[f])
    terms = [tm for tm in terms if tm]
    dims = {x: int(rng.integers(2, 7)) for x in obs + lat}
    if rng.random() < 0.3:
        for x in obs:
            dims[x] = int(rng.integers(5, 13))
    return ",".join("".join(tm) for tm in terms) + "->" + "".join(obs), dims


@pytest.mark.parametrize("seed", range(60))
def test_random_models_match_oracle(lib, seed):
    """Planner generality: random model strings (views, bond choices, grouped
    operand sources, merged index terms, contracted epilogues, the generic
    fallback), one sweep with the FP64, FP32 and BF16 plans (the host double
    runs every view in FP32 on the plan's operand copies, which BF16 plans keep
    rounded to BF16: with a handful of entries nothing averages the roundings of
    the three or four operands of a product, 2^-9 each, so BF16 plans get 1e-2),
    with and without a mask."""
    rng = np.random.default_rng(1000 + seed)
    model_str, dims = _random_model(rng)
    m = OracleModel(model_str, dims)
    a, b = [(1.0, 0.0), (0.5, 0.5), (1.0, -0.5)][seed % 3]
    for prec in (NEF_FP64, NEF_FP32, NEF_BF16):
        for masked in (False, True):
            dt = np.float64 if prec == NEF_FP64 else np.float32
            fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)).astype(dt) for l in range(m.n_factors)]
            y = rng.uniform(0.2, 3.0, size=m.y_shape).astype(dt)
            mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8) if masked else None
            rc, h = make_plan(lib, model_str, dims, prec)
            assert rc == 0, (model_str, lib.nef_last_error())
            try:
                ref = m.fit(y.astype(np.float64), mask, [f.astype(np.float64) for f in fs], a, b, 1)
                work = [f.copy() for f in fs]
                rc = lib.nef_fit(h, y.ctypes.data, None if mask is None else mask.ctypes.data, facs_arr(work),
                                 a, b, 1)
                assert rc == 0, (model_str, lib.nef_last_error())
                tol = {NEF_FP64: 1e-9, NEF_FP32: 3e-5, NEF_BF16: 1e-2}[prec]
                for l in range(m.n_factors):
                    rel = np.linalg.norm(work[l] - ref[l]) / np.linalg.norm(ref[l])
                    assert rel < tol, (model_str, dims, prec, masked, l, rel, info(lib, h))
            finally:
                lib.nef_plan_destroy(h)


@pytest.mark.parametrize("prec", [NEF_FP64, NEF_FP32, NEF_BF16])
def test_edge_cases_match_oracle(lib, prec):
    """Degenerate inputs: size-1 modes, rank 1, Y with many exact zeros, a fully
    masked slice (its factor row keeps its value: den = 0), and zero sweeps."""
    cases = [("ir,jr,kr->ijk", dict(i=1, j=5, k=3, r=2)),
             ("ir,jr,kr->ijk", dict(i=6, j=1, k=1, r=3)),
             ("ir,jr->ij", dict(i=7, j=4, r=1)),
             ("ia,ja,ab,kb,lb->ijkl", dict(i=1, j=3, k=2, l=1, a=2, b=1))]
    dt = np.float64 if prec == NEF_FP64 else np.float32
    tol = {NEF_FP64: 1e-10, NEF_FP32: 3e-5, NEF_BF16: 1e-2}[prec]  # BF16 operand copies, no averaging
    for model_str, dims in cases:
        m = OracleModel(model_str, dims)
        rng = np.random.default_rng(7)
        fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)).astype(dt) for l in range(m.n_factors)]
        y = rng.poisson(0.3, size=m.y_shape).astype(dt)          # mostly exact zeros
        mask = np.ones(m.y_shape, np.uint8)
        mask[0] = 0                                               # slice 0 of the first mode unobserved
        rc, h = make_plan(lib, model_str, dims, prec)
        assert rc == 0, lib.nef_last_error()
        try:
            work = [f.copy() for f in fs]
            assert lib.nef_fit(h, y.ctypes.data, mask.ctypes.data, facs_arr(work), 1.0, 0.0, 0) == 0
            for l in range(m.n_factors):
                np.testing.assert_array_equal(work[l], fs[l])
            ref = m.fit(y.astype(np.float64), mask, [f.astype(np.float64) for f in fs], 1.0, 0.0, 2)
            assert lib.nef_fit(h, y.ctypes.data, mask.ctypes.data, facs_arr(work), 1.0, 0.0, 2) == 0
            for l in range(m.n_factors):
                rel = np.linalg.norm(work[l] - ref[l]) / np.linalg.norm(ref[l])
                assert rel < tol, (model_str, l, rel)
            # the first factor's rows for the unobserved slice keep their starting value
            if model_str.startswith("ir,") or model_str.startswith("ia,"):
                np.testing.assert_array_equal(work[0][0], fs[0][0])
        finally:
            lib.nef_plan_destroy(h)


@pytest.mark.parametrize("bad,code", [
    ("ir,jr,kr", 2), ("ir,jr->ii", 2), ("iir,jr->ij", 2), ("ir,jr->ijk", 2), ("iR,jr->ij", 2),
])
def test_parse_errors(lib, bad, code):
    shapes = (ctypes.c_int64 * 3)(2, 2, 2)
    ranks = (ctypes.c_int64 * 2)(2, 2)
    h = ctypes.c_void_p()
    rc = lib.nef_plan(bad.encode(), shapes, 2, ranks, 1, None, ctypes.byref(h))
    assert rc == code, (bad, rc, lib.nef_last_error())
    assert not h.value


def test_argument_errors(lib):
    rc, h = make_plan(lib, "ir,jr->ij", dict(i=3, j=3, r=2), NEF_FP32)
    assert rc == 0
    y = np.ones((3, 3), np.float32)
    fs = [np.ones((3, 2), np.float32), np.ones((3, 2), np.float32)]
    try:
        assert lib.nef_fit(h, y.ctypes.data, None, facs_arr(fs), 0.0, 0.5, 1) == 3  # unsupported
        assert lib.nef_fit(h, None, None, facs_arr(fs), 1.0, 0.0, 1) == 1
        assert lib.nef_fit(h, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0, -1) == 1
        assert lib.nef_update(h, 5, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0) == 1
    finally:
        lib.nef_plan_destroy(h)
    shapes = (ctypes.c_int64 * 2)(3, 0)
    ranks = (ctypes.c_int64 * 1)(2)
    hh = ctypes.c_void_p()
    assert lib.nef_plan(b"ir,jr->ij", shapes, 2, ranks, 1, None, ctypes.byref(hh)) == 1


# ----------------------------------------------- loss trace, tol, graph replay

@pytest.mark.parametrize("model_str,dims", [MODELS[0], MODELS[2], MODELS[4], MODELS[8]])
@pytest.mark.parametrize("masked", [False, True])
def test_loss_trace_and_graph_replay(lib, model_str, dims, masked):
    """Sweeps 2.. replayed from a captured sweep equal the eagerly launched ones
    exactly, and loss_trace[k] is the oracle's loss after k sweeps (Eq. 3.1)."""
    a, b = 1.0, 0.0
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(7)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape)
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8) if masked else None
    iters = 5
    _, ref_trace = m.fit(y, mask, [f.copy() for f in fs], a, b, iters, trace=True)
    outs = []
    for eager in (True, False):
        rc, h = make_plan(lib, model_str, dims, NEF_FP64, eager=eager)
        assert rc == 0, lib.nef_last_error()
        try:
            work = [f.copy() for f in fs]
            tr = np.full(iters + 1, np.nan)
            done = ctypes.c_int(0)
            for rep in range(2):  # the second call reuses the captured graph
                work = [f.copy() for f in fs]
                tr[:] = np.nan
                rc = lib.nef_fit_ex(h, y.ctypes.data, None if mask is None else mask.ctypes.data,
                                    facs_arr(work), a, b, iters, 0.0, tr.ctypes.data, ctypes.byref(done))
                assert rc == 0, lib.nef_last_error()
                assert done.value == iters
            outs.append(([w.copy() for w in work], tr.copy()))
        finally:
            lib.nef_plan_destroy(h)
    (w_e, tr_e), (w_g, tr_g) = outs
    for l in range(m.n_factors):
        assert np.array_equal(w_e[l], w_g[l]), l
    np.testing.assert_array_equal(tr_e, tr_g)
    np.testing.assert_allclose(tr_e, np.asarray(ref_trace[: iters + 1]), rtol=1e-10)


@pytest.mark.parametrize("tol", [0.5, 1e-2, 1e-9])
def test_tol_stops_after_small_decrease(lib, tol):
    """App. B's stopping rule: stop after the first sweep k >= 2 whose preceding
    relative decrease (L[k-2] - L[k-1]) / L[k-2] is below tol."""
    model_str, dims = MODELS[0]
    a, b = 1.0, 0.0
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(3)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape)
    iters = 12
    _, ref = m.fit(y, None, [f.copy() for f in fs], a, b, iters, trace=True)
    expect = iters
    for k in range(2, iters + 1):
        if (ref[k - 2] - ref[k - 1]) / ref[k - 2] < tol:
            expect = k
            break
    rc, h = make_plan(lib, model_str, dims, NEF_FP64)
    assert rc == 0
    try:
        work = [f.copy() for f in fs]
        tr = np.full(iters + 1, np.nan)
        done = ctypes.c_int(0)
        rc = lib.nef_fit_ex(h, y.ctypes.data, None, facs_arr(work), a, b, iters, tol, tr.ctypes.data,
                            ctypes.byref(done))
        assert rc == 0, lib.nef_last_error()
        assert done.value == expect
        np.testing.assert_allclose(tr[: expect + 1], np.asarray(ref[: expect + 1]), rtol=1e-10)
        assert np.all(np.isnan(tr[expect + 1:]))
        _, ref_f = None, m.fit(y, None, [f.copy() for f in fs], a, b, expect)
        for l in range(m.n_factors):
            assert np.linalg.norm(work[l] - ref_f[l]) / np.linalg.norm(ref_f[l]) < 1e-10
    finally:
        lib.nef_plan_destroy(h)


# ------------------------------------------------------------------ autotune

def test_autotune_cache_roundtrip(lib, tmp_path):
    """nef_plan_autotune writes one line per fused pass to its cache, reads it
    back on the next plan, and a fit with the cached (different) splits still
    matches the oracle."""
    vp = ctypes.c_void_p
    lib.nef_plan_autotune.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    model_str, dims = "ir,jr,kr->ijk", dict(i=40, j=36, k=300, r=3)
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(9)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.uniform(0.2, 3.0, size=m.y_shape)
    cache = tmp_path / "splits.txt"
    rc, h = make_plan(lib, model_str, dims, NEF_FP64)
    assert rc == 0
    out = (ctypes.c_int * 3)()
    try:
        rc = lib.nef_plan_autotune(h, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0, str(cache).encode(), out)
        assert rc == 0, lib.nef_last_error()
    finally:
        lib.nef_plan_destroy(h)
    first = list(out)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == sum(1 for s in first if s > 0) and all("\t" in ln for ln in lines)
    # rewrite every cached split to 2 and tune a fresh plan from the cache
    cache.write_text("".join(ln.rsplit("\t", 1)[0] + "\t2\n" for ln in lines))
    rc, h = make_plan(lib, model_str, dims, NEF_FP64)
    try:
        rc = lib.nef_plan_autotune(h, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0, str(cache).encode(), out)
        assert rc == 0, lib.nef_last_error()
        assert [s for s in out if s > 0] == [2] * len(lines)
        assert "splits=2" in info(lib, h)
        work = [f.copy() for f in fs]
        rc = lib.nef_fit(h, y.ctypes.data, None, facs_arr(work), 1.0, 0.0, 3)
        assert rc == 0, lib.nef_last_error()
        ref = m.fit(y, None, [f.copy() for f in fs], 1.0, 0.0, 3)
        for l in range(3):
            assert np.linalg.norm(work[l] - ref[l]) / np.linalg.norm(ref[l]) < 1e-10
    finally:
        lib.nef_plan_destroy(h)


LIK = {"negbin": 1, "binomial": 2, "js": 3}


def make_lik_plan(lib, model_str, dims, prec, kind, par):
    obs, lat, _ = split(model_str)
    shapes = (ctypes.c_int64 * max(1, len(obs)))(*[dims[c] for c in obs])
    ranks = (ctypes.c_int64 * max(1, len(lat)))(*[dims[c] for c in lat])
    o = Opt()
    lib.nef_default_options(ctypes.byref(o))
    o.precision = prec
    o.loss = LIK[kind]
    o.loss_par = par
    h = ctypes.c_void_p()
    rc = lib.nef_plan(model_str.encode(), shapes, len(obs), ranks, len(lat), ctypes.byref(o), ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("model_str,dims", [MODELS[0], MODELS[4], MODELS[5], MODELS[8]])
@pytest.mark.parametrize("prec", [NEF_FP64, NEF_FP32])
@pytest.mark.parametrize("kind,par", [("negbin", 2.5), ("binomial", 1.0), ("binomial", 6.0), ("js", 0.0)])
@pytest.mark.parametrize("masked", [False, True])
def test_likelihood_fit_matches_oracle(lib, model_str, dims, prec, kind, par, masked):
    """The likelihood families of App. B (negative binomial, binomial on the odds,
    Jensen-Shannon) through the planner and sweep driver: two sweeps and the loss
    against the oracle's or_lik_fit / or_lik_loss (the alpha, beta arguments are
    ignored by these families)."""
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(hash((model_str, kind, par, masked)) % 2**32)
    dt = np.float64 if prec == NEF_FP64 else np.float32
    fs = [rng.uniform(0.3, 1.2, size=m.factor_shape(l)).astype(dt) for l in range(m.n_factors)]
    if kind == "binomial":
        y = rng.integers(0, int(par) + 1, size=m.y_shape).astype(dt)
    else:
        y = rng.poisson(1.5, size=m.y_shape).astype(dt)
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8) if masked else None
    ntr = None if kind != "binomial" else np.full(m.y_shape, par)
    rc, h = make_lik_plan(lib, model_str, dims, prec, kind, par)
    assert rc == 0, lib.nef_last_error()
    try:
        ref = m.lik_fit(y, mask, [f.astype(np.float64) for f in fs], kind, 2, par=par, ntrials=ntr)
        work = [f.copy() for f in fs]
        rc = lib.nef_fit(h, y.ctypes.data, None if mask is None else mask.ctypes.data, facs_arr(work),
                         float("nan"), float("nan"), 2)
        assert rc == 0, lib.nef_last_error()
        tol = 1e-10 if prec == NEF_FP64 else 3e-5
        for l in range(m.n_factors):
            rel = np.linalg.norm(work[l] - ref[l]) / np.linalg.norm(ref[l])
            assert rel < tol, (l, rel, info(lib, h))
        out = (ctypes.c_double * 2)()
        assert lib.nef_loss(h, y.ctypes.data, None if mask is None else mask.ctypes.data, facs_arr(work),
                            0.0, 0.0, out) == 0, lib.nef_last_error()
        lref, cnt = m.lik_loss(y, mask, [w.astype(np.float64) for w in work], kind, par=par, ntrials=ntr)
        assert out[1] == cnt
        assert out[0] == pytest.approx(lref, rel=1e-9 if prec == NEF_FP64 else 1e-5)
    finally:
        lib.nef_plan_destroy(h)


def test_likelihood_plan_argument_checks(lib):
    """A dispersion or trial count outside (0, inf) and an unknown family are
    rejected at plan time; the (alpha, beta) family still checks its arguments."""
    for kind, par in (("negbin", 0.0), ("negbin", -1.0), ("binomial", 0.0), ("binomial", float("inf"))):
        rc, h = make_lik_plan(lib, "ir,jr,kr->ijk", dict(i=3, j=3, k=3, r=2), NEF_FP64, kind, par)
        assert rc == 1 and not h.value, (kind, par)
    o = Opt()
    lib.nef_default_options(ctypes.byref(o))
    assert o.loss == 0 and o.loss_par == 0.0 and o.wait_cycles == 0
    o.loss = 9
    h = ctypes.c_void_p()
    shapes = (ctypes.c_int64 * 3)(3, 3, 3)
    ranks = (ctypes.c_int64 * 1)(2)
    assert lib.nef_plan(b"ir,jr,kr->ijk", shapes, 3, ranks, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    o.loss = 0
    o.wait_cycles = -1
    assert lib.nef_plan(b"ir,jr,kr->ijk", shapes, 3, ranks, 1, ctypes.byref(o), ctypes.byref(h)) == 1
    rc, h = make_plan(lib, "ir,jr,kr->ijk", dict(i=3, j=3, k=3, r=2), NEF_FP64)
    try:
        y = np.ones((3, 3, 3))
        fs = [np.ones((3, 2)) for _ in range(3)]
        assert lib.nef_fit(h, y.ctypes.data, None, facs_arr(fs), float("nan"), 0.0, 1) == 1
        assert lib.nef_fit(h, y.ctypes.data, None, facs_arr(fs), 0.0, 0.5, 1) == 3
    finally:
        lib.nef_plan_destroy(h)


# ------------------------------------------- stopping rules evaluated on the device

def _oracle_traces(m, y, train, val, init, a, b, iters):
    """The oracle's training loss L[k] (over the training mask) and validation loss
    V[k] (over the validation mask) after k = 0..iters sweeps, one sweep at a time."""
    fs = [f.astype(np.float64) for f in init]
    L, V = [m.loss(y, train, fs, a, b)[0]], [m.loss(y, val, fs, a, b)[0]]
    for _ in range(iters):
        fs = m.fit(y, train, fs, a, b, 1)
        L.append(m.loss(y, train, fs, a, b)[0])
        V.append(m.loss(y, val, fs, a, b)[0])
    return np.array(L), np.array(V)


def _stop_tol(L, tol, iters):
    """Sweeps run under App. B's training-loss rule: stop after the first sweep k >= 2
    with (L[k-2] - L[k-1]) / L[k-2] < tol."""
    for k in range(2, iters + 1):
        if (L[k - 2] - L[k - 1]) / L[k - 2] < tol:
            return k
    return iters


def _stop_val(V, patience, iters):
    """Sweeps run under App. B's validation rule: stop after the sweep k at which
    V rose for the patience-th consecutive time."""
    rises = 0
    for k in range(1, iters + 1):
        rises = rises + 1 if V[k] > V[k - 1] else 0
        if rises >= patience:
            return k
    return iters


def _overfit_problem(seed=41):
    """A CP model of rank 6 on a small noisy Poisson tensor with half of the entries
    held out: the training loss keeps falling while the validation loss turns up."""
    model_str, dims = "ir,jr,kr->ijk", dict(i=9, j=8, k=10, r=6)
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(seed)
    truth = [rng.gamma(2.0, 0.5, m.factor_shape(l)) for l in range(3)]
    y = rng.poisson(np.einsum(model_str, *truth) * 0.3).astype(np.float64)
    u = rng.random(m.y_shape)
    train = (u < 0.5).astype(np.uint8)
    val = (u >= 0.5).astype(np.uint8)
    init = [rng.uniform(0.5, 1.5, m.factor_shape(l)) for l in range(3)]
    return model_str, dims, m, y, train, val, init


@pytest.mark.parametrize("eager", [False, True])
def test_device_stopping_rules_match_oracle(lib, eager):
    """The tol rule and the validation-loss rule of App. B, run by the check kernel
    inside the sweep loop (a conditional graph loop, or read back per sweep with
    eager launches), stop at the sweep the oracle's FP64 traces predict; the loss
    traces match the oracle's, and entries past the stop stay untouched."""
    model_str, dims, m, y, train, val, init = _overfit_problem()
    iters = 60
    L, V = _oracle_traces(m, y, train, val, init, 1.0, 0.0, iters)
    tol = 3e-3
    k_tol = _stop_tol(L, tol, iters)
    k_val = _stop_val(V, 5, iters)
    assert 2 < k_tol < iters and 5 < k_val < iters, (k_tol, k_val)
    for mode, want in (("tol", k_tol), ("val", k_val), ("both", min(k_tol, k_val))):
        rc, h = make_plan(lib, model_str, dims, NEF_FP64, eager=eager)
        assert rc == 0
        try:
            work = [f.copy() for f in init]
            lt = np.full(iters + 1, np.nan)
            vt = np.full(iters + 1, np.nan)
            c = FitControl(tol if mode != "val" else 0.0, lt.ctypes.data, val.ctypes.data,
                           5 if mode != "tol" else 0, vt.ctypes.data)
            done = ctypes.c_int(0)
            rc = lib.nef_fit_ctl(h, y.ctypes.data, train.ctypes.data, facs_arr(work), 1.0, 0.0, iters,
                                 ctypes.byref(c), ctypes.byref(done))
            assert rc == 0, lib.nef_last_error()
            assert done.value == want == lib.nef_plan_sweeps(h), (mode, done.value, want)
            np.testing.assert_allclose(lt[: want + 1], L[: want + 1], rtol=1e-10)
            np.testing.assert_allclose(vt[: want + 1], V[: want + 1], rtol=1e-10)
            assert np.all(np.isnan(lt[want + 1:])) and np.all(np.isnan(vt[want + 1:]))
            ref = m.fit(y, train, [f.astype(np.float64) for f in init], 1.0, 0.0, want)
            for q in range(3):
                np.testing.assert_allclose(work[q], ref[q], rtol=1e-10)
        finally:
            lib.nef_plan_destroy(h)


def test_fit_ctl_argument_checks(lib):
    rc, h = make_plan(lib, "ir,jr,kr->ijk", dict(i=3, j=3, k=3, r=2), NEF_FP64)
    try:
        y = np.ones((3, 3, 3))
        fs = [np.ones((3, 2)) for _ in range(3)]
        vm = np.ones((3, 3, 3), np.uint8)
        for c in (FitControl(-1.0, None, None, 0, None), FitControl(0.0, None, None, 3, None),
                  FitControl(0.0, None, None, 0, vm.ctypes.data), FitControl(0.0, None, vm.ctypes.data, -1, None)):
            assert lib.nef_fit_ctl(h, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0, 2, ctypes.byref(c), None) == 1
        assert lib.nef_fit_ctl(h, y.ctypes.data, None, facs_arr(fs), 1.0, 0.0, 2, None, None) == 0
        assert lib.nef_plan_sweeps(h) == 2
    finally:
        lib.nef_plan_destroy(h)
