"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated per result):
  * NEF_FP64 sweeps: factors within 1e-9 relative (Frobenius) after the full run.
  * NEF_FP32 sweeps: factors within 1e-5 relative after one sweep; final loss
    within 1e-6 relative.
  * NEF_BF16 (tcgen05) passes: one factor update within 2e-3 relative; final
    loss within 1e-3 relative of the FP64 oracle started from the same point.
  * Layout probe: BF16 products with FP32 accumulation, 1e-5 relative to an
    FP64 product of the same BF16 values.
"""
import numpy as np
import pytest

import synth
from oracle import OracleModel

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


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def bf16_round(x):
    t = torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16)
    return t.to(torch.float32).numpy()


# ------------------------------------------------------------- layout probe

@pytest.mark.parametrize("a_in_tmem", [0, 1])
@pytest.mark.parametrize("bp", [16, 32, 64])
def test_tc_probe_layouts(bp, a_in_tmem):
    nef = _nef()
    rng = np.random.default_rng(bp)
    P = rng.uniform(0, 1, (128, bp)).astype(np.float32)
    Q = rng.uniform(0, 1, (64, bp)).astype(np.float32)
    W = rng.uniform(0, 1, (128, 64)).astype(np.float32)
    tP, tQ, tW = (torch.as_tensor(x).to("cuda").to(torch.bfloat16).contiguous() for x in (P, Q, W))
    D1 = torch.zeros(128, 64, device="cuda")
    D2 = torch.zeros(128, bp, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    lib = _probe()
    rc = lib.nef_tc_probe(bp, a_in_tmem, tP.data_ptr(), tQ.data_ptr(), tW.data_ptr(), D1.data_ptr(), D2.data_ptr(),
                          err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    Pb, Qb, Wb = (t.to(torch.float64).cpu().numpy() for t in (tP, tQ, tW))
    np.testing.assert_allclose(D1.cpu().numpy(), Pb @ Qb.T, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(D2.cpu().numpy(), Wb @ Qb, rtol=1e-5, atol=1e-5)


# ------------------------------------------------------------ config 1

@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_config1_full_fit(prec):
    """CP 30x40x50 R5, KL, 10% missing, 200 sweeps."""
    nef = _nef()
    p = synth.config1()
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    ref, trace = m.fit(p.y, p.mask, init, 1.0, 0.0, 200, trace=True)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = nef.Plan(p.model_str, p.dims, precision=prec)
    Y, M = dev(p.y, dt), dev(p.mask, torch.uint8)
    fs = [dev(f, dt) for f in init]
    plan.fit(Y, M, fs, 1.0, 0.0, 200)
    plan.check()
    out = [f.cpu().numpy() for f in fs]
    lo, cnt = plan.loss(Y, M, fs, 1.0, 0.0)
    assert cnt == int(p.mask.sum())
    if prec == "fp64":
        for a, b in zip(out, ref):
            assert rel(a, b) < 1e-9
        assert lo == pytest.approx(trace[-1], rel=1e-10)
    else:
        assert lo == pytest.approx(trace[-1], rel=1e-6)


def test_config1_fp32_one_sweep_factors():
    nef = _nef()
    p = synth.config1()
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    ref = m.fit(p.y, p.mask, init, 1.0, 0.0, 1)
    plan = nef.Plan(p.model_str, p.dims, precision="fp32")
    fs = [dev(f) for f in init]
    plan.fit(dev(p.y), dev(p.mask, torch.uint8), fs, 1.0, 0.0, 1)
    for a, b in zip(fs, ref):
        assert rel(a.cpu().numpy(), b) < 1e-5


# ---------------------------------------------------- model family, FP32/FP64

FAMILY = [
    ("ir,jr,kr->ijk", dict(i=37, j=70, k=129, r=7)),
    ("ia,ja,ab,kb,lb->ijkl", dict(i=9, j=70, k=13, l=20, a=5, b=3)),
    ("ir,js,kt,rst->ijk", dict(i=20, j=33, k=65, r=3, s=4, t=2)),
    ("iab,jbc,kca->ijk", dict(i=31, j=18, k=67, a=2, b=3, c=2)),
    ("ij,jk,ik->ijk", dict(i=17, j=23, k=29)),
    ("ir,jr,ak,kr,tr->ijat", dict(i=21, j=19, a=6, t=35, k=2, r=5)),
    ("wr,dr,hr,irk,jrk->wdhij", dict(w=3, d=7, h=6, i=10, j=12, r=3, k=2)),
]


@pytest.mark.parametrize("model_str,dims", FAMILY)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (0.5, 0.5), (1.0, -0.5)])
def test_family_two_sweeps(model_str, dims, prec, ab):
    nef = _nef()
    a, b = ab
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(abs(hash((model_str, prec, a, b))) % 2**32)
    init = [rng.uniform(0.3, 1.7, m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.poisson(np.einsum(model_str, *init) * 0.8).astype(np.float64)
    mask = (rng.random(m.y_shape) > 0.25).astype(np.uint8)
    ref = m.fit(y, mask, init, a, b, 2)
    dt = torch.float64 if prec == "fp64" else torch.float32
    plan = nef.Plan(model_str, dims, precision=prec)
    fs = [dev(f, dt) for f in init]
    plan.fit(dev(y, dt), dev(mask, torch.uint8), fs, a, b, 2)
    plan.check()
    tol = 1e-10 if prec == "fp64" else 5e-5
    for q in range(m.n_factors):
        assert rel(fs[q].cpu().numpy(), ref[q]) < tol, (q, plan.info())


@pytest.mark.parametrize("dims", [dict(i=8, j=8, k=2000), dict(i=5, j=300, k=7), dict(i=6, j=100, k=9)])
def test_generic_long_contractions_fp64(dims):
    """'ij,jk,ik->ijk' has no fused view: its numerators are einsums over the
    materialised weights with 2000, 300 or 100 free combinations per output (and
    7-9 for the other factors), which run on the grouped contraction kernels
    (256, 32 and 8 threads per output)."""
    nef = _nef()
    model_str = "ij,jk,ik->ijk"
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(21)
    init = [rng.uniform(0.3, 1.7, m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.poisson(np.einsum(model_str, *init)).astype(np.float64)
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8)
    ref = m.fit(y, mask, init, 1.0, 0.0, 2)
    plan = nef.Plan(model_str, dims, precision="fp64")
    assert "generic" in plan.info()
    fs = [dev(f, torch.float64) for f in init]
    plan.fit(dev(y, torch.float64), dev(mask, torch.uint8), fs, 1.0, 0.0, 2)
    plan.check()
    for q in range(m.n_factors):
        assert rel(fs[q].cpu().numpy(), ref[q]) < 1e-10


# ------------------------------------------------------ tensor-core path

TC_CASES = [
    # (model, dims, alpha, beta, masked)
    ("ir,jr,kr->ijk", dict(i=200, j=132, k=256, r=32), 1.0, 0.0, False),
    ("ir,jr,kr->ijk", dict(i=160, j=96, k=192, r=64), 1.0, -0.5, False),
    ("ir,jr,kr->ijk", dict(i=136, j=100, k=68, r=16), 1.0, 0.0, True),
    ("ia,ja,ab,kb,lb->ijkl", dict(i=32, j=40, k=16, l=8, a=16, b=8), 0.5, 0.5, True),
    ("ir,jr,kr->ijk", dict(i=96, j=64, k=128, r=20), 1.0, 1.0, False),
    ("wr,dr,hr,irk,jrk->wdhij", dict(w=9, d=7, h=8, i=30, j=40, r=5, k=3), 1.0, 0.0, True),
    ("ir,jr,ak,kr,tr->ijat", dict(i=60, j=50, a=20, t=40, r=8, k=3), 1.0, 0.0, False),
]


@pytest.mark.parametrize("model_str,dims,a,b,masked", TC_CASES)
def test_bf16_single_updates(model_str, dims, a, b, masked):
    nef = _nef()
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(7)
    truth = [rng.gamma(0.5, 1.0, m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.poisson(np.einsum(model_str, *truth)).astype(np.float32)
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8) if masked else None
    init = [rng.uniform(0.5, 1.5, m.factor_shape(l)) for l in range(m.n_factors)]
    plan = nef.Plan(model_str, dims, precision="bf16", profile=True)
    assert "generic" not in plan.info() and "simt" not in plan.info(), plan.info()
    Y = dev(y)
    M = None if mask is None else dev(mask, torch.uint8)
    for l in range(m.n_factors):
        ref, _, _ = m.update_factor(l, y, mask, init, a, b)
        fs = [dev(f) for f in init]
        plan.update(l, Y, M, fs, a, b)
        plan.check()
        got = fs[l].cpu().numpy()
        assert plan.profile()["tcgen05"][1] == 1, "the tensor-core pass did not run"
        assert np.all(np.isfinite(got))
        assert rel(got, ref[l]) < 2e-3, (l, rel(got, ref[l]), plan.info())


@pytest.mark.parametrize("model_str,dims,a,b,masked", TC_CASES[:4])
def test_bf16_fit_loss_matches_oracle(model_str, dims, a, b, masked):
    nef = _nef()
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(8)
    truth = [rng.gamma(0.5, 1.0, m.factor_shape(l)) for l in range(m.n_factors)]
    y = rng.poisson(np.einsum(model_str, *truth)).astype(np.float32)
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8) if masked else None
    init = [rng.uniform(0.5, 1.5, m.factor_shape(l)) for l in range(m.n_factors)]
    iters = 15
    ref, trace = m.fit(y, mask, init, a, b, iters, trace=True)
    plan = nef.Plan(model_str, dims, precision="bf16", profile=True)
    fs = [dev(f) for f in init]
    Y = dev(y)
    M = None if mask is None else dev(mask, torch.uint8)
    plan.fit(Y, M, fs, a, b, iters)
    plan.check()
    assert plan.profile()["tcgen05"][1] == iters * m.n_factors
    lo, _ = plan.loss(Y, M, fs, a, b)
    assert lo == pytest.approx(trace[-1], rel=1e-3)


# --------------------------------------------- full size, sampled outputs

@pytest.mark.parametrize("prec,beta", [("bf16", 0.0), ("fp32", 0.0), ("bf16", -0.5)])
def test_config2_sampled_update(prec, beta):
    """512^3 rank-64 CP in the launch configuration the benchmark times: one
    update of factor l per mode, checked on sampled rows against the oracle."""
    nef = _nef()
    p = synth.config2(beta=beta)
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    plan = nef.Plan(p.model_str, p.dims, precision=prec, profile=True)
    Y = dev(p.y)
    rng = np.random.default_rng(11)
    tol = 2e-3 if prec == "bf16" else 1e-5
    for l in range(3):
        fs = [dev(f) for f in init]
        plan.update(l, Y, None, fs, 1.0, beta)
        plan.check()
        kern = plan.profile()
        assert kern["tcgen05" if prec == "bf16" else "simt"][1] == 1
        got = fs[l].cpu().numpy()
        rows = rng.choice(512, size=2, replace=False)
        cols = rng.choice(64, size=4, replace=False)
        elems = np.array([r * 64 + c for r in rows for c in cols])
        num, den = m.numden_sampled(l, elems, p.y, None, init, 1.0, beta)
        eta = 1.0 if beta == 0.0 else 2.0 / 3.0
        expect = np.maximum(1e-10, init[l].reshape(-1)[elems] * (num / den) ** eta)
        np.testing.assert_allclose(got.reshape(-1)[elems], expect, rtol=tol)
        assert np.all(np.isfinite(got)) and np.all(got >= 1e-10)


def test_config3_sampled_update():
    """Custom 4-way model 'ia,ja,ab,kb,lb->ijkl' at 256x256x64x32 (a = 16, b = 8),
    (1/2, 1/2), 30 % missing, BF16, in the launch configuration the benchmark
    times: one update each of factors ia, ja (256-row views whose Q operand is the
    product of B or A with the contracted group sum_b C K L) and kb (a 2048-row
    transposed view), checked on sampled elements against the oracle."""
    nef = _nef()
    p = synth.config3()
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    plan = nef.Plan(p.model_str, p.dims, precision="bf16", profile=True)
    Y, M = dev(p.y), dev(p.mask, torch.uint8)
    rng = np.random.default_rng(12)
    for l in (0, 1, 3):
        fs = [dev(f) for f in init]
        plan.update(l, Y, M, fs, p.alpha, p.beta)
        plan.check()
        assert plan.profile(reset=True)["tcgen05"][1] == 1, plan.info()
        got = fs[l].cpu().numpy().reshape(-1)
        elems = rng.choice(got.size, size=2, replace=False)
        num, den = m.numden_sampled(l, elems, p.y, p.mask, init, p.alpha, p.beta)
        expect = m.apply_update(init[l].reshape(-1)[elems], num, den, p.alpha, p.beta)
        np.testing.assert_allclose(got[elems], expect, rtol=2e-3)
        assert np.all(np.isfinite(got)) and np.all(got >= 1e-10)


def test_uber_shape_sampled_update():
    """The Uber model 'wr,dr,hr,irk,jrk->wdhij' at the Uber tensor's shape
    27x7x24x100x100 (R = 10, K = 6), BF16: the dr update runs on the 4536-row
    view 'wdh' (a contracted epilogue), the irk update on the 10000-row view 'ij';
    sampled elements against the oracle."""
    nef = _nef()
    p = synth.config_uber()
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    plan = nef.Plan(p.model_str, p.dims, precision="bf16", profile=True)
    info = plan.info().splitlines()
    assert "rows='wdh'" in info[1] and "kernel=tcgen05" in info[1], info
    Y = dev(p.y)
    rng = np.random.default_rng(13)
    for l in (1, 3):
        fs = [dev(f) for f in init]
        plan.update(l, Y, None, fs, p.alpha, p.beta)
        plan.check()
        assert plan.profile(reset=True)["tcgen05"][1] == 1, plan.info()
        got = fs[l].cpu().numpy().reshape(-1)
        elems = rng.choice(got.size, size=2, replace=False)
        num, den = m.numden_sampled(l, elems, p.y, None, init, p.alpha, p.beta)
        expect = m.apply_update(init[l].reshape(-1)[elems], num, den, p.alpha, p.beta)
        np.testing.assert_allclose(got[elems], expect, rtol=2e-3)


def test_uber_mesh_update_matches_oracle_and_fp32():
    """The Uber model on a 200 x 200 pick-up mesh (27x7x24x200x200 = 181 M entries,
    a quarter of the paper's largest Uber mesh), BF16: one update of each factor from
    the same start, every element against the plain FP32 CUDA-core update (2e-3) and
    sampled elements against the FP64 oracle (2e-3)."""
    nef = _nef()
    p = synth.config_uber(dims=(27, 7, 24, 200, 200))
    m = OracleModel(p.model_str, p.dims)
    init = [f.astype(np.float64) for f in p.inits[0]]
    pb = nef.Plan(p.model_str, p.dims, precision="bf16")
    pf = nef.Plan(p.model_str, p.dims, precision="fp32")
    assert all("kernel=tcgen05" in ln for ln in pb.info().splitlines() if ln.startswith("factor")), pb.info()
    Y = dev(p.y)
    rng = np.random.default_rng(17)
    for l in range(5):
        fb = [dev(f) for f in init]
        ff = [dev(f) for f in init]
        pb.update(l, Y, None, fb, p.alpha, p.beta)
        pf.update(l, Y, None, ff, p.alpha, p.beta)
        pb.check()
        pf.check()
        gb = fb[l].cpu().numpy().reshape(-1)
        np.testing.assert_allclose(gb, ff[l].cpu().numpy().reshape(-1), rtol=2e-3)
        elems = rng.choice(gb.size, size=3, replace=False)
        num, den = m.numden_sampled(l, elems, p.y, None, init, p.alpha, p.beta)
        expect = m.apply_update(init[l].reshape(-1)[elems], num, den, p.alpha, p.beta)
        np.testing.assert_allclose(gb[elems], expect, rtol=2e-3)


# ------------------------------------------------------------------ autotune

def test_autotune_bf16_then_fit(tmp_path):
    """nef_plan_autotune picks a split per pass on the GPU, a second plan reads the
    same choices from the cache, and the tuned plan's fit still matches the FP64
    oracle's loss within 1e-3."""
    nef = _nef()
    model_str, dims = "ir,jr,kr->ijk", dict(i=256, j=160, k=288, r=32)
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(21)
    truth = [rng.gamma(0.5, 1.0, m.factor_shape(l)) for l in range(3)]
    y = rng.poisson(np.einsum(model_str, *truth)).astype(np.float32)
    init = [rng.uniform(0.5, 1.5, m.factor_shape(l)) for l in range(3)]
    Y = dev(y)
    cache = tmp_path / "splits.txt"
    plan = nef.Plan(model_str, dims, precision="bf16")
    splits = plan.autotune(Y, None, [dev(f) for f in init], 1.0, 0.0, cache=cache)
    assert all(s >= 1 for s in splits), splits
    plan2 = nef.Plan(model_str, dims, precision="bf16")
    assert plan2.autotune(Y, None, [dev(f) for f in init], 1.0, 0.0, cache=cache) == splits
    assert all("ring=" in ln for ln in plan.info().splitlines() if "kernel=tcgen05" in ln), plan.info()
    iters = 10
    _, trace = m.fit(y, None, init, 1.0, 0.0, iters, trace=True)
    fs = [dev(f) for f in init]
    plan.fit(Y, None, fs, 1.0, 0.0, iters)
    plan.check()
    lo, _ = plan.loss(Y, None, fs, 1.0, 0.0)
    assert lo == pytest.approx(trace[-1], rel=1e-3)
    # every tile configuration the tuner may choose (the deeper-ring instances and
    # the gathered Q path), forced through the cache, fits like the oracle
    lines = cache.read_text().strip().splitlines()
    for ring, gather in ((1, 0), (0, 1)):
        cache.write_text("".join(ln.split("\t")[0] + f"\t2 {ring} {gather}\n" for ln in lines))
        forced = nef.Plan(model_str, dims, precision="bf16", profile=True)
        forced.autotune(Y, None, [dev(f) for f in init], 1.0, 0.0, cache=cache)
        tc_lines = [ln for ln in forced.info().splitlines() if "kernel=tcgen05" in ln]
        # the deeper rings exist for staged Q rows; a pass with gathered rows keeps ring 0
        staged = [ln for ln in tc_lines if "q=staged" in ln]
        assert staged or gather, forced.info()
        assert all(f"ring={ring}" in ln for ln in staged), forced.info()
        assert all("ring=0" in ln for ln in tc_lines if "q=gathered" in ln), forced.info()
        if gather:
            assert all("q=gathered" in ln for ln in tc_lines), forced.info()
        fs = [dev(f) for f in init]
        forced.profile(reset=True)
        forced.fit(Y, None, fs, 1.0, 0.0, iters)
        forced.check()
        assert forced.profile(reset=True)["tcgen05"][1] >= iters
        lo, _ = forced.loss(Y, None, fs, 1.0, 0.0)
        assert lo == pytest.approx(trace[-1], rel=1e-3), (ring, gather)


def test_launch_count_of_a_recorded_sweep():
    """nef_plan_launches reports the kernels a sweep launched, as counted by the
    launchers: for the CP model on the tensor cores, three per factor update (fused
    pass, finish, column sums of the updated factor's copies)."""
    nef = _nef()
    model_str, dims = "ir,jr,kr->ijk", dict(i=256, j=160, k=288, r=32)
    rng = np.random.default_rng(5)
    y = rng.poisson(2.0, (256, 160, 288)).astype(np.float32)
    fs = [dev(rng.uniform(0.5, 1.5, (n, 32))) for n in (256, 160, 288)]
    plan = nef.Plan(model_str, dims, precision="bf16")
    plan.fit(dev(y), None, fs, 1.0, 0.0, 3)
    plan.check()
    assert plan.launches(False) == 9, plan.launches(False)
