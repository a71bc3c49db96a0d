"""Pins of the oracle's likelihood losses of App. B (negative binomial,
binomial / Bernoulli on odds, Jensen-Shannon) against library routines and
theorems, not against themselves:
  * the loss differences equal the negative log-likelihood differences of
    scipy.stats.nbinom / scipy.stats.binom (the dropped terms are constant in
    the mean), and Jensen-Shannon equals half the relative entropies to the
    midpoint (scipy.special.rel_entr);
  * the loss does not increase after any factor update (the MM argument of
    Thm. 3.1 applies to every convex-concave split);
  * calculus: num - den = -grad L for the two likelihoods (c = 1, g = id) and
    num = -2 grad L for Jensen-Shannon (c = 1/2, b = 1), by central differences;
  * limits and special cases: the negative binomial update tends to the KL
    update as phi grows; n = 1 everywhere is the Bernoulli default; a model
    whose reconstruction equals the data (for the binomial: n times the
    success probability) is a fixed point.
"""
import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")
scipy_special = pytest.importorskip("scipy.special")

import oracle  # noqa: E402
from oracle import OracleModel  # noqa: E402

MODELS = [
    ("ir,jr,kr->ijk", dict(i=3, j=4, k=5, r=2)),
    ("ir,jr->ij", dict(i=5, j=4, r=3)),
    ("ia,ja,ab,kb,lb->ijkl", dict(i=3, j=2, k=3, l=2, a=2, b=2)),
    ("ir,js,kt,rst->ijk", dict(i=3, j=2, k=3, r=2, s=2, t=2)),
]
KINDS = [("negbin", 2.5), ("binomial", 0.0), ("js", 0.0)]


def _data(m, rng, kind):
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    ntr = None
    if kind == "binomial":
        ntr = rng.integers(1, 6, size=m.y_shape).astype(np.float64)
        y = np.floor(rng.uniform(0, 1, size=m.y_shape) * (ntr + 1))
    elif kind == "negbin":
        y = rng.poisson(2.0, size=m.y_shape).astype(np.float64)
    else:
        y = rng.uniform(0.0, 3.0, size=m.y_shape)
        y[rng.random(m.y_shape) < 0.2] = 0.0
    return fs, y, ntr


def test_negbin_matches_scipy_loglik_differences():
    rng = np.random.default_rng(0)
    for phi in (0.5, 1.0, 4.0):
        for _ in range(20):
            x = float(rng.integers(0, 12))
            y1, y2 = rng.uniform(0.1, 8.0, size=2)
            d = oracle.lik_divergence("negbin", x, y1, phi) - oracle.lik_divergence("negbin", x, y2, phi)
            nll = (-scipy_stats.nbinom.logpmf(x, phi, phi / (phi + y1))
                   + scipy_stats.nbinom.logpmf(x, phi, phi / (phi + y2)))
            assert d == pytest.approx(nll, rel=1e-10, abs=1e-10)


def test_binomial_matches_scipy_loglik_differences():
    rng = np.random.default_rng(1)
    for _ in range(40):
        n = float(rng.integers(1, 10))
        x = float(rng.integers(0, n + 1))
        m1, m2 = rng.uniform(0.05, 6.0, size=2)  # odds
        d = oracle.lik_divergence("binomial", x, m1, 0.0, n) - oracle.lik_divergence("binomial", x, m2, 0.0, n)
        nll = (-scipy_stats.binom.logpmf(x, n, m1 / (1 + m1)) + scipy_stats.binom.logpmf(x, n, m2 / (1 + m2)))
        assert d == pytest.approx(nll, rel=1e-10, abs=1e-10)


def test_js_is_half_relative_entropy_to_midpoint():
    rng = np.random.default_rng(2)
    for _ in range(40):
        x, y = rng.uniform(0.0, 5.0, size=2)
        if rng.random() < 0.2:
            x = 0.0
        mid = 0.5 * (x + y)
        ref = 0.5 * (scipy_special.rel_entr(x, mid) + scipy_special.rel_entr(y, mid))
        assert oracle.lik_divergence("js", x, y) == pytest.approx(ref, rel=1e-12, abs=1e-14)
        assert oracle.lik_divergence("js", x, y) == pytest.approx(oracle.lik_divergence("js", y, x), rel=1e-12)


@pytest.mark.parametrize("model_str,dims", MODELS)
@pytest.mark.parametrize("kind,par", KINDS)
def test_monotone_every_factor_update(model_str, dims, kind, par):
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(hash((model_str, kind)) % 2**32)
    fs, y, ntr = _data(m, rng, kind)
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8)
    prev = m.lik_loss(y, mask, fs, kind, par, ntr)[0]
    for _ in range(3):
        for l in range(m.n_factors):
            fs, _, _ = m.lik_update_factor(l, y, mask, fs, kind, par, ntr)
            cur = m.lik_loss(y, mask, fs, kind, par, ntr)[0]
            assert cur <= prev + 1e-10 * abs(prev), (kind, l, prev, cur)
            prev = cur


@pytest.mark.parametrize("model_str,dims", MODELS[:3])
@pytest.mark.parametrize("kind,par", KINDS)
def test_numden_against_finite_differences(model_str, dims, kind, par):
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(5)
    fs, y, ntr = _data(m, rng, kind)
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8)
    h = 1e-6
    for l in range(m.n_factors):
        _, num, den = m.lik_update_factor(l, y, mask, fs, kind, par, ntr)
        grad = np.empty(m.factor_shape(l))
        for e in range(grad.size):
            fp = [f.copy() for f in fs]
            fm = [f.copy() for f in fs]
            fp[l].reshape(-1)[e] += h
            fm[l].reshape(-1)[e] -= h
            grad.reshape(-1)[e] = (m.lik_loss(y, mask, fp, kind, par, ntr)[0]
                                   - m.lik_loss(y, mask, fm, kind, par, ntr)[0]) / (2 * h)
        lhs = num if kind == "js" else num - den
        rhs = -2.0 * grad if kind == "js" else -grad
        np.testing.assert_allclose(lhs, rhs, rtol=1e-5, atol=1e-6 * np.abs(rhs).max())


def test_negbin_tends_to_kl():
    m = OracleModel("ir,jr,kr->ijk", dict(i=3, j=4, k=5, r=2))
    rng = np.random.default_rng(6)
    fs, y, _ = _data(m, rng, "negbin")
    for l in range(3):
        nb, _, _ = m.lik_update_factor(l, y, None, fs, "negbin", 1e9)
        kl, _, _ = m.update_factor(l, y, None, fs, 1.0, 0.0)
        np.testing.assert_allclose(nb[l], kl[l], rtol=1e-7)


def test_bernoulli_is_binomial_with_one_trial():
    m = OracleModel("ir,jr->ij", dict(i=6, j=5, r=2))
    rng = np.random.default_rng(7)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(2)]
    y = (rng.random(m.y_shape) < 0.4).astype(np.float64)
    a = m.lik_fit(y, None, fs, "binomial", 3)
    b = m.lik_fit(y, None, fs, "binomial", 3, ntrials=np.ones(m.y_shape))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("kind,par", KINDS)
def test_exact_fit_is_fixed_point(kind, par):
    m = OracleModel("ia,ja,ab,kb,lb->ijkl", dict(i=3, j=2, k=3, l=2, a=2, b=2))
    rng = np.random.default_rng(8)
    fs = [rng.uniform(0.3, 1.7, size=m.factor_shape(l)) for l in range(m.n_factors)]
    yhat = m.reconstruct(fs)
    ntr = None
    if kind == "binomial":
        ntr = rng.integers(1, 6, size=m.y_shape).astype(np.float64)
        y = ntr * yhat / (1.0 + yhat)      # n times the success probability of the odds yhat
    else:
        y = yhat
    out = m.lik_fit(y, None, fs, kind, 2, par, ntr)
    for u, v in zip(out, fs):
        np.testing.assert_allclose(u, v, rtol=1e-10)
