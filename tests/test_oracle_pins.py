"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these compare the oracle with itself: each checks it against a
library routine (numpy.einsum), a textbook update (Lee-Seung NMF), a closed
form (the named divergences, hand-evaluated in tests/golden/), a theorem of
the paper (monotone loss, Thm. 3.1 / Thm. 4.3) or calculus (central finite
differences of the loss against num - den).  A plausible slip in the oracle
(a dropped term, a wrong exponent, a transposed operand, a wrong mask use)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import OracleModel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

MODELS = [
    # (model string, dims) -- tiny shapes covering the paper's model family (Sec. 2)
    ("ir,jr,kr->ijk", dict(i=2, j=3, k=4, r=3)),                          # CP
    ("ir,jr->ij", dict(i=4, j=5, r=2)),                                   # NMF
    ("ir,js,kt,rst->ijk", dict(i=3, j=2, k=4, r=2, s=3, t=2)),            # Tucker
    ("iab,jbc,kca->ijk", dict(i=3, j=2, k=3, a=1, b=2, c=3)),             # tensor train
    ("ia,ja,ab,kb,lb->ijkl", dict(i=3, j=2, k=4, l=5, a=2, b=3)),         # LR core custom
    ("ij,jk,ik->ijk", dict(i=2, j=3, k=4)),                               # many-body
    ("i,jr,kr->ijk", dict(i=3, j=2, k=4, r=2)),                           # factor without latent
    ("ir,jkr->ijk", dict(i=3, j=2, k=4, r=2)),                            # two-mode factor
    ("ir,jr,ak,kr,tr->ijat", dict(i=2, j=3, a=3, t=2, k=2, r=3)),         # ICEWS-shaped custom
]

AB_PAIRS = [(1.0, 0.0), (1.0, 1.0), (1.0, -1.0), (0.5, 0.5), (1.0, -0.5), (2.0, -1.0),
            (0.0, 1.0), (1.3, 0.0), (0.7, 1.0), (1.2, -0.5), (0.8, 0.0)]


def _rand_factors(m, rng, lo=0.3, hi=1.7):
    return [rng.uniform(lo, hi, size=m.factor_shape(l)) for l in range(m.n_factors)]


def _rand_data(m, rng, kind="poisson"):
    if kind == "poisson":
        y = rng.poisson(2.0, size=m.y_shape).astype(np.float64)
        y[y == 0] = 0.0
        return y
    return rng.uniform(0.2, 3.0, size=m.y_shape)


# ------------------------------------------------------------ contraction pins

@pytest.mark.parametrize("model_str,dims", MODELS)
def test_reconstruct_matches_numpy_einsum(model_str, dims):
    """Eq. 2.1 loop nest vs numpy.einsum (a library routine)."""
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(1)
    f = _rand_factors(m, rng)
    np.testing.assert_allclose(m.reconstruct(f), np.einsum(model_str, *f), rtol=1e-13)


@pytest.mark.parametrize("model_str,dims", MODELS)
def test_einstr_matches_numpy_einsum(model_str, dims):
    """Eq. 3.8 loop nest vs numpy.einsum of swap(model_str, l) built here."""
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(2)
    f = _rand_factors(m, rng)
    T = rng.uniform(-1, 1, size=m.y_shape)
    lhs, rhs = model_str.split("->")
    terms = lhs.split(",")
    for l in range(len(terms)):
        swapped = ",".join(rhs if q == l else t for q, t in enumerate(terms)) + "->" + terms[l]
        assert m.einstr(l) == swapped
        ops = [T if q == l else f[q] for q in range(len(terms))]
        np.testing.assert_allclose(m.einstr_contract(l, T, f), np.einsum(swapped, *ops),
                                   rtol=1e-12, atol=1e-13)


def test_cp_reconstruct_closed_form():
    """CP (Eq. 2.4) written as an explicit triple loop."""
    m = OracleModel("ir,jr,kr->ijk", dict(i=2, j=3, k=4, r=3))
    rng = np.random.default_rng(3)
    A, B, C = _rand_factors(m, rng)
    yh = m.reconstruct([A, B, C])
    for i in range(2):
        for j in range(3):
            for k in range(4):
                ref = sum(A[i, r] * B[j, r] * C[k, r] for r in range(3))
                assert abs(yh[i, j, k] - ref) < 1e-14


def test_relabel_invariance():
    rng = np.random.default_rng(4)
    m1 = OracleModel("ir,jr,kr->ijk", dict(i=3, j=4, k=2, r=2))
    m2 = OracleModel("xz,yz,wz->xyw", dict(x=3, y=4, w=2, z=2))
    f = _rand_factors(m1, rng)
    y = _rand_data(m1, rng)
    for l in range(3):
        a, _, _ = m1.update_factor(l, y, None, f, 1.0, 0.0)
        b, _, _ = m2.update_factor(l, y, None, f, 1.0, 0.0)
        for u, v in zip(a, b):
            np.testing.assert_array_equal(u, v)


# ---------------------------------------------------------- textbook reductions

def test_lee_seung_euclidean():
    """'ir,jr->ij' with (1,1) is Lee-Seung's Euclidean NMF update:
    H <- H * (W^T X) / (W^T W H), here with Theta2 = H^T."""
    rng = np.random.default_rng(5)
    I, J, R = 6, 7, 3
    m = OracleModel("ir,jr->ij", dict(i=I, j=J, r=R))
    W = rng.uniform(0.2, 1.5, size=(I, R))
    Ht = rng.uniform(0.2, 1.5, size=(J, R))
    X = rng.uniform(0.0, 3.0, size=(I, J))
    new, _, _ = m.update_factor(1, X, None, [W, Ht], 1.0, 1.0, eps=0.0)
    H = Ht.T
    ref = H * (W.T @ X) / (W.T @ W @ H)
    np.testing.assert_allclose(new[1], ref.T, rtol=1e-12)
    new0, _, _ = m.update_factor(0, X, None, [W, Ht], 1.0, 1.0, eps=0.0)
    refW = W * (X @ H.T) / (W @ H @ H.T)
    np.testing.assert_allclose(new0[0], refW, rtol=1e-12)


def test_lee_seung_kl():
    """'ir,jr->ij' with (1,0) is Lee-Seung's KL NMF update:
    H_rj <- H_rj * sum_i W_ir X_ij/(WH)_ij / sum_i W_ir."""
    rng = np.random.default_rng(6)
    I, J, R = 5, 8, 2
    m = OracleModel("ir,jr->ij", dict(i=I, j=J, r=R))
    W = rng.uniform(0.2, 1.5, size=(I, R))
    Ht = rng.uniform(0.2, 1.5, size=(J, R))
    X = rng.poisson(2.0, size=(I, J)).astype(float)
    new, _, _ = m.update_factor(1, X, None, [W, Ht], 1.0, 0.0, eps=0.0)
    H = Ht.T
    WH = W @ H
    ref = H * (W.T @ (X / WH)) / W.sum(axis=0)[:, None]
    np.testing.assert_allclose(new[1], ref.T, rtol=1e-12)


@pytest.mark.parametrize("beta_c", [-1.0, 0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0])
def test_eta_matches_beta_divergence_mm_exponent(beta_c):
    """At alpha = 1 the App. B g-table must give the MM exponent of the
    beta-divergence MU (Fevotte & Idier 2011): 1/(2-b) for b < 1, 1 for
    1 <= b <= 2, 1/(b-1) for b > 2, where b = beta + 1 is their index."""
    if beta_c < 1:
        ref = 1.0 / (2.0 - beta_c)
    elif beta_c <= 2:
        ref = 1.0
    else:
        ref = 1.0 / (beta_c - 1.0)
    assert oracle.eta_of(1.0, beta_c - 1.0) == pytest.approx(ref, rel=1e-15)
    assert oracle.ginv(2.0, 1.0, beta_c - 1.0) == pytest.approx(2.0 ** ref, rel=1e-14)


def test_ginv_log_case():
    """alpha = 0, beta = 1: g = log, so g^{-1} = exp."""
    assert oracle.ginv(0.3, 0.0, 1.0) == pytest.approx(math.exp(0.3), rel=1e-15)


# ------------------------------------------------------------- divergence pins

def test_divergence_golden():
    rows = []
    with open(os.path.join(GOLDEN, "divergence_cases.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    assert len(rows) >= 10
    for a, b, x, y, ref in rows:
        assert oracle.divergence(x, y, a, b) == pytest.approx(ref, rel=1e-13, abs=1e-15), (a, b, x, y)


def test_divergence_continuity_in_beta():
    for x, y in [(2.0, 1.0), (0.5, 3.0)]:
        d0 = oracle.divergence(x, y, 1.0, 0.0)
        for b in (1e-7, -1e-7):
            assert oracle.divergence(x, y, 1.0, b) == pytest.approx(d0, rel=1e-5)


def test_divergence_zero_at_equality_and_nonnegative():
    rng = np.random.default_rng(7)
    for a, b in AB_PAIRS + [(0.0, 0.0), (-1.0, 2.0)]:
        for _ in range(20):
            x, y = rng.uniform(0.1, 5.0, size=2)
            assert oracle.divergence(x, x, a, b) == pytest.approx(0.0, abs=1e-12)
            assert oracle.divergence(x, y, a, b) >= -1e-12


def test_unsupported_alpha_zero():
    m = OracleModel("ir,jr->ij", dict(i=2, j=2, r=1))
    f = [np.ones((2, 1)), np.ones((2, 1))]
    with pytest.raises(ValueError):
        m.update_factor(0, np.ones((2, 2)), None, f, 0.0, 0.5)


# --------------------------------------------------------------- theory pins

def _loss(m, y, mask, f, a, b):
    return m.loss(y, mask, f, a, b)[0]


@pytest.mark.parametrize("model_str,dims", MODELS)
@pytest.mark.parametrize("ab", AB_PAIRS)
def test_monotone_every_factor_update(model_str, dims, ab):
    """Thm. 3.1 / Thm. 4.3: the loss never increases after any factor update."""
    a, b = ab
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(8)
    f = _rand_factors(m, rng)
    y = _rand_data(m, rng, "poisson" if a >= 1.0 or b <= 0 else "uniform")
    if a == 0.0:  # reverse KL needs x > 0 for log(x / y)
        y = _rand_data(m, rng, "uniform")
    mask = (rng.random(m.y_shape) > 0.2).astype(np.uint8)
    prev = _loss(m, y, mask, f, a, b)
    for sweep in range(4):
        for l in range(m.n_factors):
            f, _, _ = m.update_factor(l, y, mask, f, a, b)
            cur = _loss(m, y, mask, f, a, b)
            assert cur <= prev * (1 + 1e-12) + 1e-12, (sweep, l, prev, cur)
            prev = cur


@pytest.mark.parametrize("model_str,dims", MODELS[:6])
@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.0, 1.0), (0.5, 0.5), (1.0, -0.5), (2.0, -1.0),
                                (0.0, 1.0), (1.3, 0.0)])
def test_num_minus_den_is_scaled_negative_gradient(model_str, dims, ab):
    """Eq. 3.3 at lambda = 1 gives dD/dy = c(1) [g(1) b - a].  For the
    (alpha,beta)-divergence with alpha != 0: c(1) = 1/alpha and g(1) = 1, so
    num - den = -alpha dL/dtheta; for (0,1): g = log, g(1) = 0 and c = 1, so
    num = -dL/dtheta.  Checked by central finite differences of the masked loss."""
    a, b = ab
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(9)
    f = _rand_factors(m, rng)
    y = _rand_data(m, rng, "uniform")
    mask = (rng.random(m.y_shape) > 0.25).astype(np.uint8)
    for l in range(m.n_factors):
        _, num, den = m.update_factor(l, y, mask, f, a, b)
        g = np.zeros_like(f[l])
        flat = f[l].reshape(-1)
        for e in range(flat.size):
            h = 1e-6 * max(1.0, abs(flat[e]))
            fp = [x.copy() for x in f]
            fm = [x.copy() for x in f]
            fp[l].reshape(-1)[e] += h
            fm[l].reshape(-1)[e] -= h
            g.reshape(-1)[e] = (_loss(m, y, mask, fp, a, b) - _loss(m, y, mask, fm, a, b)) / (2 * h)
        if a != 0.0:
            np.testing.assert_allclose(num - den, -a * g, rtol=1e-6, atol=1e-7)
        else:
            np.testing.assert_allclose(num, -g, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("model_str,dims", MODELS)
@pytest.mark.parametrize("ab", [(1.0, 0.0), (1.0, 1.0), (0.5, 0.5), (1.0, -0.5), (0.0, 1.0)])
def test_exact_fit_is_fixed_point(model_str, dims, ab):
    """If Y = Yhat(Theta*) then a = b entrywise, num = den and Theta* is kept."""
    a, b = ab
    m = OracleModel(model_str, dims)
    rng = np.random.default_rng(10)
    f = _rand_factors(m, rng)
    y = np.einsum(model_str, *f)
    for l in range(m.n_factors):
        new, _, _ = m.update_factor(l, y, None, f, a, b, eps=0.0)
        np.testing.assert_allclose(new[l], f[l], rtol=1e-11)


def test_zeros_stay_zero():
    m = OracleModel("ir,jr,kr->ijk", dict(i=4, j=3, k=5, r=3))
    rng = np.random.default_rng(11)
    f = _rand_factors(m, rng)
    f[0][1, 2] = 0.0
    f[2][0, 0] = 0.0
    y = _rand_data(m, rng)
    for a, b in [(1.0, 0.0), (1.0, 1.0), (0.5, 0.5)]:
        g = [x.copy() for x in f]
        for _ in range(3):
            for l in range(3):
                g, _, _ = m.update_factor(l, y, None, g, a, b, eps=0.0)
        assert g[0][1, 2] == 0.0 and g[2][0, 0] == 0.0


def test_masked_entries_do_not_matter():
    m = OracleModel("ia,ja,ab,kb,lb->ijkl", dict(i=3, j=2, k=4, l=3, a=2, b=2))
    rng = np.random.default_rng(12)
    f = _rand_factors(m, rng)
    y = _rand_data(m, rng, "uniform")
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8)
    y2 = y.copy()
    y2[mask == 0] = 1e6
    for l in range(m.n_factors):
        a1, n1, d1 = m.update_factor(l, y, mask, f, 0.5, 0.5)
        a2, n2, d2 = m.update_factor(l, y2, mask, f, 0.5, 0.5)
        np.testing.assert_array_equal(n1, n2)
        np.testing.assert_array_equal(d1, d2)


def test_epsilon_floor():
    m = OracleModel("ir,jr->ij", dict(i=3, j=3, r=2))
    f = [np.full((3, 2), 1.0), np.full((3, 2), 1.0)]
    y = np.zeros((3, 3))
    new, _, _ = m.update_factor(0, y, None, f, 1.0, 0.0, eps=1e-3)
    assert np.all(new[0] == 1e-3)


def test_fully_masked_slice_keeps_theta():
    """den == 0 (a fully masked slice) leaves the factor row unchanged."""
    m = OracleModel("ir,jr->ij", dict(i=3, j=4, r=2))
    rng = np.random.default_rng(13)
    f = _rand_factors(m, rng)
    y = _rand_data(m, rng, "uniform")
    mask = np.ones((3, 4), np.uint8)
    mask[1, :] = 0
    new, num, den = m.update_factor(0, y, mask, f, 1.0, 0.0)
    assert np.all(den[1] == 0.0)
    np.testing.assert_array_equal(new[0][1], f[0][1])


def test_fit_trace_and_sampled_numden():
    m = OracleModel("ia,ja,ab,kb,lb->ijkl", dict(i=4, j=3, k=5, l=2, a=3, b=2))
    rng = np.random.default_rng(14)
    f = _rand_factors(m, rng)
    y = _rand_data(m, rng, "uniform")
    mask = (rng.random(m.y_shape) > 0.3).astype(np.uint8)
    out, tr = m.fit(y, mask, f, 0.5, 0.5, 3, trace=True)
    assert np.all(np.diff(tr) <= 1e-12 * tr[:-1])
    assert tr[-1] == pytest.approx(m.loss(y, mask, out, 0.5, 0.5)[0], rel=1e-14)
    for l in range(m.n_factors):
        _, num, den = m.update_factor(l, y, mask, f, 0.5, 0.5)
        el = np.arange(num.size)
        sn, sd = m.numden_sampled(l, el, y, mask, f, 0.5, 0.5)
        np.testing.assert_allclose(sn, num.reshape(-1), rtol=1e-12)
        np.testing.assert_allclose(sd, den.reshape(-1), rtol=1e-12)
