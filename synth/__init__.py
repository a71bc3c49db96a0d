"""Seeded synthetic inputs for the nonnegative einsum factorization workloads.

This module is shared by the oracle tests and the CUDA-path tests and holds
none of the method's arithmetic: it draws ground-truth factors, data and masks
with ``numpy.random.default_rng(seed)`` in a fixed order, and forms the
synthetic data mean with ``numpy.einsum`` (a library call used only to make
data, never as an expected value).

Draw order for one problem (fixed, so every consumer sees identical bytes):
  1. ground-truth factors, one per term in model-string order;
  2. Y: Poisson(mean) counts, or mean * Gamma(k, theta) multiplicative noise;
  3. mask: Bernoulli(1 - missing) observed indicators (1 = observed);
  4. initial factors per restart, uniform on [lo, hi), term order.

Gamma(k, theta) is shape-scale: Gamma(0.3, 1) has mean 0.3 and Gamma(2, 0.5)
has mean 1.  Workload recipes (shapes, ranks, distributions) follow the five
configurations the benchmarks and parity tests use.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def parse_terms(model_str: str):
    lhs, rhs = model_str.replace(" ", "").split("->")
    return lhs.split(","), rhs


@dataclass
class Problem:
    model_str: str
    dims: dict
    y: np.ndarray                      # float32, shape of the observed letters (RHS order)
    mask: np.ndarray | None            # uint8 (1 = observed) or None
    truth: list                        # ground-truth factors (float64)
    inits: list = field(default_factory=list)  # list over restarts of lists of float32 factors
    alpha: float = 1.0
    beta: float = 0.0
    note: str = ""

    def factor_shapes(self):
        terms, _ = parse_terms(self.model_str)
        return [tuple(self.dims[c] for c in t) for t in terms]


def draw_data(mean, rng, data="poisson", noise=(2.0, 0.5), par=1.0):
    """Data around a nonnegative mean tensor: Poisson(mean) counts; mean *
    Gamma(k, theta) multiplicative noise (positive values); negative binomial
    counts Poisson(mean * Gamma(par, 1/par)) with dispersion par; or binomial
    counts Binomial(n = par, mean / (1 + mean)), mean being the odds."""
    if data == "poisson":
        return rng.poisson(mean)
    if data == "gamma_noise":
        return mean * rng.gamma(noise[0], noise[1], size=mean.shape)
    if data == "negbin":
        return rng.poisson(mean * rng.gamma(par, 1.0 / par, size=mean.shape))
    if data == "binomial":
        return rng.binomial(int(par), mean / (1.0 + mean))
    raise ValueError(data)


def make_problem(model_str: str, dims: dict, seed: int = 0, *,
                 gamma=(0.3, 1.0), data="poisson", noise=(2.0, 0.5), par=1.0,
                 missing=0.0, restarts=1, init=(0.5, 1.5), alpha=1.0, beta=0.0,
                 y_dtype=np.float32) -> Problem:
    terms, rhs = parse_terms(model_str)
    rng = np.random.default_rng(seed)
    truth = []
    for t in terms:
        shp = tuple(int(dims[c]) for c in t)
        truth.append(rng.gamma(gamma[0], gamma[1], size=shp))
    mean = np.einsum(model_str, *truth, optimize=True)
    y = draw_data(mean, rng, data, noise, par).astype(y_dtype)
    del mean
    mask = None
    if missing > 0.0:
        mask = (rng.random(size=y.shape) >= missing).astype(np.uint8)
    inits = []
    for _ in range(restarts):
        fs = []
        for t in terms:
            shp = tuple(int(dims[c]) for c in t)
            fs.append(rng.uniform(init[0], init[1], size=shp).astype(np.float32))
        inits.append(fs)
    return Problem(model_str, {c: int(v) for c, v in dims.items()}, y, mask, truth, inits,
                   alpha, beta)


# ----------------------------------------------------------------- recipes
# (alpha, beta) are the paper's parameters (App. B): "KL" is (1, 0); the
# beta-divergence index 0.5 is (1, -0.5); the explicit AB pair (0.5, 0.5) is
# taken literally.

def config1(seed=0) -> Problem:
    """Plain CP 30x40x50, rank 5, Gamma(0.3,1) truth, Poisson data, 10% missing,
    KL, init U(0.5,1.5)."""
    p = make_problem("ir,jr,kr->ijk", {"i": 30, "j": 40, "k": 50, "r": 5}, seed,
                     gamma=(0.3, 1.0), missing=0.10, alpha=1.0, beta=0.0)
    p.note = "cp 30x40x50 R5 KL 10% missing"
    return p


def config2(seed=0, beta=0.0, n=512, rank=64) -> Problem:
    """Large dense CP n^3 rank 64, Poisson counts from Gamma(0.3,1) factors, no
    mask.  beta = 0 (KL) or -0.5 (beta-divergence index 0.5)."""
    p = make_problem("ir,jr,kr->ijk", {"i": n, "j": n, "k": n, "r": rank}, seed,
                     gamma=(0.3, 1.0), missing=0.0, alpha=1.0, beta=beta)
    p.note = f"cp {n}^3 R{rank} (1,{beta})"
    return p


def config3(seed=0, shape=(256, 256, 64, 32), a=16, b=8) -> Problem:
    """Custom 'ia,ja,ab,kb,lb->ijkl', Gamma(0.5,1) factors, Y = mean * Gamma(2,0.5),
    30% missing, (alpha, beta) = (0.5, 0.5)."""
    i, j, k, l = shape
    p = make_problem("ia,ja,ab,kb,lb->ijkl",
                     {"i": i, "j": j, "k": k, "l": l, "a": a, "b": b}, seed,
                     gamma=(0.5, 1.0), data="gamma_noise", noise=(2.0, 0.5),
                     missing=0.30, alpha=0.5, beta=0.5)
    p.note = f"ia,ja,ab,kb,lb->ijkl {shape} a{a} b{b} (0.5,0.5) 30% missing"
    return p


# loss families of the 512^3 CP workload beyond KL: the data each one models
LOSS_WORKLOADS = {
    "rkl": dict(data="gamma_noise", alpha=0.0, beta=1.0, loss="ab", par=0.0,
                note="reverse KL (0,1), Y = mean * Gamma(2, 0.5)"),
    "negbin": dict(data="negbin", alpha=1.0, beta=0.0, loss="negbin", par=2.0,
                   note="negative binomial phi = 2, Y ~ Poisson(mean * Gamma(2, 1/2))"),
    "bernoulli": dict(data="binomial", alpha=1.0, beta=0.0, loss="binomial", par=1.0,
                      note="Bernoulli on the odds, Y ~ Bernoulli(mean / (1 + mean))"),
    "js": dict(data="poisson", alpha=1.0, beta=0.0, loss="js", par=0.0,
               note="Jensen-Shannon, Y ~ Poisson(mean)"),
}


def config2_loss(kind, seed=0, n=512, rank=64) -> Problem:
    """The 512^3 rank-64 CP workload (Gamma(0.3,1) truth, no mask) with the data
    of loss family `kind` (LOSS_WORKLOADS); p.loss / p.loss_par name the family."""
    w = LOSS_WORKLOADS[kind]
    p = make_problem("ir,jr,kr->ijk", {"i": n, "j": n, "k": n, "r": rank}, seed,
                     gamma=(0.3, 1.0), data=w["data"], par=w["par"], missing=0.0,
                     alpha=w["alpha"], beta=w["beta"])
    p.loss, p.loss_par = w["loss"], w["par"]
    p.note = f"cp {n}^3 R{rank} {w['note']}"
    return p


def batched_specs(n_problems=512, seed=0, lo=20, hi=300, rlo=4, rhi=32):
    """Shapes and ranks of the batched CP workload: dims ~ U{lo..hi} per mode,
    ranks ~ U{rlo..rhi}; drawn from a generator of their own (seed + 1)."""
    rng = np.random.default_rng(seed + 1)
    dims = rng.integers(lo, hi + 1, size=(n_problems, 3))
    ranks = rng.integers(rlo, rhi + 1, size=n_problems)
    return [(tuple(int(v) for v in d), int(r)) for d, r in zip(dims, ranks)]


def batched_problem(shape, rank, seed, restarts=8) -> Problem:
    i, j, k = shape
    return make_problem("ir,jr,kr->ijk", {"i": i, "j": j, "k": k, "r": rank}, seed,
                        gamma=(0.3, 1.0), missing=0.10, restarts=restarts,
                        alpha=1.0, beta=0.0)


def random_factors(model_str, dims, seed, lo=0.5, hi=1.5):
    terms, _ = parse_terms(model_str)
    rng = np.random.default_rng(seed)
    return [rng.uniform(lo, hi, size=tuple(dims[c] for c in t)) for t in terms]


def config_uber(seed=0, dims=(27, 7, 24, 100, 100), r=10, k=6) -> Problem:
    """The paper's Uber model 'wr,dr,hr,irk,jrk->wdhij' at the Uber tensor's shape
    27x7x24x100x100 (45.4 M entries) with R = 10, K = 6 (the ranks of the paper's
    qualitative Uber fit); Gamma(0.3,1) truth, Poisson data, no mask, KL."""
    w, d, h, i, j = dims
    p = make_problem("wr,dr,hr,irk,jrk->wdhij", {"w": w, "d": d, "h": h, "i": i, "j": j, "r": r, "k": k},
                     seed, gamma=(0.3, 1.0), missing=0.0, alpha=1.0, beta=0.0)
    p.note = f"uber-shaped wr,dr,hr,irk,jrk->wdhij {dims} R{r} K{k} KL"
    return p


def config_icews(seed=0, dims=(249, 249, 20, 228), r=16, k=4) -> Problem:
    """The paper's ICEWS model 'ir,jr,ak,kr,tr->ijat' at the ICEWS tensor's shape
    249x249x20x228 (282.7 M entries) with R = 16, K = 4 (the paper does not state
    the ranks of its ICEWS fits); Gamma(0.3,1) truth, Poisson data, no mask, KL."""
    i, j, a, t = dims
    p = make_problem("ir,jr,ak,kr,tr->ijat", {"i": i, "j": j, "a": a, "t": t, "r": r, "k": k}, seed,
                     gamma=(0.3, 1.0), missing=0.0, alpha=1.0, beta=0.0)
    p.note = f"icews-shaped ir,jr,ak,kr,tr->ijat {dims} R{r} K{k} KL"
    return p


def config5(seed=0, n=2048, jk=(128, 128), rank=32, n_train=1536) -> Problem:
    """Fold-in workload: CP 'ir,jr,kr->ijk' n x J x K rank 32, Gamma(0.3,1) truth,
    Poisson data, no mask, KL.  Slices 0..n_train-1 train the model and the
    encoder; the rest are held out."""
    j, k = jk
    p = make_problem("ir,jr,kr->ijk", {"i": n, "j": j, "k": k, "r": rank}, seed,
                     gamma=(0.3, 1.0), missing=0.0, alpha=1.0, beta=0.0)
    p.note = f"fold-in cp {n}x{j}x{k} R{rank}, {n_train} train slices"
    return p


def mlp_params(sizes, seed=0):
    """Initial encoder parameters: He-uniform weights U(-sqrt(6/fan_in), +),
    zero biases, for layer widths sizes = (d_in, h, h, d_out); returned as the
    list W1, b1, W2, b2, W3, b3 (float64, weights [fan_in x fan_out])."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / a)
        params.append(rng.uniform(-lim, lim, size=(a, b)))
        params.append(np.zeros(b))
    return params
