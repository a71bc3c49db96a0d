"""ctypes front end of the FP64 C oracle (``nef_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The einsum model string is parsed here, independently of the CUDA planner:
``model_str = "i1r1,...,iLrL->i1...iM"`` (Eq. 2.2).  Letters on the right are
the observed modes (ids 0..M-1 in RHS order); letters that appear only on the
left are contracted (latent) and get ids M.. in order of first appearance.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libnef_oracle.so")
_SRC = os.path.join(_HERE, "nef_oracle.c")

MAXLET = 26
MAXFAC = 16

_lock = threading.Lock()
_lib = None


class _Spec(ctypes.Structure):
    _fields_ = [
        ("n_obs", ctypes.c_int32),
        ("n_let", ctypes.c_int32),
        ("dim", ctypes.c_int64 * MAXLET),
        ("n_fac", ctypes.c_int32),
        ("fac_nlet", ctypes.c_int32 * MAXFAC),
        ("fac_let", (ctypes.c_int32 * MAXLET) * MAXFAC),
    ]


def build(force: bool = False) -> str:
    """Compile nef_oracle.c with gcc (-O2, OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            dpp = P(dp)
            u8p = P(ctypes.c_uint8)
            i64p = P(ctypes.c_int64)
            sp = P(_Spec)
            lib.or_reconstruct.argtypes = [sp, dpp, dp]
            lib.or_einstr.argtypes = [sp, ctypes.c_int, dp, dpp, dp]
            lib.or_weights.argtypes = [ctypes.c_int64, dp, u8p, dp, ctypes.c_double,
                                       ctypes.c_double, dp, dp]
            lib.or_update_factor.argtypes = [sp, ctypes.c_int, dp, u8p, dpp,
                                             ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, dp, dp]
            lib.or_update_factor.restype = ctypes.c_int
            lib.or_loss.argtypes = [sp, dp, u8p, dpp, ctypes.c_double, ctypes.c_double,
                                    i64p]
            lib.or_loss.restype = ctypes.c_double
            lib.or_fit.argtypes = [sp, dp, u8p, dpp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, dp]
            lib.or_fit.restype = ctypes.c_int
            lib.or_numden_sampled.argtypes = [sp, ctypes.c_int, ctypes.c_int64, i64p, dp,
                                              u8p, dpp, ctypes.c_double, ctypes.c_double,
                                              dp, dp]
            lib.or_numden_sampled.restype = ctypes.c_int
            lib.or_divergence.argtypes = [ctypes.c_double] * 4
            lib.or_divergence.restype = ctypes.c_double
            lib.or_ginv.argtypes = [ctypes.c_double] * 3
            lib.or_ginv.restype = ctypes.c_double
            lib.or_ab_supported.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.or_ab_supported.restype = ctypes.c_int
            lib.or_lik_divergence.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
            lib.or_lik_divergence.restype = ctypes.c_double
            lib.or_lik_weights.argtypes = [ctypes.c_int64, dp, u8p, dp, dp, ctypes.c_int,
                                           ctypes.c_double, dp, dp]
            lib.or_lik_loss.argtypes = [sp, dp, u8p, dp, dpp, ctypes.c_int, ctypes.c_double, i64p]
            lib.or_lik_loss.restype = ctypes.c_double
            lib.or_lik_update_factor.argtypes = [sp, ctypes.c_int, dp, u8p, dp, dpp, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_double, dp, dp]
            lib.or_lik_update_factor.restype = ctypes.c_int
            lib.or_lik_fit.argtypes = [sp, dp, u8p, dp, dpp, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, dp]
            lib.or_lik_fit.restype = ctypes.c_int
            lib.or_num_threads.restype = ctypes.c_int
            lib.or_set_num_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(int(n))


def divergence(x: float, y: float, alpha: float, beta: float) -> float:
    """D_{alpha,beta}(x, y), App. B (five cases)."""
    return float(_load().or_divergence(float(x), float(y), float(alpha), float(beta)))


def ginv(z: float, alpha: float, beta: float) -> float:
    """g^{-1}(z) for the (alpha,beta)-divergence, App. B case table."""
    return float(_load().or_ginv(float(z), float(alpha), float(beta)))


def eta_of(alpha: float, beta: float) -> float:
    """Exponent eta with g^{-1}(z) = z^eta (App. B); NaN for the log case."""
    if alpha == 0.0 and beta == 1.0:
        return float("nan")
    q = 1.0 / alpha - beta / alpha
    if q > 1.0:
        p = 1.0 - beta
    elif q < 0.0:
        p = alpha + beta - 1.0
    else:
        p = alpha
    return 1.0 / p


# Likelihood losses of App. B outside the (alpha,beta) family (see nef_oracle.c).
LIK_KINDS = {"negbin": 1, "binomial": 2, "js": 3}


def lik_divergence(kind: str, x: float, y: float, par: float = 0.0, n: float = 1.0) -> float:
    """D(x, y) of a likelihood loss of App. B: 'negbin' (dispersion par),
    'binomial' on odds y with n trials (n = 1: Bernoulli), 'js' (Jensen-Shannon)."""
    return float(_load().or_lik_divergence(LIK_KINDS[kind], float(x), float(y), float(par), float(n)))


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_uint8)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


class OracleModel:
    """A parsed model string plus dimensions (Eq. 2.2).

    ``dims`` maps every letter to its size: observed letters take the
    dimensions of Y, latent letters the ranks.
    """

    def __init__(self, model_str: str, dims: dict):
        model_str = model_str.replace(" ", "")
        if model_str.count("->") != 1:
            raise ValueError("model string needs exactly one '->'")
        lhs, rhs = model_str.split("->")
        terms = lhs.split(",")
        for ch in rhs + "".join(terms):
            if not ("a" <= ch <= "z"):
                raise ValueError(f"bad letter {ch!r}")
        if len(set(rhs)) != len(rhs):
            raise ValueError("repeated output letter")
        for t in terms:
            if len(set(t)) != len(t):
                raise ValueError(f"repeated letter inside term {t!r}")
        for ch in rhs:
            if not any(ch in t for t in terms):
                raise ValueError(f"output letter {ch!r} not in any term")
        latent = []
        for t in terms:
            for ch in t:
                if ch not in rhs and ch not in latent:
                    latent.append(ch)
        self.model_str = model_str
        self.terms = terms
        self.observed = list(rhs)
        self.latent = latent
        self.letters = self.observed + self.latent
        self.lid = {ch: k for k, ch in enumerate(self.letters)}
        self.dims = {ch: int(dims[ch]) for ch in self.letters}
        if len(self.letters) > MAXLET or len(terms) > MAXFAC:
            raise ValueError("too many letters or factors")
        s = _Spec()
        s.n_obs = len(self.observed)
        s.n_let = len(self.letters)
        for ch, k in self.lid.items():
            s.dim[k] = self.dims[ch]
        s.n_fac = len(terms)
        for f, t in enumerate(terms):
            s.fac_nlet[f] = len(t)
            for p, ch in enumerate(t):
                s.fac_let[f][p] = self.lid[ch]
        self._spec = s

    # ------------------------------------------------------------- shapes
    @property
    def y_shape(self):
        return tuple(self.dims[ch] for ch in self.observed)

    def factor_shape(self, l: int):
        return tuple(self.dims[ch] for ch in self.terms[l])

    @property
    def n_factors(self) -> int:
        return len(self.terms)

    def einstr(self, l: int) -> str:
        """swap(model_str, l): the output and the l-th term exchange places."""
        terms = list(self.terms)
        out = terms[l]
        terms[l] = "".join(self.observed)
        return ",".join(terms) + "->" + out

    # ------------------------------------------------------------ helpers
    def _fac_ptrs(self, factors):
        arr = (ctypes.POINTER(ctypes.c_double) * len(factors))()
        for k, f in enumerate(factors):
            arr[k] = _dptr(f)
        return arr

    def _check(self, y=None, mask=None, factors=None):
        out = []
        if y is not None:
            y = np.ascontiguousarray(y, dtype=np.float64)
            assert y.shape == self.y_shape, (y.shape, self.y_shape)
            out.append(y)
        if mask is not None:
            mask = np.ascontiguousarray(mask, dtype=np.uint8)
            assert mask.shape == self.y_shape
        if factors is not None:
            fs = []
            for l, f in enumerate(factors):
                f = np.ascontiguousarray(f, dtype=np.float64)
                assert f.shape == self.factor_shape(l), (l, f.shape)
                fs.append(f)
            factors = fs
        return y, mask, factors

    # -------------------------------------------------------- paper steps
    def reconstruct(self, factors) -> np.ndarray:
        """Eq. 2.1: Yhat = einsum(model_str, Theta)."""
        _, _, factors = self._check(factors=factors)
        out = np.empty(self.y_shape, dtype=np.float64)
        _load().or_reconstruct(ctypes.byref(self._spec), self._fac_ptrs(factors), _dptr(out))
        return out

    def einstr_contract(self, l: int, T, factors) -> np.ndarray:
        """Eq. 3.8: einsum(einstr_l, Theta^(1..l-1), T, Theta^(l+1..L))."""
        _, _, factors = self._check(factors=factors)
        T = np.ascontiguousarray(T, dtype=np.float64)
        assert T.shape == self.y_shape
        out = np.empty(self.factor_shape(l), dtype=np.float64)
        _load().or_einstr(ctypes.byref(self._spec), int(l), _dptr(T),
                          self._fac_ptrs(factors), _dptr(out))
        return out

    def weights(self, y, mask, yhat, alpha, beta):
        """Masked a(Y,Yhat), b(Y,Yhat) (App. B)."""
        y = np.ascontiguousarray(y, dtype=np.float64)
        yhat = np.ascontiguousarray(yhat, dtype=np.float64)
        mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        wa = np.empty_like(y)
        wb = np.empty_like(y)
        _load().or_weights(y.size, _dptr(y), _u8ptr(mask), _dptr(yhat), float(alpha),
                           float(beta), _dptr(wa), _dptr(wb))
        return wa, wb

    def update_factor(self, l, y, mask, factors, alpha, beta, eps=1e-10):
        """One inner step of Algorithm 1 on a copy of the factors.

        Returns (new_factors, num, den)."""
        y, mask, factors = self._check(y, mask, factors)
        factors = [f.copy() for f in factors]
        num = np.empty(self.factor_shape(l))
        den = np.empty(self.factor_shape(l))
        rc = _load().or_update_factor(ctypes.byref(self._spec), int(l), _dptr(y),
                                      _u8ptr(mask), self._fac_ptrs(factors), float(alpha),
                                      float(beta), float(eps), _dptr(num), _dptr(den))
        if rc == 1:
            raise ValueError("alpha == 0 with beta != 1 has no decomposition (App. B)")
        if rc:
            raise MemoryError("oracle allocation failed")
        return factors, num, den

    def loss(self, y, mask, factors, alpha, beta):
        """Sum over observed entries of D_{alpha,beta}(y, yhat); returns (sum, count)."""
        y, mask, factors = self._check(y, mask, factors)
        cnt = ctypes.c_int64(0)
        tot = _load().or_loss(ctypes.byref(self._spec), _dptr(y), _u8ptr(mask),
                              self._fac_ptrs(factors), float(alpha), float(beta),
                              ctypes.byref(cnt))
        return float(tot), int(cnt.value)

    def fit(self, y, mask, factors, alpha, beta, iters, eps=1e-10, trace=False):
        """Algorithm 1 for `iters` sweeps on copies of the factors.

        Returns new factors (and the loss trace of iters+1 values if asked)."""
        y, mask, factors = self._check(y, mask, factors)
        factors = [f.copy() for f in factors]
        tr = np.empty(iters + 1) if trace else None
        rc = _load().or_fit(ctypes.byref(self._spec), _dptr(y), _u8ptr(mask),
                            self._fac_ptrs(factors), float(alpha), float(beta), float(eps),
                            int(iters),
                            _dptr(tr) if trace else ctypes.POINTER(ctypes.c_double)())
        if rc == 1:
            raise ValueError("alpha == 0 with beta != 1 has no decomposition (App. B)")
        if rc:
            raise MemoryError("oracle allocation failed")
        return (factors, tr) if trace else factors

    def _ntr(self, ntrials):
        if ntrials is None:
            return None
        ntrials = np.ascontiguousarray(ntrials, dtype=np.float64)
        if ntrials.shape != self.y_shape:
            raise ValueError("ntrials must have the shape of Y")
        return ntrials

    def lik_update_factor(self, l, y, mask, factors, kind, par=0.0, ntrials=None, eps=1e-10):
        """One inner step of Algorithm 1 under a likelihood loss of App. B
        ('negbin', 'binomial', 'js') on a copy of the factors; returns
        (new_factors, num, den)."""
        y, mask, factors = self._check(y, mask, factors)
        nt = self._ntr(ntrials)
        factors = [f.copy() for f in factors]
        num = np.empty(self.factor_shape(l))
        den = np.empty(self.factor_shape(l))
        rc = _load().or_lik_update_factor(ctypes.byref(self._spec), int(l), _dptr(y), _u8ptr(mask),
                                          _dptr(nt) if nt is not None else ctypes.POINTER(ctypes.c_double)(),
                                          self._fac_ptrs(factors), LIK_KINDS[kind], float(par), float(eps),
                                          _dptr(num), _dptr(den))
        if rc:
            raise ValueError("unknown loss kind" if rc == 1 else "oracle allocation failed")
        return factors, num, den

    def lik_loss(self, y, mask, factors, kind, par=0.0, ntrials=None):
        """Sum over observed entries of D(y, yhat) for a likelihood loss; (sum, count)."""
        y, mask, factors = self._check(y, mask, factors)
        nt = self._ntr(ntrials)
        cnt = ctypes.c_int64(0)
        tot = _load().or_lik_loss(ctypes.byref(self._spec), _dptr(y), _u8ptr(mask),
                                  _dptr(nt) if nt is not None else ctypes.POINTER(ctypes.c_double)(),
                                  self._fac_ptrs(factors), LIK_KINDS[kind], float(par), ctypes.byref(cnt))
        return float(tot), int(cnt.value)

    def lik_fit(self, y, mask, factors, kind, iters, par=0.0, ntrials=None, eps=1e-10, trace=False):
        """Algorithm 1 under a likelihood loss for `iters` sweeps on copies of the
        factors; returns new factors (and the loss trace of iters+1 values if asked)."""
        y, mask, factors = self._check(y, mask, factors)
        nt = self._ntr(ntrials)
        factors = [f.copy() for f in factors]
        tr = np.empty(iters + 1) if trace else None
        rc = _load().or_lik_fit(ctypes.byref(self._spec), _dptr(y), _u8ptr(mask),
                                _dptr(nt) if nt is not None else ctypes.POINTER(ctypes.c_double)(),
                                self._fac_ptrs(factors), LIK_KINDS[kind], float(par), float(eps), int(iters),
                                _dptr(tr) if trace else ctypes.POINTER(ctypes.c_double)())
        if rc:
            raise ValueError("unknown loss kind" if rc == 1 else "oracle allocation failed")
        return (factors, tr) if trace else factors

    def numden_sampled(self, l, elems, y, mask, factors, alpha, beta):
        """num/den (Eq. 3.6-3.8) for selected flat elements of factor l."""
        y, mask, factors = self._check(y, mask, factors)
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        num = np.empty(elems.size)
        den = np.empty(elems.size)
        rc = _load().or_numden_sampled(
            ctypes.byref(self._spec), int(l), elems.size,
            elems.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(y), _u8ptr(mask),
            self._fac_ptrs(factors), float(alpha), float(beta), _dptr(num), _dptr(den))
        if rc:
            raise ValueError("unsupported (alpha, beta)")
        return num, den

    def apply_update(self, theta, num, den, alpha, beta, eps=1e-10):
        """Eq. 3.4 elementwise, in Python over the C g^{-1} (den == 0 keeps theta)."""
        theta = np.array(theta, dtype=np.float64, copy=True)
        flat = theta.reshape(-1)
        n = np.asarray(num, dtype=np.float64).reshape(-1)
        d = np.asarray(den, dtype=np.float64).reshape(-1)
        for e in range(flat.size):
            if d[e] == 0.0:
                continue
            flat[e] = max(eps, flat[e] * ginv(n[e] / d[e], alpha, beta))
        return theta
