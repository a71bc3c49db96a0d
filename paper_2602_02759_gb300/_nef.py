"""ctypes binding of the C ABI in include/nef.h (argument marshalling only).

Every step of the sweep runs in libnef.so's CUDA kernels; torch only provides
device memory and the stream.  The library is built in-tree by
``paper_2602_02759_gb300.build`` (or ``__graft_entry__.build()``); if it is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnef.so")

NEF_FP32, NEF_BF16, NEF_FP64 = 0, 1, 2
NEF_LOSS_AB, NEF_LOSS_NEGBIN, NEF_LOSS_BINOMIAL, NEF_LOSS_JS = 0, 1, 2, 3
LOSSES = {"ab": NEF_LOSS_AB, "negbin": NEF_LOSS_NEGBIN, "binomial": NEF_LOSS_BINOMIAL, "js": NEF_LOSS_JS}
STATUS = {0: "NEF_OK", 1: "NEF_EINVAL", 2: "NEF_EPARSE", 3: "NEF_EUNSUPPORTED", 4: "NEF_ENOMEM",
          5: "NEF_ECUDA", 6: "NEF_EDATA", 7: "NEF_ETIMEOUT"}
PRECISIONS = {"fp32": NEF_FP32, "bf16": NEF_BF16, "fp64": NEF_FP64}

# every symbol include/nef.h declares
EXPORTS = ["nef_default_options", "nef_plan", "nef_plan_destroy", "nef_fit", "nef_fit_ex", "nef_fit_ctl",
           "nef_plan_sweeps", "nef_plan_autotune", "nef_update", "nef_numden", "nef_apply_update", "nef_loss",
           "nef_plan_info", "nef_plan_launches",
           "nef_plan_profile", "nef_tc_trace", "nef_check", "nef_fit_batched", "nef_fit_batched_tune", "nef_cp3_update_static",
           "nef_last_error",
           "nef_foldin_num_params", "nef_foldin_create", "nef_foldin_destroy", "nef_foldin_grad",
           "nef_foldin_train_step", "nef_foldin_predict", "nef_foldin_load_batch", "nef_foldin_params"]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eps", ctypes.c_double),
                ("check_data", ctypes.c_int), ("force_generic", ctypes.c_int),
                ("profile", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("tol", ctypes.c_double), ("loss_trace", ctypes.c_void_p), ("eager", ctypes.c_int),
                ("loss", ctypes.c_int), ("loss_par", ctypes.c_double), ("wait_cycles", ctypes.c_int64),
                ("batch_tiles", ctypes.c_int)]


class FitControl(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("loss_trace", ctypes.c_void_p), ("val_mask", ctypes.c_void_p),
                ("val_patience", ctypes.c_int), ("val_trace", ctypes.c_void_p)]


class NefError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libnef.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libnef.so not built at {path}; run paper_2602_02759_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    lib.nef_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.nef_plan.argtypes = [ctypes.c_char_p, i64p, ctypes.c_int, i64p, ctypes.c_int,
                             ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.nef_plan.restype = ctypes.c_int
    lib.nef_plan_destroy.argtypes = [vp]
    lib.nef_fit.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                            ctypes.c_int]
    lib.nef_fit.restype = ctypes.c_int
    lib.nef_fit_ex.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                               ctypes.c_int, ctypes.c_double, vp, ctypes.POINTER(ctypes.c_int)]
    lib.nef_fit_ex.restype = ctypes.c_int
    lib.nef_fit_ctl.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                ctypes.c_int, ctypes.POINTER(FitControl), ctypes.POINTER(ctypes.c_int)]
    lib.nef_fit_ctl.restype = ctypes.c_int
    lib.nef_plan_autotune.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    lib.nef_plan_autotune.restype = ctypes.c_int
    lib.nef_plan_sweeps.argtypes = [vp]
    lib.nef_plan_sweeps.restype = ctypes.c_int
    lib.nef_update.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(vp), ctypes.c_double,
                               ctypes.c_double]
    lib.nef_update.restype = ctypes.c_int
    lib.nef_numden.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double,
                               vp, vp]
    lib.nef_numden.restype = ctypes.c_int
    lib.nef_apply_update.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), vp, vp, ctypes.c_double,
                                     ctypes.c_double]
    lib.nef_apply_update.restype = ctypes.c_int
    lib.nef_loss.argtypes = [vp, vp, vp, ctypes.POINTER(vp), ctypes.c_double, ctypes.c_double, dp]
    lib.nef_loss.restype = ctypes.c_int
    lib.nef_plan_info.argtypes = [vp, ctypes.c_char_p, ctypes.c_int]
    lib.nef_plan_info.restype = ctypes.c_int
    lib.nef_plan_launches.argtypes = [vp, ctypes.c_int]
    lib.nef_plan_launches.restype = ctypes.c_int
    lib.nef_plan_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                     ctypes.c_int]
    lib.nef_plan_profile.restype = ctypes.c_int
    lib.nef_check.argtypes = [vp]
    lib.nef_check.restype = ctypes.c_int
    lib.nef_last_error.restype = ctypes.c_char_p
    lib.nef_fit_batched.argtypes = [ctypes.c_int, i64p, i64p, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.POINTER(Options), dp]
    lib.nef_fit_batched.restype = ctypes.c_int
    lib.nef_fit_batched_tune.argtypes = [ctypes.c_int, i64p, i64p, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                         ctypes.POINTER(vp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_int), dp]
    lib.nef_fit_batched_tune.restype = ctypes.c_int
    lib.nef_cp3_update_static.argtypes = [vp, i64p, ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, vp]
    lib.nef_cp3_update_static.restype = ctypes.c_int
    ci, dbl = ctypes.c_int, ctypes.c_double
    lib.nef_foldin_num_params.argtypes = [ci, ci, ci]
    lib.nef_foldin_num_params.restype = ctypes.c_int64
    lib.nef_foldin_create.argtypes = [ci, ci, ci, ci, vp, vp, ctypes.POINTER(vp)]
    lib.nef_foldin_create.restype = ci
    lib.nef_foldin_destroy.argtypes = [vp]
    lib.nef_foldin_grad.argtypes = [vp, vp, vp, ci, vp, dp]
    lib.nef_foldin_grad.restype = ci
    lib.nef_foldin_train_step.argtypes = [vp, vp, vp, ci, dbl, dbl, dbl, dbl, dp]
    lib.nef_foldin_train_step.restype = ci
    lib.nef_foldin_predict.argtypes = [vp, vp, ci, vp]
    lib.nef_foldin_load_batch.argtypes = [vp, vp, ci]
    lib.nef_foldin_load_batch.restype = ctypes.c_int
    lib.nef_foldin_predict.restype = ci
    lib.nef_foldin_params.argtypes = [vp, vp]
    lib.nef_foldin_params.restype = ci
    lib.nef_tc_trace.argtypes = [vp, ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_int]
    lib.nef_tc_trace.restype = ctypes.c_int
    _lib = lib
    return lib


def check(status: int):
    if status != 0:
        msg = load().nef_last_error().decode(errors="replace")
        raise NefError(status, msg)


def split_model(model_str: str):
    """Observed letters (RHS order) and latent letters (order of first appearance)."""
    s = model_str.replace(" ", "")
    lhs, rhs = s.split("->")
    latent = []
    for ch in lhs.replace(",", ""):
        if ch not in rhs and ch not in latent:
            latent.append(ch)
    return list(rhs), latent, lhs.split(",")


def _batched_args(Ys, masks, factors, eps, stream, tiles):
    import torch
    n = len(Ys)
    restarts = len(factors[0])
    if stream is None:
        stream = torch.cuda.current_stream()
    shapes = (ctypes.c_int64 * (3 * n))(*[int(d) for y in Ys for d in y.shape])
    ranks = (ctypes.c_int64 * n)(*[int(factors[p][0][0].shape[1]) for p in range(n)])
    ys = (ctypes.c_void_p * n)(*[y.data_ptr() for y in Ys])
    ms = None if masks is None else (ctypes.c_void_p * n)(*[m.data_ptr() for m in masks])
    fs = (ctypes.c_void_p * (3 * n * restarts))(
        *[f.data_ptr() for p in range(n) for k in range(restarts) for f in factors[p][k]])
    opt = Options()
    load().nef_default_options(ctypes.byref(opt))
    opt.precision = NEF_BF16
    opt.eps = float(eps)
    opt.stream = ctypes.c_void_p(stream.cuda_stream)
    opt.batch_tiles = int(tiles)
    return n, restarts, shapes, ranks, ys, ms, fs, opt


def fit_batched(Ys, masks, factors, alpha, beta, iters, eps=1e-10, stream=None, losses=True, tiles=0):
    """nef_fit_batched: fit many CP models 'ir,jr,kr->ijk', each with several restarts.

    Ys: list of n CUDA float32 [I, J, K] tensors; masks: None or a list of n uint8
    tensors; factors: list over problems of lists over restarts of [A, B, C]
    (CUDA float32, updated in place); tiles: column tiles per work item (0 = the
    default; see fit_batched_tune).  Returns an n x restarts list of losses."""
    n, restarts, shapes, ranks, ys, ms, fs, opt = _batched_args(Ys, masks, factors, eps, stream, tiles)
    out = (ctypes.c_double * (n * restarts))() if losses else None
    check(load().nef_fit_batched(n, shapes, ranks, ys, ms, fs, restarts, float(alpha), float(beta), int(iters),
                                 ctypes.byref(opt), out))
    if not losses:
        return None
    return [[out[p * restarts + k] for k in range(restarts)] for p in range(n)]


def fit_batched_tune(Ys, masks, factors, alpha, beta, eps=1e-10, stream=None):
    """nef_fit_batched_tune: the column tiles per work item (16 .. 256) with which
    two sweeps of fit_batched run fastest on this workload (timed on copies of the
    factors, which are left unchanged).  Returns (tiles, {tiles: ms})."""
    n, restarts, shapes, ranks, ys, ms, fs, opt = _batched_args(Ys, masks, factors, eps, stream, 0)
    best = ctypes.c_int()
    times = (ctypes.c_double * 5)()
    check(load().nef_fit_batched_tune(n, shapes, ranks, ys, ms, fs, restarts, float(alpha), float(beta),
                                      ctypes.byref(opt), ctypes.byref(best), times))
    return best.value, dict(zip((16, 32, 64, 128, 256), list(times)))


def cp3_update_static(Y, factors, l, alpha, beta, eps=1e-10, stream=None):
    """nef_cp3_update_static: update factor l of 'ir,jr,kr->ijk' in place without any
    device allocation (see include/nef.h).  Y: contiguous CUDA float32 [I, J, K];
    factors: three contiguous CUDA float32 tensors [I, R], [J, R], [K, R] with one R.
    The C entry point cannot see the factors' sizes, so they are checked here and a
    mismatch raises NefError(NEF_EINVAL) before anything is launched."""
    import torch
    lib = load()

    def bad(msg):
        raise NefError(1, msg)

    if not isinstance(Y, torch.Tensor) or Y.dim() != 3 or Y.dtype != torch.float32 or not Y.is_cuda \
            or not Y.is_contiguous():
        bad("Y must be a contiguous 3-d CUDA float32 tensor")
    if len(factors) != 3:
        bad("three factors are needed")
    rank = int(factors[0].shape[1]) if factors[0].dim() == 2 else -1
    for m, f in enumerate(factors):
        if not isinstance(f, torch.Tensor) or f.dtype != torch.float32 or not f.is_cuda or not f.is_contiguous() \
                or f.dim() != 2 or tuple(f.shape) != (int(Y.shape[m]), rank) or f.device != Y.device:
            bad(f"factor {m} must be a contiguous CUDA float32 tensor of shape ({int(Y.shape[m])}, R) "
                f"on Y's device, R the same for all three")
    if stream is None:
        stream = torch.cuda.current_stream()
    shape = (ctypes.c_int64 * 3)(*[int(s) for s in Y.shape])
    arr = (ctypes.c_void_p * 3)(*[f.data_ptr() for f in factors])
    check(lib.nef_cp3_update_static(ctypes.c_void_p(Y.data_ptr()), shape, rank, arr, int(l), float(alpha),
                                    float(beta), float(eps), ctypes.c_void_p(stream.cuda_stream)))


class Plan:
    """A plan for one model string and shape (nef_plan).

    ``dims`` maps letters to sizes (observed dims and latent ranks).  ``stream``
    is a torch.cuda.Stream (or a raw cudaStream_t integer); None uses torch's
    current stream at plan time.  ``loss`` selects the loss family (App. B):
    "ab" (the (alpha,beta)-divergence given to each call), "negbin" (dispersion
    ``loss_par``), "binomial" (``loss_par`` trials; 1 = Bernoulli) or "js".
    ``wait_cycles`` bounds every wait inside the tensor-core pass (0 = default).
    """

    def __init__(self, model_str: str, dims: dict, precision: str = "fp32", eps: float = 1e-10,
                 check_data: bool = False, force_generic: bool = False, profile: int = 0,
                 stream=None, eager: bool = False, loss: str = "ab", loss_par: float = 0.0,
                 wait_cycles: int = 0):
        lib = load()
        obs, lat, terms = split_model(model_str)
        self.model_str = model_str
        self.terms = terms
        self.dims = dict(dims)
        self.precision = precision
        shapes = (ctypes.c_int64 * max(1, len(obs)))(*[int(dims[c]) for c in obs])
        ranks = (ctypes.c_int64 * max(1, len(lat)))(*[int(dims[c]) for c in lat])
        opt = Options()
        lib.nef_default_options(ctypes.byref(opt))
        opt.precision = PRECISIONS[precision]
        opt.eps = float(eps)
        opt.check_data = int(bool(check_data))
        opt.force_generic = int(bool(force_generic))
        opt.profile = int(profile)
        opt.eager = int(bool(eager))
        opt.loss = LOSSES[loss]
        opt.loss_par = float(loss_par)
        opt.wait_cycles = int(wait_cycles)
        self.loss_kind = loss
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        self.stream = stream
        opt.stream = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        h = ctypes.c_void_p()
        check(lib.nef_plan(model_str.encode(), shapes, len(obs), ranks, len(lat),
                           ctypes.byref(opt), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().nef_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ----------------------------------------------------------- helpers
    @staticmethod
    def _ptr(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    def _facs(self, factors):
        arr = (ctypes.c_void_p * len(factors))()
        for k, f in enumerate(factors):
            arr[k] = f.data_ptr()
        return arr

    def _check_args(self, Y, mask, factors):
        import torch
        want = torch.float64 if self.precision == "fp64" else torch.float32
        if Y.dtype != want or not Y.is_contiguous() or not Y.is_cuda:
            raise ValueError(f"Y must be a contiguous CUDA {want} tensor")
        if mask is not None and (mask.dtype != torch.uint8 or not mask.is_contiguous()
                                 or mask.numel() != Y.numel() or not mask.is_cuda):
            raise ValueError("mask must be a contiguous CUDA uint8 tensor shaped like Y")
        if len(factors) != len(self.terms):
            raise ValueError("wrong number of factors")
        for t, f in zip(self.terms, factors):
            shp = tuple(int(self.dims[c]) for c in t)
            if f.dtype != want or not f.is_contiguous() or tuple(f.shape) != shp or not f.is_cuda:
                raise ValueError(f"factor {t} must be a contiguous CUDA {want} tensor of shape {shp}")

    # -------------------------------------------------------------- ABI
    def fit(self, Y, mask, factors, alpha, beta, iters, tol: float = 0.0, loss_trace=None,
            val_mask=None, val_patience: int = 0, val_trace=None, sweeps: bool = True):
        """Run up to `iters` sweeps (nef_fit_ctl).  ``loss_trace`` / ``val_trace``:
        float64 CUDA tensors of at least iters + 1 entries receiving the training
        loss / the loss over ``val_mask`` (a uint8 CUDA tensor shaped like Y) after
        each sweep; ``tol`` > 0 and ``val_patience`` > 0 are App. B's stopping rules,
        evaluated on the device.  Returns the number of sweeps run (reading it
        synchronises the stream; ``sweeps=False`` returns None without waiting)."""
        import torch
        self._check_args(Y, val_mask, factors)
        self._check_args(Y, mask, factors)
        for name, tr in (("loss_trace", loss_trace), ("val_trace", val_trace)):
            if tr is not None and (tr.dtype != torch.float64 or not tr.is_cuda or tr.numel() < int(iters) + 1):
                raise ValueError(f"{name} must be a float64 CUDA tensor with iters + 1 entries")
        def addr(t):
            return None if t is None else t.data_ptr()

        ctl = FitControl(float(tol), addr(loss_trace), addr(val_mask), int(val_patience), addr(val_trace))
        done = ctypes.c_int(0)
        check(load().nef_fit_ctl(self._h, self._ptr(Y), self._ptr(mask), self._facs(factors),
                                 float(alpha), float(beta), int(iters), ctypes.byref(ctl),
                                 ctypes.byref(done) if sweeps else None))
        return int(done.value) if sweeps else None

    def sweeps(self) -> int:
        """Sweeps run by the last fit (nef_plan_sweeps)."""
        return int(load().nef_plan_sweeps(self._h))

    def autotune(self, Y, mask, factors, alpha, beta, cache=None):
        """Time candidate column splits of every fused pass (nef_plan_autotune);
        returns the chosen split per factor (-1: no fused kernel)."""
        self._check_args(Y, mask, factors)
        n = len(factors)
        out = (ctypes.c_int * n)()
        check(load().nef_plan_autotune(self._h, self._ptr(Y), self._ptr(mask), self._facs(factors),
                                       float(alpha), float(beta), None if cache is None else str(cache).encode(),
                                       out))
        return [int(v) for v in out]

    def update(self, l, Y, mask, factors, alpha, beta):
        self._check_args(Y, mask, factors)
        check(load().nef_update(self._h, int(l), self._ptr(Y), self._ptr(mask),
                                self._facs(factors), float(alpha), float(beta)))

    def numden(self, l, Y, mask, factors, alpha, beta):
        """num and den of Eq. 3.6-3.8 for factor l (nef_numden), as new CUDA tensors."""
        import torch
        self._check_args(Y, mask, factors)
        num = torch.empty_like(factors[l])
        den = torch.empty_like(factors[l])
        check(load().nef_numden(self._h, int(l), self._ptr(Y), self._ptr(mask), self._facs(factors),
                                float(alpha), float(beta), self._ptr(num), self._ptr(den)))
        return num, den

    def apply_update(self, l, factors, num, den, alpha, beta):
        """Eq. 3.4 for factor l from num and den (nef_apply_update)."""
        f = factors[l]
        for t in (num, den):
            if t.dtype != f.dtype or t.shape != f.shape or not t.is_cuda or not t.is_contiguous():
                raise ValueError("num and den must be contiguous CUDA tensors shaped like factor l")
        check(load().nef_apply_update(self._h, int(l), self._facs(factors), self._ptr(num), self._ptr(den),
                                      float(alpha), float(beta)))

    def loss(self, Y, mask, factors, alpha, beta):
        self._check_args(Y, mask, factors)
        out = (ctypes.c_double * 2)()
        check(load().nef_loss(self._h, self._ptr(Y), self._ptr(mask), self._facs(factors),
                              float(alpha), float(beta), out))
        return float(out[0]), int(out[1])

    def check(self):
        """Synchronise and raise if a kernel reported a bounded-wait timeout."""
        check(load().nef_check(self._h))

    def profile(self, reset: bool = True):
        """Summed device ms and launch counts of the fused passes since the last reset:
        {"tcgen05": (ms, n), "simt": (ms, n)}."""
        ms = (ctypes.c_double * 2)()
        cnt = (ctypes.c_int * 2)()
        check(load().nef_plan_profile(self._h, ms, cnt, int(bool(reset))))
        return {"tcgen05": (ms[0], cnt[0]), "simt": (ms[1], cnt[1])}

    def tc_trace(self, reset: bool = True):
        """Wait-cycle counters of the tensor-core pass (nef_tc_trace in include/nef.h)."""
        out = (ctypes.c_ulonglong * 32)()
        rc = load().nef_tc_trace(self._h, out, int(bool(reset)))
        if rc:
            raise NefError(rc, "tensor-core trace unavailable (plan needs profile=2)")
        return list(out)

    def info(self) -> str:
        n = load().nef_plan_info(self._h, None, 0)
        buf = ctypes.create_string_buffer(n)
        load().nef_plan_info(self._h, buf, n)
        return buf.value.decode()

    def launches(self, has_mask: bool) -> int:
        return int(load().nef_plan_launches(self._h, int(bool(has_mask))))


class FoldIn:
    """The fold-in encoder (nef_foldin_*): an MLP from a slice Y[i, :, :] to its
    loading row, trained and run by the library's kernels.  ``params`` is a
    float32 CUDA tensor holding W1, b1, W2, b2, W3, b3 packed (weights
    [fan_in x fan_out]); slices and targets are float32 CUDA tensors
    [n, d_in] and [n, d_out]."""

    def __init__(self, d_in: int, d_h: int, d_out: int, max_batch: int, params, stream=None):
        import torch
        lib = load()
        self.d_in, self.d_h, self.d_out, self.max_batch = int(d_in), int(d_h), int(d_out), int(max_batch)
        self.n_params = int(lib.nef_foldin_num_params(self.d_in, self.d_h, self.d_out))
        if params.dtype != torch.float32 or not params.is_cuda or params.numel() != self.n_params:
            raise ValueError(f"params must be a float32 CUDA tensor of {self.n_params} values")
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        check(lib.nef_foldin_create(self.d_in, self.d_h, self.d_out, self.max_batch,
                                    ctypes.c_void_p(params.contiguous().data_ptr()),
                                    ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream),
                                    ctypes.byref(h)))
        self._h = h

    @staticmethod
    def num_params(d_in: int, d_h: int, d_out: int) -> int:
        return int(load().nef_foldin_num_params(int(d_in), int(d_h), int(d_out)))

    def close(self):
        if getattr(self, "_h", None):
            load().nef_foldin_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, x, cols):
        import torch
        if x.dtype != torch.float32 or not x.is_cuda or x.dim() != 2 or x.shape[1] != cols or not x.is_contiguous():
            raise ValueError(f"expected a contiguous float32 CUDA tensor [n, {cols}]")

    def grad(self, slices, targets):
        """(packed gradient tensor, loss) at the current parameters, on `slices` or, when
        slices is None, on the batch kept by load_batch."""
        import torch
        if slices is not None:
            self._check(slices, self.d_in)
        self._check(targets, self.d_out)
        g = torch.empty(self.n_params, dtype=torch.float32, device=targets.device)
        loss = ctypes.c_double(0.0)
        check(load().nef_foldin_grad(self._h, ctypes.c_void_p(None if slices is None else slices.data_ptr()),
                                     ctypes.c_void_p(targets.data_ptr()), int(targets.shape[0]),
                                     ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)))
        return g, float(loss.value)

    def load_batch(self, slices):
        """nef_foldin_load_batch: keep the features of this batch for full-batch steps
        (train_step / grad with slices=None)."""
        self._check(slices, self.d_in)
        self._kept = int(slices.shape[0])
        check(load().nef_foldin_load_batch(self._h, ctypes.c_void_p(slices.data_ptr()), self._kept))

    def train_step(self, slices, targets, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=True):
        """One Adam step on `slices`, or on the batch kept by load_batch when slices is None."""
        if slices is not None:
            self._check(slices, self.d_in)
        self._check(targets, self.d_out)
        loss = ctypes.c_double(0.0)
        check(load().nef_foldin_train_step(self._h, ctypes.c_void_p(None if slices is None else slices.data_ptr()),
                                           ctypes.c_void_p(targets.data_ptr()), int(targets.shape[0]),
                                           float(lr), float(beta1), float(beta2), float(eps),
                                           ctypes.byref(loss) if want_loss else None))
        return float(loss.value) if want_loss else None

    def predict(self, slices):
        import torch
        self._check(slices, self.d_in)
        out = torch.empty(slices.shape[0], self.d_out, dtype=torch.float32, device=slices.device)
        check(load().nef_foldin_predict(self._h, ctypes.c_void_p(slices.data_ptr()), int(slices.shape[0]),
                                        ctypes.c_void_p(out.data_ptr())))
        return out

    def params(self):
        import torch
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        check(load().nef_foldin_params(self._h, ctypes.c_void_p(out.data_ptr())))
        return out


def pack_params(arrays):
    """Concatenate W1, b1, W2, b2, W3, b3 (numpy arrays) into one float32 vector."""
    import numpy as np
    return np.concatenate([np.asarray(a, np.float32).reshape(-1) for a in arrays])
