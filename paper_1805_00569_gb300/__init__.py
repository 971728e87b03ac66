"""Python binding of libkrr, the sm_103a implementation of the partitioned
kernel ridge regression hot path (DKRR, BKRR2, KKRR2).

Thin marshalling over the C ABI of ``include/krr.h``: every function here has
the name of the C entry point it calls, takes torch CUDA tensors, allocates the
output tensors the C call fills, and raises ``KrrError`` on a non-OK status.
All arithmetic runs in the CUDA kernels of the shared library; there is no
host or CPU fallback: importing this package without the built library, or
calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

KRR_OK, KRR_ERR_ARG, KRR_ERR_OOM, KRR_ERR_BUDGET, KRR_ERR_CUDA = 0, 1, 2, 3, 4
KRR_ERR_NOT_SPD, KRR_ERR_NO_CONVERGE, KRR_ERR_TIMEOUT, KRR_ERR_UNSUPPORTED = 5, 6, 7, 8
KRR_PART_RANDOM, KRR_PART_KMEANS, KRR_PART_KBALANCE = 0, 1, 2
KRR_KERNEL_GAUSSIAN, KRR_KERNEL_LINEAR = 0, 1
KRR_PREC_FP64, KRR_PREC_FP32, KRR_PREC_TF32, KRR_PREC_BF16X3 = 0, 1, 2, 3
KRR_SEL_PER_MODEL, KRR_SEL_ROUTED, KRR_SEL_AVERAGE, KRR_SEL_ORACLE = 0, 1, 2, 3
PREC_NAMES = {"fp64": KRR_PREC_FP64, "fp32": KRR_PREC_FP32, "tf32": KRR_PREC_TF32, "bf16x3": KRR_PREC_BF16X3}
STATUS_NAMES = {0: "OK", 1: "ARG", 2: "OOM", 3: "BUDGET", 4: "CUDA", 5: "NOT_SPD", 6: "NO_CONVERGE",
                7: "TIMEOUT", 8: "UNSUPPORTED"}
# kernel classes timed by krr_ctx_profile
PROF_KINDS = ["partition", "stage", "kbuild", "potrf", "trsm", "update", "matvec", "precond", "pcgvec",
              "predict", "select"]

_lib = None


class KrrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%s)" % (msg, STATUS_NAMES.get(status, status)))
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkrr.so, building it first if it is missing or stale."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.stale():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libkrr.so is not built; run paper_1805_00569_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P, i32, i64, u64, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                 ctypes.c_double, ctypes.c_size_t)
    st = ctypes.c_int
    L.krr_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, sz]
    L.krr_ctx_destroy.argtypes = [P]
    L.krr_last_error.argtypes = [P]
    L.krr_last_error.restype = ctypes.c_char_p
    L.krr_ctx_bytes_in_use.argtypes = [P]
    L.krr_ctx_bytes_in_use.restype = sz
    L.krr_ctx_set_profiling.argtypes = [P, ctypes.c_int]
    L.krr_ctx_profile.argtypes = [P, ctypes.c_int, ctypes.POINTER(f64), ctypes.POINTER(ctypes.c_longlong)]
    L.krr_ctx_set_panel_width.argtypes = [P, ctypes.c_int]
    L.krr_ctx_get_panel_width.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.krr_ctx_set_target_error.argtypes = [P, ctypes.c_double]
    L.krr_ctx_set_escalation.argtypes = [P, ctypes.c_double]
    L.krr_ctx_wait_probe.argtypes = [P, ctypes.c_double]
    L.krr_ctx_set_fp64_fallback.argtypes = [P, ctypes.c_int]
    L.krr_launch_count.restype = ctypes.c_longlong
    L.krr_partition.argtypes = [P, P, i64, i32, P, i64, ctypes.c_int, i32, i32, u64, P, P, P, P, P, P]
    L.krr_fit_batch.argtypes = [P, P, P, i64, i32, P, P, i32, P, i32, P, i32, ctypes.c_int,
                                ctypes.POINTER(P), P, P]
    L.krr_fit_jobs.argtypes = [P, P, P, i64, i32, P, P, i32, P, P, ctypes.c_int, ctypes.POINTER(P), P, P]
    L.krr_predict.argtypes = [P, P, P, i64, P, P]
    L.krr_select.argtypes = [P, P, P, i64, i32, i32, ctypes.c_int, P, P]
    L.krr_model_stats.argtypes = [P, P, P, P, P]
    L.krr_model_free.argtypes = [P, P]
    L.krr_model_factor_class.argtypes = [P, P, P]
    L.krr_group_rows.argtypes = [P, P, i64, i32, P, P]
    L.krr_kmeans_assign.argtypes = [P, P, i64, i32, P, i32, P]
    L.krr_kmeans_block_sums.argtypes = [P, P, i64, i32, P, i32, P, P]
    L.krr_kmeans_combine.argtypes = [P, P, P, i64, i32, i32, P]
    for name in ("krr_ctx_create", "krr_ctx_destroy", "krr_ctx_set_profiling", "krr_ctx_profile",
                 "krr_ctx_set_panel_width", "krr_ctx_get_panel_width", "krr_ctx_set_target_error",
                 "krr_ctx_set_escalation", "krr_ctx_wait_probe", "krr_ctx_set_fp64_fallback", "krr_partition", "krr_fit_batch", "krr_fit_jobs", "krr_predict", "krr_select",
                 "krr_model_stats", "krr_model_free", "krr_model_factor_class", "krr_group_rows", "krr_kmeans_assign",
                 "krr_kmeans_block_sums", "krr_kmeans_combine"):
        getattr(L, name).restype = st
    _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    return t.contiguous()


class Context:
    """A libkrr context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, hbm_budget_bytes: int = 0):
        if not torch.cuda.is_available():
            raise KrrError(KRR_ERR_CUDA, "libkrr needs a CUDA device")
        self.lib = load()
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        rc = self.lib.krr_ctx_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream),
                                     hbm_budget_bytes)
        if rc != KRR_OK:
            raise KrrError(rc, "krr_ctx_create failed")
        self.handle = h

    def check(self, rc: int, what: str):
        if rc != KRR_OK:
            raise KrrError(rc, "%s: %s" % (what, self.lib.krr_last_error(self.handle).decode()))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.krr_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bytes_in_use(self) -> int:
        return int(self.lib.krr_ctx_bytes_in_use(self.handle))


class Model:
    def __init__(self, ctx: Context, handle, p: int, ns: int, nl: int):
        self.ctx, self.handle, self.p, self.ns, self.nl = ctx, handle, p, ns, nl

    @property
    def G(self):
        return self.ns * self.nl

    def free(self):
        if self.handle:
            krr_model_free(self.ctx, self)


# ---------------------------------------------------------------- entry points
def krr_ctx_create(device: int = 0, stream=None, hbm_budget_bytes: int = 0) -> Context:
    return Context(device, stream, hbm_budget_bytes)


def krr_ctx_destroy(ctx: Context):
    ctx.close()


def krr_ctx_set_profiling(ctx: Context, on: bool):
    ctx.check(ctx.lib.krr_ctx_set_profiling(ctx.handle, 1 if on else 0), "krr_ctx_set_profiling")


def krr_ctx_profile(ctx: Context) -> dict:
    out = {}
    for k, name in enumerate(PROF_KINDS):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        ctx.check(ctx.lib.krr_ctx_profile(ctx.handle, k, ctypes.byref(ms), ctypes.byref(n)), "krr_ctx_profile")
        out[name] = (ms.value, n.value)
    return out


def krr_ctx_set_kernel(ctx: Context, kind: int):
    ctx.check(ctx.lib.krr_ctx_set_kernel(ctx.handle, int(kind)), "krr_ctx_set_kernel")


def krr_ctx_set_panel_width(ctx: Context, W: int):
    ctx.check(ctx.lib.krr_ctx_set_panel_width(ctx.handle, int(W)), "krr_ctx_set_panel_width")


def krr_ctx_set_target_error(ctx: Context, rel: float):
    ctx.check(ctx.lib.krr_ctx_set_target_error(ctx.handle, float(rel)), "krr_ctx_set_target_error")


def krr_ctx_set_escalation(ctx: Context, kappa_u: float):
    ctx.check(ctx.lib.krr_ctx_set_escalation(ctx.handle, float(kappa_u)), "krr_ctx_set_escalation")


def krr_ctx_set_fp64_fallback(ctx: Context, on: bool):
    ctx.check(ctx.lib.krr_ctx_set_fp64_fallback(ctx.handle, 1 if on else 0), "krr_ctx_set_fp64_fallback")


def krr_ctx_wait_probe(ctx: Context, seconds: float) -> int:
    """Runs the bounded-wait self-check; returns its status (KRR_ERR_TIMEOUT
    when the wait expired as designed and the context stays usable)."""
    return int(ctx.lib.krr_ctx_wait_probe(ctx.handle, float(seconds)))


def krr_partition(ctx: Context, X: torch.Tensor, Xt: torch.Tensor | None, mode: int, p: int, iters: int = 0,
                  seed: int = 0, init_idx: torch.Tensor | None = None):
    """Returns (assign, route, perm, offsets, centers) as device tensors."""
    X = _dev(X, torch.float64, "X")
    n, d = X.shape
    dev = X.device
    t = 0 if Xt is None else Xt.shape[0]
    if Xt is not None:
        Xt = _dev(Xt, torch.float64, "Xt")
    assign = torch.empty(n, dtype=torch.int32, device=dev)
    route = torch.empty(t, dtype=torch.int32, device=dev) if t > 0 else None
    perm = torch.empty(n, dtype=torch.int64, device=dev)
    offsets = torch.empty(p + 1, dtype=torch.int64, device=dev)
    centers = (torch.empty((p, d), dtype=torch.float64, device=dev)
               if mode in (KRR_PART_KMEANS, KRR_PART_KBALANCE) else None)
    if init_idx is not None:
        init_idx = _dev(init_idx, torch.int64, "init_idx")
    rc = ctx.lib.krr_partition(ctx.handle, _ptr(X), n, d, _ptr(Xt), t, mode, p, iters,
                               ctypes.c_uint64(int(seed) & (2**64 - 1)), _ptr(init_idx), _ptr(assign), _ptr(route),
                               _ptr(perm), _ptr(offsets), _ptr(centers))
    ctx.check(rc, "krr_partition")
    return assign, route, perm, offsets, centers


def krr_fit_batch(ctx: Context, X, y, perm, offsets, sigmas, lambdas, prec=KRR_PREC_TF32, want_alpha=False):
    """Returns (Model, solve_status[p*G] int32 device tensor, alpha or None)."""
    X = _dev(X, torch.float64, "X")
    y = _dev(y, torch.float64, "y")
    perm = _dev(perm, torch.int64, "perm")
    offsets = _dev(offsets, torch.int64, "offsets")
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    n, d = X.shape
    p = offsets.shape[0] - 1
    sig = (ctypes.c_double * len(sigmas))(*[float(s) for s in sigmas])
    lam = (ctypes.c_double * len(lambdas))(*[float(v) for v in lambdas])
    G = len(sigmas) * len(lambdas)
    status = torch.empty(p * G, dtype=torch.int32, device=X.device)
    alpha = torch.empty(perm.shape[0] * G, dtype=torch.float64, device=X.device) if want_alpha else None
    h = ctypes.c_void_p()
    rc = ctx.lib.krr_fit_batch(ctx.handle, _ptr(X), _ptr(y), n, d, _ptr(perm), _ptr(offsets), p, sig, len(sigmas),
                               lam, len(lambdas), int(prec), ctypes.byref(h), _ptr(status), _ptr(alpha))
    ctx.check(rc, "krr_fit_batch")
    return Model(ctx, h, p, len(sigmas), len(lambdas)), status, alpha


def krr_fit_jobs(ctx: Context, X, y, perm, offsets, sigmas, lambdas, prec=KRR_PREC_TF32, want_alpha=False):
    """One independent problem per partition with its own sigma and lambda.
    Returns (Model with p models, solve_status[p], alpha or None)."""
    X = _dev(X, torch.float64, "X")
    y = _dev(y, torch.float64, "y")
    perm = _dev(perm, torch.int64, "perm")
    offsets = _dev(offsets, torch.int64, "offsets")
    if isinstance(prec, str):
        prec = PREC_NAMES[prec]
    n, d = X.shape
    p = offsets.shape[0] - 1
    if len(sigmas) != p or len(lambdas) != p:
        raise KrrError(KRR_ERR_ARG, "krr_fit_jobs: one sigma and one lambda per partition")
    sig = (ctypes.c_double * p)(*[float(s) for s in sigmas])
    lam = (ctypes.c_double * p)(*[float(v) for v in lambdas])
    status = torch.empty(p, dtype=torch.int32, device=X.device)
    alpha = torch.empty(perm.shape[0], dtype=torch.float64, device=X.device) if want_alpha else None
    h = ctypes.c_void_p()
    rc = ctx.lib.krr_fit_jobs(ctx.handle, _ptr(X), _ptr(y), n, d, _ptr(perm), _ptr(offsets), p, sig, lam, int(prec),
                              ctypes.byref(h), _ptr(status), _ptr(alpha))
    ctx.check(rc, "krr_fit_jobs")
    return Model(ctx, h, p, 1, 1), status, alpha


def krr_predict(ctx: Context, model: Model, Xt, route=None, out=None):
    """All-models yhat [p*G, t] (route None) or routed yhat [G, t]."""
    Xt = _dev(Xt, torch.float64, "Xt")
    t = Xt.shape[0]
    rows = model.G if route is not None else model.p * model.G
    if route is not None:
        route = _dev(route, torch.int32, "route")
    yhat = out if out is not None else torch.empty((rows, t), dtype=torch.float64, device=Xt.device)
    rc = ctx.lib.krr_predict(ctx.handle, model.handle, _ptr(Xt), t, _ptr(route), _ptr(yhat))
    ctx.check(rc, "krr_predict")
    return yhat


def krr_select(ctx: Context, yhat, yt, p: int, G: int, mode: int):
    """Returns (mse device tensor, best device int32 tensor of one element)."""
    yhat = _dev(yhat, torch.float64, "yhat")
    yt = _dev(yt, torch.float64, "yt")
    rows = p * G if mode == KRR_SEL_PER_MODEL else G
    mse = torch.empty(rows, dtype=torch.float64, device=yt.device)
    best = torch.empty(1, dtype=torch.int32, device=yt.device)
    rc = ctx.lib.krr_select(ctx.handle, _ptr(yhat), _ptr(yt), yt.shape[0], p, G, mode, _ptr(mse), _ptr(best))
    ctx.check(rc, "krr_select")
    return mse, best


def krr_model_stats(ctx: Context, model: Model):
    """Returns (iterations, condition estimates, scaled residuals) as host tensors."""
    n = model.p * model.G
    it = torch.zeros(n, dtype=torch.int32)
    ka = torch.zeros(n, dtype=torch.float64)
    rs = torch.zeros(n, dtype=torch.float64)
    rc = ctx.lib.krr_model_stats(ctx.handle, model.handle, ctypes.c_void_p(it.data_ptr()),
                                 ctypes.c_void_p(ka.data_ptr()), ctypes.c_void_p(rs.data_ptr()))
    ctx.check(rc, "krr_model_stats")
    return it, ka, rs


def krr_group_rows(ctx: Context, assign, p: int):
    """Rows grouped by partition: (perm int64 [n], offsets int64 [p+1]) device tensors."""
    assign = _dev(assign, torch.int32, "assign")
    n = assign.shape[0]
    perm = torch.empty(n, dtype=torch.int64, device=assign.device)
    offsets = torch.empty(p + 1, dtype=torch.int64, device=assign.device)
    ctx.check(ctx.lib.krr_group_rows(ctx.handle, _ptr(assign), n, p, _ptr(perm), _ptr(offsets)), "krr_group_rows")
    return perm, offsets


def krr_kmeans_assign(ctx: Context, X, C):
    """Alg. 2 assignment step of the rows of X to the centres C (int32 device tensor)."""
    X = _dev(X, torch.float64, "X")
    C = _dev(C, torch.float64, "C")
    out = torch.empty(X.shape[0], dtype=torch.int32, device=X.device)
    ctx.check(ctx.lib.krr_kmeans_assign(ctx.handle, _ptr(X), X.shape[0], X.shape[1], _ptr(C), C.shape[0], _ptr(out)),
              "krr_kmeans_assign")
    return out


def krr_kmeans_block_sums(ctx: Context, X, assign, k: int):
    """Per 1024-row block: centre member sums [nblk, k, d] and counts [nblk, k]."""
    X = _dev(X, torch.float64, "X")
    assign = _dev(assign, torch.int32, "assign")
    n, d = X.shape
    nblk = -(-n // 1024)
    sums = torch.empty((nblk, k, d), dtype=torch.float64, device=X.device)
    counts = torch.empty((nblk, k), dtype=torch.int64, device=X.device)
    ctx.check(ctx.lib.krr_kmeans_block_sums(ctx.handle, _ptr(X), n, d, _ptr(assign), k, _ptr(sums), _ptr(counts)),
              "krr_kmeans_block_sums")
    return sums, counts


def krr_kmeans_combine(ctx: Context, sums, counts, C):
    """Centres from the block sums of all blocks (canonical tree); returns a new tensor."""
    sums = _dev(sums, torch.float64, "sums")
    counts = _dev(counts, torch.int64, "counts")
    out = _dev(C, torch.float64, "C").clone()
    nblk, k, d = sums.shape
    ctx.check(ctx.lib.krr_kmeans_combine(ctx.handle, _ptr(sums), _ptr(counts), nblk, k, d, _ptr(out)),
              "krr_kmeans_combine")
    return out


def krr_model_factor_class(ctx: Context, model: Model):
    """Factor class of every solve (host int32 tensor; see include/krr.h)."""
    cls = torch.zeros(model.p * model.G, dtype=torch.int32)
    ctx.check(ctx.lib.krr_model_factor_class(ctx.handle, model.handle, ctypes.c_void_p(cls.data_ptr())),
              "krr_model_factor_class")
    return cls


def krr_model_free(ctx: Context, model: Model):
    rc = ctx.lib.krr_model_free(ctx.handle, model.handle)
    model.handle = None
    ctx.check(rc, "krr_model_free")
